"""CUDA path vs the CPU oracle, element by element (bit-exact).

Every stage of the method (arXiv 1703.02563, Sec. 3) is compared on the same
seeded inputs: level features, the seeding search, the state after each
sweep of each level, the final flows and costs, and the consistency mask.
All calls go through the C ABI (``paper_1703_02563_gb300.ff``).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1703_02563_gb300 import ff, workloads

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _ctx(C, S, I, W, H, R=8, leaf=8, stride=1, eps=8, seed=20261203):
    cfg = ff.Config(channels=C, scales=S, iters=I, radius_q3=R, seed_leaf=leaf,
                    seed_stride=stride, eps_q3=eps, seed=seed, max_width=W, max_height=H)
    return ff.Context(cfg)


def _params(C, S, I, R=8, leaf=8, stride=1, seed=20261203):
    return O.Params(channels=C, scales=S, iters=I, radius_q3=R, seed_leaf=leaf,
                    seed_stride=stride, seed=seed)


def _dev(a):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    _torch().cuda.synchronize()
    return t.cpu().numpy()


def _load(ctx, pair):
    ctx.features(0, _dev(pair.img1))
    ctx.features(1, _dev(pair.img2))


def _gt_seeds(pair, S):
    N = 1 << (S - 1)
    WS, HS = O.level_dims(pair.width, pair.height, S - 1)
    gt = np.rint(pair.flow * 8).astype(np.int16)
    return np.ascontiguousarray(gt[::N, ::N][:HS, :WS])


FEATURE_CASES = [(1, 128, 96, 3), (1, 37, 29, 4), (3, 97, 71, 3), (3, 16, 9, 2), (1, 1, 1, 1),
                 (1, 200, 3, 3), (3, 65, 130, 4),
                 # one launch covers every level: up to the eight the ABI allows, down
                 # to levels 2 px across
                 (3, 300, 170, 8), (1, 513, 257, 6), (3, 37, 300, 7)]


@pytest.mark.parametrize("C,W,H,S", FEATURE_CASES)
def test_features_bit_exact(C, W, H, S):
    pair = workloads.random_pair(seed=W * 7 + H, width=W, height=H, channels=C)
    ctx = _ctx(C, S, 1, W, H)
    _load(ctx, pair)
    for slot, img in ((0, pair.img1), (1, pair.img2)):
        ref = O.features_all(img, S)
        for L in range(S):
            np.testing.assert_array_equal(_host(ctx.features_of(slot, L)), ref[L])
    ctx.close()


@pytest.mark.parametrize("tc", [1, 0])
@pytest.mark.parametrize("C,W,H,S,stride", [(1, 128, 96, 3, 1), (3, 97, 71, 3, 2),
                                            (1, 45, 33, 2, 1), (3, 20, 12, 1, 3),
                                            (3, 200, 120, 3, 1), (1, 301, 77, 2, 1),
                                            (3, 320, 240, 4, 1)])
def test_seed_knn_bit_exact(C, W, H, S, stride, tc):
    if C == 1:
        pair = workloads.translation_pair(seed=W, width=W, height=H) if W >= 64 else \
            workloads.random_pair(seed=W, width=W, height=H, channels=1)
    else:
        pair = workloads.layered_pair(seed=W, width=W, height=H, channels=3, max_disp=12)
    ctx = _ctx(C, S, 1, W, H, stride=stride)
    ff.ff_debug_set(ctx.ctx, ff.FF_DEBUG_SEED_TC, tc)
    _load(ctx, pair)
    f1 = O.features_all(pair.img1, S)
    f2 = O.features_all(pair.img2, S)
    for d, (a, b) in enumerate(((f1, f2), (f2, f1))):
        idx, dist = ctx.seed_knn(d)
        ridx, rdist = O.seed_knn(a[0], b[0], S, 8, stride)
        np.testing.assert_array_equal(_host(idx), ridx)
        np.testing.assert_array_equal(_host(dist), rdist)
    ctx.close()


def test_every_stage_bit_exact_tiny():
    pair, prm = workloads.make_workload("tiny128x96")
    S, I = prm["scales"], prm["iters"]
    ctx = _ctx(1, S, I, pair.width, pair.height)
    _load(ctx, pair)
    P = _params(1, S, I)
    for d, (a, b) in enumerate(((pair.img1, pair.img2), (pair.img2, pair.img1))):
        for L in range(S - 1, -1, -1):
            for k in range(I + 1):
                flow, cost = ctx.match(d, 3, until_level=L, until_sweeps=k)
                rf, rc, _ = O.match(P, a, b, d, 3, until_level=L, until_sweeps=k)
                np.testing.assert_array_equal(_host(flow), rf, err_msg=f"dir {d} L {L} k {k}")
                np.testing.assert_array_equal(_host(cost), rc, err_msg=f"dir {d} L {L} k {k}")
    ctx.close()


def test_every_stage_bit_exact_lab_multistrip():
    # 16-row strips on every level: 5, 3 and 2 strips; 5 sweeps visit all four
    # directions and wrap to the first
    pair = workloads.layered_pair(seed=9, width=97, height=71, channels=3, max_disp=15)
    S, I = 3, 5
    ctx = _ctx(3, S, I, pair.width, pair.height, R=12)
    _load(ctx, pair)
    P = _params(3, S, I, R=12)
    for L in range(S - 1, -1, -1):
        for k in range(I + 1):
            flow, cost = ctx.match(0, 11, until_level=L, until_sweeps=k)
            rf, rc, _ = O.match(P, pair.img1, pair.img2, 0, 11, until_level=L, until_sweeps=k)
            np.testing.assert_array_equal(_host(flow), rf, err_msg=f"L {L} k {k}")
            np.testing.assert_array_equal(_host(cost), rc, err_msg=f"L {L} k {k}")
    ctx.close()


@pytest.mark.parametrize("lanes", [4, 2, 8])
@pytest.mark.parametrize("C", [1, 3])
def test_sweep_lane_layouts_bit_exact(C, lanes):
    # both lane layouts of the sweep kernel give the oracle's result
    if C == 1:
        pair = workloads.translation_pair(seed=31, width=150, height=77)
    else:
        pair = workloads.layered_pair(seed=31, width=101, height=67, channels=3, max_disp=18)
    S, I = 3, 5
    ctx = _ctx(C, S, I, pair.width, pair.height)
    ff.ff_debug_set(ctx.ctx, ff.FF_DEBUG_SWEEP_LANES, lanes)
    _load(ctx, pair)
    P = _params(C, S, I)
    for d, (a, b) in enumerate(((pair.img1, pair.img2), (pair.img2, pair.img1))):
        flow, cost = ctx.match(d, 4)
        rf, rc, _ = O.match(P, a, b, d, 4)
        np.testing.assert_array_equal(_host(flow), rf)
        np.testing.assert_array_equal(_host(cost), rc)
    ctx.close()


FULL_CASES = [
    ("tiny", lambda: workloads.make_workload("tiny128x96")[0], 1, 3, 4, 8),
    ("lab97x71", lambda: workloads.layered_pair(seed=4, width=97, height=71, channels=3,
                                                max_disp=20), 3, 3, 5, 8),
    ("gray150x50", lambda: workloads.translation_pair(seed=3, width=150, height=50), 1, 2, 6, 12),
    ("gray33x17", lambda: workloads.random_pair(seed=5, width=33, height=17), 1, 2, 3, 8),
    ("gray5x1", lambda: workloads.random_pair(seed=6, width=5, height=1), 1, 2, 4, 8),
    ("gray1x7", lambda: workloads.random_pair(seed=7, width=1, height=7), 1, 1, 2, 8),
    ("gray1x1", lambda: workloads.random_pair(seed=8, width=1, height=1), 1, 1, 2, 8),
    ("lab2x3", lambda: workloads.random_pair(seed=9, width=2, height=3, channels=3), 3, 2, 3, 8),
    # the largest frame side the library takes (4096), as a thin strip
    ("gray4096x9", lambda: workloads.random_pair(seed=10, width=4096, height=9), 1, 2, 2, 8),
    ("lab5x4096", lambda: workloads.random_pair(seed=11, width=5, height=4096, channels=3), 3, 2,
     2, 8),
]


@pytest.mark.parametrize("name,make,C,S,I,R", FULL_CASES, ids=[c[0] for c in FULL_CASES])
def test_match_and_filter_bit_exact(name, make, C, S, I, R):
    pair = make()
    ctx = _ctx(C, S, I, pair.width, pair.height, R=R)
    _load(ctx, pair)
    P = _params(C, S, I, R=R)
    fwd, cf = ctx.match(0, 17)
    bwd, cb = ctx.match(1, 17)
    mask = ctx.filter(fwd, bwd)
    rf, rcf, _ = O.match(P, pair.img1, pair.img2, 0, 17)
    rb, rcb, _ = O.match(P, pair.img2, pair.img1, 1, 17)
    np.testing.assert_array_equal(_host(fwd), rf)
    np.testing.assert_array_equal(_host(cf), rcf)
    np.testing.assert_array_equal(_host(bwd), rb)
    np.testing.assert_array_equal(_host(cb), rcb)
    np.testing.assert_array_equal(_host(mask), O.filter_mask(rf, rb, 8))
    ctx.sync()
    ctx.close()


@pytest.mark.parametrize("C", [1, 3])
def test_seeds_in_bit_exact(C):
    if C == 1:
        pair = workloads.translation_pair(seed=12)
    else:
        pair = workloads.layered_pair(seed=12, width=120, height=80, channels=3, max_disp=25)
    S, I = 3, 4
    seeds = _gt_seeds(pair, S)
    seeds[0, 0] = (ff.INVALID, ff.INVALID)          # unset seeds stay unset
    seeds[1, 2] = (30000, -30000)                    # far outside: clamped
    ctx = _ctx(C, S, I, pair.width, pair.height)
    _load(ctx, pair)
    P = _params(C, S, I)
    flow, cost = ctx.match(0, 2, seeds_in=_dev(seeds))
    rf, rc, _ = O.match(P, pair.img1, pair.img2, 0, 2, seeds_in=seeds)
    np.testing.assert_array_equal(_host(flow), rf)
    np.testing.assert_array_equal(_host(cost), rc)
    ctx.close()


def test_filter_bit_exact_on_arbitrary_flows():
    rng = np.random.default_rng(3)
    W, H = 61, 47
    pair = workloads.random_pair(seed=1, width=W, height=H)
    ctx = _ctx(1, 1, 1, W, H, eps=13)
    _load(ctx, pair)
    fwd = rng.integers(-80, 80, (H, W, 2)).astype(np.int16)
    bwd = rng.integers(-80, 80, (H, W, 2)).astype(np.int16)
    fwd[3, 4] = (ff.INVALID, ff.INVALID)
    bwd[10:20, 10:20] = -fwd[10:20, 10:20]
    mask = ctx.filter(_dev(fwd), _dev(bwd))
    np.testing.assert_array_equal(_host(mask), O.filter_mask(fwd, bwd, 13))
    ctx.close()


@pytest.mark.parametrize("name", ["sintel1024x436", "kitti1242x375"])
def test_full_size_workloads(name):
    """Full-size frames in the benchmark's launch configuration.

    Propagation, random search and upsampling are checked element by element
    on every pixel from seeds derived from the generator's ground truth; the
    seeding search is checked on sampled queries against brute force over
    all candidates.
    """
    pair, prm = workloads.make_workload(name)
    C, S, I, R = prm["channels"], prm["scales"], prm["iters"], prm["radius_q3"]
    W, H = pair.width, pair.height
    ctx = _ctx(C, S, I, W, H, R=R)
    _load(ctx, pair)
    f1 = O.features_all(pair.img1, S)
    f2 = O.features_all(pair.img2, S)
    for L in range(S):
        np.testing.assert_array_equal(_host(ctx.features_of(0, L)), f1[L])
    seeds = _gt_seeds(pair, S)
    flow, cost = ctx.match(0, 1, seeds_in=_dev(seeds))
    P = _params(C, S, I, R=R)
    rf, rc, _ = O.match_features(P, f1, f2, W, H, 0, 1, seeds_in=seeds)
    np.testing.assert_array_equal(_host(flow), rf)
    np.testing.assert_array_equal(_host(cost), rc)
    # seeding: sampled queries vs brute force
    idx, dist = ctx.seed_knn(0)
    idx, dist = _host(idx), _host(dist)
    N = 1 << (S - 1)
    cand = f2[0].reshape(-1, 9 * C).astype(np.int64)
    rng = np.random.default_rng(0)
    HS, WS = idx.shape[:2]
    for _ in range(24):
        gy, gx = int(rng.integers(0, HS)), int(rng.integers(0, WS))
        q = f1[0][gy * N, gx * N].astype(np.int64)
        d = ((cand - q) ** 2).sum(axis=1)
        order = np.lexsort((np.arange(d.size), d))[:8]
        np.testing.assert_array_equal(idx[gy, gx], order)
        np.testing.assert_array_equal(dist[gy, gx], d[order])
    ctx.close()


@pytest.mark.parametrize("name", ["sintel1024x436", "kitti1242x375"])
def test_full_size_end_to_end(name):
    """The benchmark's step at full size, compared element by element.

    Features of both frames, the seeding search (the bound pass and the
    tcgen05 full pass) and its Eq. 1 rerank, every level's sweeps and
    searches, both directions on two streams as the benchmark launches them,
    and the consistency mask.  The oracle's seeding lists are computed row
    band by row band on a thread pool; the rerank and everything after it run
    in the oracle itself.
    """
    from concurrent.futures import ThreadPoolExecutor
    torch = _torch()
    pair, prm = workloads.make_workload(name)
    C, S, I, R = prm["channels"], prm["scales"], prm["iters"], prm["radius_q3"]
    W, H = pair.width, pair.height
    ctx = _ctx(C, S, I, W, H, R=R)
    main, side = torch.cuda.Stream(), torch.cuda.Stream()
    img1, img2 = _dev(pair.img1), _dev(pair.img2)
    fwd = torch.empty((H, W, 2), dtype=torch.int16, device="cuda")
    bwd = torch.empty_like(fwd)
    cf = torch.empty((H, W), dtype=torch.int32, device="cuda")
    cb = torch.empty_like(cf)
    mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    ff.ff_set_stream(ctx.ctx, main)
    ctx.features(0, img1)
    ctx.features(1, img2)
    ev = torch.cuda.Event()
    ev.record(main)
    side.wait_event(ev)
    ff.ff_set_stream(ctx.ctx, side)
    ff.ff_match(ctx.ctx, ff.FF_BWD, 3, None, bwd, cb)
    ff.ff_set_stream(ctx.ctx, main)
    ff.ff_match(ctx.ctx, ff.FF_FWD, 3, None, fwd, cf)
    ev2 = torch.cuda.Event()
    ev2.record(side)
    main.wait_event(ev2)
    ff.ff_filter(ctx.ctx, fwd, bwd, mask)
    torch.cuda.synchronize()
    ctx.sync()
    f1 = O.features_all(pair.img1, S)
    f2 = O.features_all(pair.img2, S)
    for L in range(S):
        np.testing.assert_array_equal(_host(ctx.features_of(0, L)), f1[L])
        np.testing.assert_array_equal(_host(ctx.features_of(1, L)), f2[L])
    P = _params(C, S, I, R=R)
    refs = []
    for d, (a, b) in enumerate(((f1, f2), (f2, f1))):
        ki, kd = O.seed_knn_threaded(a[0], b[0], S, 8, 1)
        gi, gd = ctx.seed_knn(d)
        np.testing.assert_array_equal(_host(gi), ki)
        np.testing.assert_array_equal(_host(gd), kd)
        refs.append((a, b, d, ki))
    with ThreadPoolExecutor(max_workers=2) as ex:
        outs = list(ex.map(lambda r: O.match_features_knn(P, r[0], r[1], W, H, r[2], 3, r[3]),
                           refs))
    (rf, rcf, _), (rb, rcb, _) = outs
    np.testing.assert_array_equal(_host(fwd), rf)
    np.testing.assert_array_equal(_host(cf), rcf)
    np.testing.assert_array_equal(_host(bwd), rb)
    np.testing.assert_array_equal(_host(cb), rcb)
    np.testing.assert_array_equal(_host(mask), O.filter_mask(rf, rb, 8))
    ctx.close()


def test_profile_modes_record_the_same_sweeps():
    # per-launch timing and per-run timing of the sweeps count the same sweep
    # launches; the run mode records nothing else; flows are unchanged by either
    pair, prm = workloads.make_workload("tiny128x96")
    S, I = prm["scales"], prm["iters"]
    ctx = _ctx(1, S, I, pair.width, pair.height)
    _load(ctx, pair)
    ref = _host(ctx.match(ff.FF_FWD, 5)[0])
    got = {}
    for mode in (ff.FF_PROFILE_LAUNCHES, ff.FF_PROFILE_SWEEP_RUNS):
        ff.ff_profile(ctx.ctx, mode)
        f = ctx.match(ff.FF_FWD, 5)[0]
        ctx.match(ff.FF_BWD, 5)
        ctx.sync()
        ff.ff_profile(ctx.ctx, 0)
        np.testing.assert_array_equal(_host(f), ref)
        got[mode] = {k: ff.ff_kernel_stats(ctx.ctx, k) for k in ff.KERNELS}
    per_launch, runs = got[ff.FF_PROFILE_LAUNCHES], got[ff.FF_PROFILE_SWEEP_RUNS]
    sweeps = 2 * sum(ff.Config(channels=1, scales=S, iters=I).sweeps(L) for L in range(S))
    assert per_launch["k_sweep"][0] == runs["k_sweep"][0] == sweeps
    assert runs["k_sweep"][1] > 0 and per_launch["k_upsample"][0] > 0
    assert all(n == 0 for k, (n, _) in runs.items() if k != "k_sweep")
    with pytest.raises(ff.FFError):
        ff.ff_profile(ctx.ctx, 3)
    ctx.close()


def test_deterministic_and_concurrent_streams_agree():
    torch = _torch()
    pair = workloads.layered_pair(seed=21, width=160, height=120, channels=3, max_disp=30)
    S, I = 3, 4
    ctx = _ctx(3, S, I, pair.width, pair.height)
    _load(ctx, pair)
    f0, c0 = ctx.match(0, 5)
    b0, cb0 = ctx.match(1, 5)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    f1 = torch.empty_like(f0)
    b1 = torch.empty_like(b0)
    ff.ff_set_stream(ctx.ctx, s1)
    ff.ff_match(ctx.ctx, 0, 5, None, f1, None)
    ff.ff_set_stream(ctx.ctx, s2)
    ff.ff_match(ctx.ctx, 1, 5, None, b1, None)
    ff.ff_set_stream(ctx.ctx, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.equal(f0, f1) and torch.equal(b0, b1)
    ctx.sync()
    ctx.close()


def test_pair_host_matches_device_calls():
    torch = _torch()
    pair, prm = workloads.make_workload("tiny128x96")
    W, H = pair.width, pair.height
    ctx = _ctx(1, prm["scales"], prm["iters"], W, H)
    fwd = torch.empty((H, W, 2), dtype=torch.int16).pin_memory()
    bwd = torch.empty((H, W, 2), dtype=torch.int16).pin_memory()
    mask = torch.empty((H, W), dtype=torch.uint8).pin_memory()
    i1 = torch.from_numpy(pair.img1.copy()).pin_memory()
    i2 = torch.from_numpy(pair.img2.copy()).pin_memory()
    ff.ff_pair_host(ctx.ctx, i1, i2, W, H, 9, fwd, bwd, mask)
    P = _params(1, prm["scales"], prm["iters"])
    rf, _, _ = O.match(P, pair.img1, pair.img2, 0, 9)
    rb, _, _ = O.match(P, pair.img2, pair.img1, 1, 9)
    np.testing.assert_array_equal(fwd.numpy(), rf)
    np.testing.assert_array_equal(bwd.numpy(), rb)
    np.testing.assert_array_equal(mask.numpy(), O.filter_mask(rf, rb, 8))
    ctx.close()


def test_bounded_wait_reports_timeout_and_context_recovers():
    # a boundary row that is never written: the loader's bounded wait runs
    # out, the kernel returns, ff_sync reports FF_ETIMEOUT; the context then
    # computes correct results again
    pair, prm = workloads.make_workload("tiny128x96")
    S, I = prm["scales"], prm["iters"]
    ctx = _ctx(1, S, I, pair.width, pair.height)
    _load(ctx, pair)
    ff.ff_debug_set(ctx.ctx, ff.FF_DEBUG_WAIT_LIMIT_NS, 50_000_000)
    ff.ff_debug_set(ctx.ctx, ff.FF_DEBUG_FORCE_TIMEOUT, 1)
    ctx.match(0, 1)
    with pytest.raises(ff.FFError) as e:
        ctx.sync()
    assert e.value.status == ff.FF_ETIMEOUT
    ff.ff_debug_set(ctx.ctx, ff.FF_DEBUG_FORCE_TIMEOUT, 0)
    flow, cost = ctx.match(0, 1)
    ctx.sync()
    rf, rc, _ = O.match(_params(1, S, I), pair.img1, pair.img2, 0, 1)
    np.testing.assert_array_equal(_host(flow), rf)
    ctx.close()


def test_argument_errors_launch_nothing():
    ctx = _ctx(1, 2, 2, 64, 64)
    torch = _torch()
    img = torch.zeros((1, 65, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(ff.FFError) as e:
        ff.ff_features(ctx.ctx, 0, img, 64, 65, 64)
    assert e.value.status == ff.FF_EINVAL
    flow = torch.empty((64, 64, 2), dtype=torch.int16, device="cuda")
    with pytest.raises(ff.FFError) as e:
        ff.ff_match(ctx.ctx, 0, 0, None, flow, None)
    assert e.value.status == ff.FF_ESTATE
    n0 = ff.ff_launch_count(ctx.ctx)
    with pytest.raises(ff.FFError):
        ff.ff_features(ctx.ctx, 2, img, 64, 64, 64)
    assert ff.ff_launch_count(ctx.ctx) == n0
    ctx.close()
