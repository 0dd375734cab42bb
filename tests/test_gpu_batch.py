"""The batched form: many pairs of mixed sizes in flight at once.

Each pair's flows and masks must equal the oracle's (bit-exact) and the
single-context path's, whichever slot the pair lands in, whether the batch is
enqueued directly or captured as a CUDA graph and replayed.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1703_02563_gb300 import ff, workloads

pytestmark = pytest.mark.gpu

SMALL_SIZES = ((64, 48), (97, 71), (40, 33), (128, 96), (17, 90))


def _outputs(pairs, cfg, two_way):
    import torch
    Lf = cfg.final_level()
    outs = []
    for k, p in enumerate(pairs):
        WL, HL = O.level_dims(p.width, p.height, Lf)
        mk = lambda: torch.full((HL, WL, 2), 77, dtype=torch.int16, device="cuda")
        outs.append(dict(fwd=mk(), bwd=mk(), bwd2=mk() if two_way[k] else None,
                         mask=torch.full((HL, WL), 9, dtype=torch.uint8, device="cuda")))
    return outs


def _descs(pairs, imgs, outs):
    return [dict(img1=i1, img2=i2, w=p.width, h=p.height, pair_id=100 + k,
                 flow_fwd=o["fwd"], flow_bwd=o["bwd"], flow_bwd2=o["bwd2"], mask=o["mask"])
            for k, (p, (i1, i2), o) in enumerate(zip(pairs, imgs, outs))]


def _upload(pairs):
    import torch
    return [(torch.from_numpy(p.img1).cuda(), torch.from_numpy(p.img2).cuda()) for p in pairs]


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("schedule", [ff.FF_SCHED_BASIC, ff.FF_SCHED_PLUS_FAST_X2])
def test_batch_equals_oracle(schedule):
    pairs = [workloads.batch_pair(7, k, SMALL_SIZES) for k in range(7)]
    two_way = [k % 3 == 0 for k in range(7)]
    S, I = 3, 4
    stride = 2 if schedule == ff.FF_SCHED_PLUS_FAST_X2 else 1
    cfg = ff.Config(channels=3, scales=S, iters=I, radius_q3=8, max_width=128, max_height=96,
                    schedule=schedule, seed_stride=stride)
    b = ff.ff_batch_create(cfg, 0, slots=3)
    imgs = _upload(pairs)
    outs = _outputs(pairs, cfg, two_way)
    ff.ff_batch_run(b, _descs(pairs, imgs, outs))
    ff.ff_batch_sync(b)
    P = O.Params(channels=3, scales=S, iters=I, radius_q3=8, schedule=schedule, seed_stride=stride)
    Lf = P.final_level()
    for k, (p, o) in enumerate(zip(pairs, outs)):
        rf, _, _ = O.match(P, p.img1, p.img2, 0, 100 + k)
        rb, _, _ = O.match(P, p.img2, p.img1, 1, 100 + k)
        np.testing.assert_array_equal(_host(o["fwd"]), rf, err_msg=f"pair {k}")
        np.testing.assert_array_equal(_host(o["bwd"]), rb, err_msg=f"pair {k}")
        if two_way[k]:
            rb2, _, _ = O.match(P, p.img2, p.img1, 2, 100 + k)
            np.testing.assert_array_equal(_host(o["bwd2"]), rb2, err_msg=f"pair {k}")
            ref_mask = O.filter_mask2(rf, rb, rb2, 8, level=Lf)
        else:
            ref_mask = O.filter_mask(rf, rb, 8, level=Lf)
        np.testing.assert_array_equal(_host(o["mask"]), ref_mask, err_msg=f"pair {k}")
    ff.ff_batch_destroy(b)


def test_batch_with_a_full_size_pair_equals_oracle():
    # a 1242x375 pair (the KITTI size, Lab) in a batch with two small pairs,
    # in the batch's own parameters (4 scales, 6 sweeps), as a replayed graph
    from concurrent.futures import ThreadPoolExecutor
    pairs = [workloads.batch_pair(5, 0, ((1242, 375),)), workloads.batch_pair(5, 1, ((97, 71),)),
             workloads.batch_pair(5, 2, ((64, 48),))]
    prm = workloads.BATCH_PARAMS
    cfg = ff.Config(channels=3, scales=prm["scales"], iters=prm["iters"],
                    radius_q3=prm["radius_q3"], max_width=1242, max_height=375)
    b = ff.ff_batch_create(cfg, 0, slots=2)
    imgs = _upload(pairs)
    two_way = [False] * 3
    outs = _outputs(pairs, cfg, two_way)
    descs = ff.pair_descs(_descs(pairs, imgs, outs))
    for _ in range(2):           # capture, then a replay
        ff.ff_batch_run(b, descs, use_graph=True)
        ff.ff_batch_sync(b)
    P = O.Params(channels=3, scales=prm["scales"], iters=prm["iters"], radius_q3=prm["radius_q3"])
    S = prm["scales"]
    for k, (p, o) in enumerate(zip(pairs, outs)):
        f1 = O.features_all(p.img1, S)
        f2 = O.features_all(p.img2, S)
        jobs = []
        for d, (a, bb) in enumerate(((f1, f2), (f2, f1))):
            ki, _ = O.seed_knn_threaded(a[0], bb[0], S)
            jobs.append((a, bb, d, ki))
        with ThreadPoolExecutor(max_workers=2) as ex:
            (rf, _, _), (rb, _, _) = ex.map(
                lambda j: O.match_features_knn(P, j[0], j[1], p.width, p.height, j[2], 100 + k,
                                               j[3]), jobs)
        np.testing.assert_array_equal(_host(o["fwd"]), rf, err_msg=f"pair {k}")
        np.testing.assert_array_equal(_host(o["bwd"]), rb, err_msg=f"pair {k}")
        np.testing.assert_array_equal(_host(o["mask"]), O.filter_mask(rf, rb, 8),
                                      err_msg=f"pair {k}")
    ff.ff_batch_destroy(b)


def test_batch_same_alone_and_in_the_mix_and_graph_replays():
    import torch
    sizes = ((320, 240), (640, 480), (200, 150))
    pairs = [workloads.batch_pair(11, k, sizes) for k in range(10)]
    two_way = [k % 4 == 1 for k in range(10)]
    cfg = ff.Config(channels=3, scales=4, iters=6, radius_q3=8, max_width=640, max_height=480)
    imgs = _upload(pairs)
    # alone: one context, one pair at a time
    ctx = ff.Context(cfg)
    alone = []
    for k, (p, (i1, i2)) in enumerate(zip(pairs, imgs)):
        ctx.features(0, i1)
        ctx.features(1, i2)
        f, _ = ctx.match(ff.FF_FWD, 100 + k, with_cost=False)
        bw, _ = ctx.match(ff.FF_BWD, 100 + k, with_cost=False)
        if two_way[k]:
            b2, _ = ctx.match(ff.FF_BWD2, 100 + k, with_cost=False)
            m = ctx.filter_2way(f, bw, b2)
        else:
            b2, m = None, ctx.filter(f, bw)
        alone.append((f, bw, b2, m))
    ctx.sync()
    ctx.close()
    b = ff.ff_batch_create(cfg, 0, slots=4)
    outs = _outputs(pairs, cfg, two_way)
    descs = ff.pair_descs(_descs(pairs, imgs, outs))

    def check(tag):
        for k, (o, a) in enumerate(zip(outs, alone)):
            assert torch.equal(o["fwd"], a[0]), f"{tag} pair {k} fwd"
            assert torch.equal(o["bwd"], a[1]), f"{tag} pair {k} bwd"
            if two_way[k]:
                assert torch.equal(o["bwd2"], a[2]), f"{tag} pair {k} bwd2"
            assert torch.equal(o["mask"], a[3]), f"{tag} pair {k} mask"

    def clobber():
        for o in outs:
            for t in o.values():
                if t is not None:
                    t.fill_(3)

    ff.ff_batch_run(b, descs)
    ff.ff_batch_sync(b)
    check("direct")
    n0 = ff.ff_batch_launch_count(b)
    for rep in range(3):      # capture, then two replays of the same graph
        clobber()
        ff.ff_batch_run(b, descs, use_graph=True)
        ff.ff_batch_sync(b)
        check(f"graph {rep}")
    per_run = (ff.ff_batch_launch_count(b) - n0) // 3
    assert per_run == n0 > 0
    ff.ff_batch_destroy(b)


def test_batch_rejects_bad_descriptors_before_launching():
    import torch
    cfg = ff.Config(channels=3, scales=2, iters=2, max_width=64, max_height=64)
    b = ff.ff_batch_create(cfg, 0, slots=2)
    img = torch.zeros((3, 64, 65), dtype=torch.uint8, device="cuda")
    flow = torch.zeros((64, 65, 2), dtype=torch.int16, device="cuda")
    good = dict(img1=img, img2=img, w=64, h=64, pitch=65, flow_fwd=flow, flow_bwd=flow)
    bad = dict(good, w=65)
    with pytest.raises(ff.FFError) as e:
        ff.ff_batch_run(b, [good, bad])
    assert e.value.status == ff.FF_EINVAL and "pair 1" in str(e.value)
    with pytest.raises(ff.FFError) as e:
        ff.ff_batch_run(b, [dict(good, flow_bwd=None)])
    assert e.value.status == ff.FF_EINVAL
    assert ff.ff_batch_launch_count(b) == 0
    ff.ff_batch_run(b, [])
    ff.ff_batch_sync(b)
    ff.ff_batch_destroy(b)


def test_autotune_times_every_candidate_and_keeps_the_fastest(tmp_path):
    from paper_1703_02563_gb300 import autotune
    pairs = [workloads.batch_pair(13, k, SMALL_SIZES) for k in range(4)]
    cfg = ff.Config(channels=3, scales=3, iters=4, radius_q3=8, max_width=128, max_height=96)
    imgs = _upload(pairs)
    outs = _outputs(pairs, cfg, [False] * 4)
    descs = ff.pair_descs(_descs(pairs, imgs, outs))
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(cfg, descs, 4, max_slots=16, steps=1, path=cache)
    cands = autotune.candidates(cfg, 16)
    assert [(t["slots"], t["lanes"]) for t in res["trials"]] == cands
    assert all(t["ms"] > 0 for t in res["trials"])
    assert res["ms"] == min(t["ms"] for t in res["trials"])
    assert autotune.lookup(cfg, 0, cache)["slots"] == res["slots"]
