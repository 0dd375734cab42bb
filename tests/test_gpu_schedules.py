"""Flow Fields+ schedules and the two-way consistency check on the GPU.

The CUDA path under the Flow Fields+ (Sec. 3.3), Flow Fields+ Fast and Fast
x2 (Sec. 3.4) schedules, the second backward flow and the two-way check of
Sec. 3.7, each compared with the oracle element by element (bit-exact).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1703_02563_gb300 import ff, workloads

pytestmark = pytest.mark.gpu


def _ctx(C, S, I, W, H, schedule, R=8, eps=8, stride=1):
    cfg = ff.Config(channels=C, scales=S, iters=I, radius_q3=R, eps_q3=eps, max_width=W,
                    max_height=H, schedule=schedule, seed_stride=stride)
    return ff.Context(cfg)


def _params(C, S, I, schedule, R=8, stride=1):
    return O.Params(channels=C, scales=S, iters=I, radius_q3=R, schedule=schedule,
                    seed_stride=stride)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _load(ctx, pair):
    ctx.features(0, _dev(pair.img1))
    ctx.features(1, _dev(pair.img2))


@pytest.mark.parametrize("schedule", [ff.FF_SCHED_PLUS, ff.FF_SCHED_PLUS_FAST,
                                      ff.FF_SCHED_PLUS_FAST_X2])
def test_schedule_every_stage_bit_exact(schedule):
    # every sweep of every level: the wide-radius phase, the missing random
    # search at its end, the narrow phase and (Fast) the short finest scale
    pair = workloads.layered_pair(seed=17, width=97, height=71, channels=3, max_disp=15)
    S, I = 3, 4
    stride = 2 if schedule == ff.FF_SCHED_PLUS_FAST_X2 else 1
    ctx = _ctx(3, S, I, pair.width, pair.height, schedule, R=12, stride=stride)
    _load(ctx, pair)
    P = _params(3, S, I, schedule, R=12, stride=stride)
    Lf = P.final_level()
    assert Lf == ctx.cfg.final_level()
    for L in range(S - 1, Lf - 1, -1):
        n = P.sweeps(L)
        assert n == ctx.cfg.sweeps(L)
        for k in range(n + 1):
            flow, cost = ctx.match(0, 6, until_level=L, until_sweeps=k)
            rf, rc, _ = O.match(P, pair.img1, pair.img2, 0, 6, until_level=L, until_sweeps=k)
            np.testing.assert_array_equal(_host(flow), rf, err_msg=f"L {L} k {k}")
            np.testing.assert_array_equal(_host(cost), rc, err_msg=f"L {L} k {k}")
    with pytest.raises(ff.FFError) as e:
        ctx.match(0, 6, until_level=Lf, until_sweeps=P.sweeps(Lf) + 1)
    assert e.value.status == ff.FF_EINVAL
    if Lf > 0:   # Fast x2 never runs the finest scale
        flow = _dev(np.zeros((pair.height, pair.width, 2), np.int16))
        with pytest.raises(ff.FFError) as e:
            ff.ff_match_until(ctx.ctx, 0, 6, None, 0, 0, flow, None)
        assert e.value.status == ff.FF_EINVAL
    ctx.close()


SCHEDULE_CASES = [
    ("tiny-plus", lambda: workloads.make_workload("tiny128x96")[0], 1, 3, ff.FF_SCHED_PLUS, 8),
    ("tiny-fast", lambda: workloads.make_workload("tiny128x96")[0], 1, 3, ff.FF_SCHED_PLUS_FAST, 8),
    ("lab120x80-plus", lambda: workloads.layered_pair(seed=23, width=120, height=80, channels=3,
                                                      max_disp=30), 3, 3, ff.FF_SCHED_PLUS, 12),
    ("gray33x17-fast", lambda: workloads.random_pair(seed=5, width=33, height=17), 1, 2,
     ff.FF_SCHED_PLUS_FAST, 8),
    ("gray1x1-plus", lambda: workloads.random_pair(seed=8, width=1, height=1), 1, 1,
     ff.FF_SCHED_PLUS, 8),
    ("tiny-x2", lambda: workloads.make_workload("tiny128x96")[0], 1, 3,
     ff.FF_SCHED_PLUS_FAST_X2, 8),
    ("lab121x79-x2", lambda: workloads.layered_pair(seed=29, width=121, height=79, channels=3,
                                                    max_disp=30), 3, 4,
     ff.FF_SCHED_PLUS_FAST_X2, 12),
    ("gray3x3-x2", lambda: workloads.random_pair(seed=10, width=3, height=3), 1, 2,
     ff.FF_SCHED_PLUS_FAST_X2, 8),
]


@pytest.mark.parametrize("name,make,C,S,schedule,R", SCHEDULE_CASES,
                         ids=[c[0] for c in SCHEDULE_CASES])
def test_three_flows_and_two_way_filter_bit_exact(name, make, C, S, schedule, R):
    pair = make()
    I = 4
    stride = 2 if schedule == ff.FF_SCHED_PLUS_FAST_X2 else 1
    ctx = _ctx(C, S, I, pair.width, pair.height, schedule, R=R, stride=stride)
    _load(ctx, pair)
    P = _params(C, S, I, schedule, R=R, stride=stride)
    Lf = P.final_level()
    fwd, cf = ctx.match(ff.FF_FWD, 29)
    bwd1, cb1 = ctx.match(ff.FF_BWD, 29)
    bwd2, cb2 = ctx.match(ff.FF_BWD2, 29)
    mask1 = ctx.filter(fwd, bwd1)
    mask2 = ctx.filter_2way(fwd, bwd1, bwd2)
    rf, rcf, _ = O.match(P, pair.img1, pair.img2, 0, 29)
    rb1, rcb1, _ = O.match(P, pair.img2, pair.img1, 1, 29)
    rb2, rcb2, _ = O.match(P, pair.img2, pair.img1, 2, 29)
    for got, ref in ((fwd, rf), (cf, rcf), (bwd1, rb1), (cb1, rcb1), (bwd2, rb2), (cb2, rcb2)):
        np.testing.assert_array_equal(_host(got), ref)
    assert rf.shape[:2] == O.level_dims(pair.width, pair.height, Lf)[::-1]
    np.testing.assert_array_equal(_host(mask1), O.filter_mask(rf, rb1, 8, level=Lf))
    np.testing.assert_array_equal(_host(mask2), O.filter_mask2(rf, rb1, rb2, 8, level=Lf))
    ctx.sync()
    ctx.close()


def test_grid_filter_bit_exact_on_arbitrary_flows():
    # Fast x2 flows live on the level-1 grid: the check reads the grid point
    # nearest to p + F(p)
    rng = np.random.default_rng(12)
    W, H = 57, 43
    pair = workloads.random_pair(seed=3, width=W, height=H)
    ctx = _ctx(1, 2, 4, W, H, ff.FF_SCHED_PLUS_FAST_X2, eps=10, stride=2)
    _load(ctx, pair)
    WL, HL = O.level_dims(W, H, 1)
    fwd = rng.integers(-70, 70, (HL, WL, 2)).astype(np.int16)
    b1 = rng.integers(-70, 70, (HL, WL, 2)).astype(np.int16)
    b2 = rng.integers(-70, 70, (HL, WL, 2)).astype(np.int16)
    b1[3:18, 3:18] = -fwd[3:18, 3:18]
    b2[8:22, 8:22] = -fwd[8:22, 8:22]
    fwd[1, 1] = (ff.INVALID, ff.INVALID)
    np.testing.assert_array_equal(_host(ctx.filter(_dev(fwd), _dev(b1))),
                                  O.filter_mask(fwd, b1, 10, level=1))
    np.testing.assert_array_equal(_host(ctx.filter_2way(_dev(fwd), _dev(b1), _dev(b2))),
                                  O.filter_mask2(fwd, b1, b2, 10, level=1))
    ctx.close()


def test_pair_host_fast_x2_returns_the_level1_grid():
    import torch
    pair, prm = workloads.make_workload("tiny128x96")
    W, H = pair.width, pair.height
    S = prm["scales"]
    ctx = _ctx(1, S, 4, W, H, ff.FF_SCHED_PLUS_FAST_X2, stride=2)
    WL, HL = O.level_dims(W, H, 1)
    fwd = torch.empty((HL, WL, 2), dtype=torch.int16).pin_memory()
    bwd = torch.empty((HL, WL, 2), dtype=torch.int16).pin_memory()
    mask = torch.empty((HL, WL), dtype=torch.uint8).pin_memory()
    i1 = torch.from_numpy(pair.img1.copy()).pin_memory()
    i2 = torch.from_numpy(pair.img2.copy()).pin_memory()
    ff.ff_pair_host(ctx.ctx, i1, i2, W, H, 4, fwd, bwd, mask)
    P = _params(1, S, 4, ff.FF_SCHED_PLUS_FAST_X2, stride=2)
    rf, _, _ = O.match(P, pair.img1, pair.img2, 0, 4)
    rb, _, _ = O.match(P, pair.img2, pair.img1, 1, 4)
    np.testing.assert_array_equal(fwd.numpy(), rf)
    np.testing.assert_array_equal(bwd.numpy(), rb)
    np.testing.assert_array_equal(mask.numpy(), O.filter_mask(rf, rb, 8, level=1))
    ctx.close()


def test_two_way_filter_bit_exact_on_arbitrary_flows():
    rng = np.random.default_rng(11)
    W, H = 53, 41
    pair = workloads.random_pair(seed=2, width=W, height=H)
    ctx = _ctx(1, 1, 1, W, H, ff.FF_SCHED_BASIC, eps=11)
    _load(ctx, pair)
    fwd = rng.integers(-60, 60, (H, W, 2)).astype(np.int16)
    b1 = rng.integers(-60, 60, (H, W, 2)).astype(np.int16)
    b2 = rng.integers(-60, 60, (H, W, 2)).astype(np.int16)
    b1[5:30, 5:30] = -fwd[5:30, 5:30]
    b2[15:40, 15:40] = -fwd[15:40, 15:40]
    fwd[2, 3] = (ff.INVALID, ff.INVALID)
    b2[20, 20] = (ff.INVALID, ff.INVALID)
    mask = ctx.filter_2way(_dev(fwd), _dev(b1), _dev(b2))
    np.testing.assert_array_equal(_host(mask), O.filter_mask2(fwd, b1, b2, 11))
    ctx.close()


@pytest.mark.parametrize("schedule,scales", [(4, 3), (-1, 3), (ff.FF_SCHED_PLUS_FAST_X2, 1)])
def test_unknown_schedule_rejected(schedule, scales):
    cfg = ff.Config(max_width=64, max_height=64, schedule=schedule, scales=scales)
    with pytest.raises(ff.FFError) as e:
        ff.Context(cfg)
    assert e.value.status == ff.FF_EINVAL
