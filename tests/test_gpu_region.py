"""The region filter (Sec. 3.7) on the GPU against the oracle, bit-exact."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1703_02563_gb300 import ff, workloads

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _block_flows(rng, H, W, block, noise, invalid=0.05, keep=0.8):
    nb = rng.integers(-6, 7, (H // block + 1, W // block + 1, 2)) * 20
    f = np.repeat(np.repeat(nb, block, 0), block, 1)[:H, :W] + rng.integers(-noise, noise + 1,
                                                                             (H, W, 2))
    f = f.astype(np.int16)
    f[rng.random((H, W)) < invalid] = (-32768, -32768)
    m = (rng.random((H, W)) < keep).astype(np.uint8)
    m[f[..., 0] == -32768] = 0
    return f, m


@pytest.mark.parametrize("W,H,block,noise", [(31, 23, 4, 14), (1, 1, 1, 0), (1, 57, 3, 10),
                                             (300, 201, 9, 12), (1024, 436, 24, 20)])
def test_region_filter_bit_exact(W, H, block, noise):
    rng = np.random.default_rng(W * 1000 + H)
    f, m = _block_flows(rng, H, W, block, noise)
    ctx = ff.Context(ff.Config(channels=1, scales=1, iters=1, max_width=W, max_height=H))
    ctx.features(0, _dev(np.zeros((1, H, W), np.uint8)))
    ctx.features(1, _dev(np.zeros((1, H, W), np.uint8)))
    df, dm = _dev(f), _dev(m)
    for s in (0, 1, 5, 40, 150, 1 << 20):
        np.testing.assert_array_equal(_host(ctx.region_filter(df, dm, s)), O.region_filter(f, m, s),
                                      err_msg=f"s {s}")
    # in place
    ff.ff_region_filter(ctx.ctx, df, dm, 40, dm)
    np.testing.assert_array_equal(_host(dm), O.region_filter(f, m, 40))
    ctx.close()


def test_region_filter_one_region_covering_the_frame():
    # a smooth ramp: every neighbour pair is close, so all kept points form
    # one region however far its ends drift; long union chains on the GPU
    H, W = 200, 300
    yy, xx = np.mgrid[0:H, 0:W]
    f = np.stack([xx * 2, yy * 3], -1).astype(np.int16)
    m = np.ones((H, W), np.uint8)
    m[100, 150] = 0
    ctx = ff.Context(ff.Config(channels=1, scales=1, iters=1, max_width=W, max_height=H))
    ctx.features(0, _dev(np.zeros((1, H, W), np.uint8)))
    ctx.features(1, _dev(np.zeros((1, H, W), np.uint8)))
    for s in (H * W - 1, H * W):
        np.testing.assert_array_equal(_host(ctx.region_filter(_dev(f), _dev(m), s)),
                                      O.region_filter(f, m, s))
    ctx.close()


@pytest.mark.parametrize("schedule", [ff.FF_SCHED_BASIC, ff.FF_SCHED_PLUS_FAST_X2])
def test_pair_path_applies_the_region_filter(schedule):
    import torch
    pair = workloads.layered_pair(seed=13, width=160, height=120, channels=3, max_disp=30)
    W, H = pair.width, pair.height
    stride = 2 if schedule == ff.FF_SCHED_PLUS_FAST_X2 else 1
    cfg = ff.Config(channels=3, scales=3, iters=4, max_width=W, max_height=H, schedule=schedule,
                    seed_stride=stride, region_min=60)
    P = O.Params(channels=3, scales=3, iters=4, schedule=schedule, seed_stride=stride)
    Lf = P.final_level()
    WL, HL = O.level_dims(W, H, Lf)
    rf, _, _ = O.match(P, pair.img1, pair.img2, 0, 5)
    rb, _, _ = O.match(P, pair.img2, pair.img1, 1, 5)
    ref = O.region_filter(rf, O.filter_mask(rf, rb, 8, level=Lf), 60)
    # the host-buffer call
    ctx = ff.Context(cfg)
    hm = torch.empty((HL, WL), dtype=torch.uint8).pin_memory()
    ff.ff_pair_host(ctx.ctx, torch.from_numpy(pair.img1.copy()), torch.from_numpy(pair.img2.copy()),
                    W, H, 5, None, None, hm)
    np.testing.assert_array_equal(hm.numpy(), ref)
    ctx.close()
    # the batched form
    b = ff.ff_batch_create(cfg, 0, slots=2)
    i1, i2 = _dev(pair.img1), _dev(pair.img2)
    outs = [dict(fwd=torch.empty((HL, WL, 2), dtype=torch.int16, device="cuda"),
                 bwd=torch.empty((HL, WL, 2), dtype=torch.int16, device="cuda"),
                 mask=torch.empty((HL, WL), dtype=torch.uint8, device="cuda")) for _ in range(3)]
    ff.ff_batch_run(b, [dict(img1=i1, img2=i2, w=W, h=H, pair_id=5, flow_fwd=o["fwd"],
                             flow_bwd=o["bwd"], mask=o["mask"]) for o in outs], use_graph=True)
    ff.ff_batch_sync(b)
    for o in outs:
        np.testing.assert_array_equal(_host(o["mask"]), ref)
    ff.ff_batch_destroy(b)


@pytest.mark.parametrize("schedule", [ff.FF_SCHED_BASIC, ff.FF_SCHED_PLUS_FAST_X2])
@pytest.mark.parametrize("W,H", [(53, 41), (1, 1), (300, 7)])
def test_sparsify_bit_exact(schedule, W, H):
    rng = np.random.default_rng(W + 17 * H + schedule)
    cfg = ff.Config(channels=1, scales=2, iters=1, max_width=W, max_height=H, schedule=schedule,
                    seed_stride=2 if schedule == ff.FF_SCHED_PLUS_FAST_X2 else 1)
    ctx = ff.Context(cfg)
    ctx.features(0, _dev(np.zeros((1, H, W), np.uint8)))
    ctx.features(1, _dev(np.zeros((1, H, W), np.uint8)))
    L = cfg.final_level()
    WL, HL = O.level_dims(W, H, L)
    fwd = rng.integers(-40, 40, (HL, WL, 2)).astype(np.int16)
    b1 = (-fwd + rng.integers(-12, 13, (HL, WL, 2))).astype(np.int16)
    b2 = (-fwd + rng.integers(-12, 13, (HL, WL, 2))).astype(np.int16)
    fwd[rng.random((HL, WL)) < 0.05] = (-32768, -32768)
    b2[rng.random((HL, WL)) < 0.05] = (-32768, -32768)
    for mask in (O.filter_mask2(fwd, b1, b2, 24, level=L),
                 (rng.random((HL, WL)) < 0.6).astype(np.uint8)):   # arbitrary: infinite errors
        dm = _dev(mask)
        for q, e in ((1, 1), (3, 0), (3, 2), (4, 5), (8, 3), (64, 1)):
            for bb in (None, b2):
                got = ctx.sparsify(_dev(fwd), _dev(b1), None if bb is None else _dev(bb), dm, q, e)
                np.testing.assert_array_equal(_host(got), O.sparsify(fwd, b1, bb, mask, q, e, L),
                                              err_msg=f"q {q} e {e} two-way {bb is not None}")
        ff.ff_sparsify(ctx.ctx, _dev(fwd), _dev(b1), None, dm, 3, 2, dm)   # in place
        np.testing.assert_array_equal(_host(dm), O.sparsify(fwd, b1, None, mask, 3, 2, L))
    with pytest.raises(ff.FFError):
        ctx.sparsify(_dev(fwd), _dev(b1), None, dm, 0, 1)
    ctx.close()
