"""The WHT on the bf16 tensor cores (the precision form of the KITTI-shaped
workload): its FP32 coefficients against the oracle's exact transform (an
FP64-exact integer WHT), and the int8 features and matching it feeds,
bit-exact."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1703_02563_gb300 import ff, workloads

pytestmark = pytest.mark.gpu

# the error bound the tests hold the tensor-core transform to: none
TC_MAX_ABS_ERROR = 0.0


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("name", ["kitti1242x375", "sintel1024x436"])
def test_tc_coefficients_equal_the_fp64_transform(name):
    import torch
    pair, prm = workloads.make_workload(name)
    C, H, W = pair.img1.shape
    img = _dev(pair.img1)
    for L in range(prm["scales"]):
        WL, HL = O.level_dims(W, H, L)
        out = torch.full((HL, WL, 9 * C), float("nan"), dtype=torch.float32, device="cuda")
        ff.ff_wht_coeffs_tc(img, W, H, W, C, L, out)
        got = _host(out).astype(np.float64)
        ref = O.wht_coeffs(O.level_image(pair.img1, L)).astype(np.float64)
        err = np.abs(got - ref)
        assert np.isfinite(got).all()
        assert err.max() <= TC_MAX_ABS_ERROR, f"level {L}: max |error| {err.max()}"


FEATURE_CASES = [(1, 1242, 375, 4), (3, 97, 71, 3), (1, 37, 29, 4), (3, 16, 9, 2), (1, 1, 1, 1),
                 (1, 200, 3, 3)]


@pytest.mark.parametrize("C,W,H,S", FEATURE_CASES)
def test_tc_features_bit_exact(C, W, H, S):
    pair = workloads.random_pair(seed=W * 3 + H, width=W, height=H, channels=C)
    ctx = ff.Context(ff.Config(channels=C, scales=S, iters=1, max_width=W, max_height=H,
                               wht_tensor_cores=1))
    ctx.features(0, _dev(pair.img1))
    ctx.features(1, _dev(pair.img2))
    for slot, img in ((0, pair.img1), (1, pair.img2)):
        ref = O.features_all(img, S)
        for L in range(S):
            np.testing.assert_array_equal(_host(ctx.features_of(slot, L)), ref[L])
    ctx.close()


def test_tc_path_matches_bit_exact():
    # the KITTI-shaped precision form: tensor-core features, int8/int32
    # matching, on a reduced frame so the oracle finishes in seconds
    pair = workloads.expansion_pair(seed=3, width=310, height=94)
    cfg = ff.Config(channels=1, scales=3, iters=4, radius_q3=12, max_width=310, max_height=94,
                    wht_tensor_cores=1)
    ctx = ff.Context(cfg)
    ctx.features(0, _dev(pair.img1))
    ctx.features(1, _dev(pair.img2))
    fwd, cf = ctx.match(0, 2)
    bwd, _ = ctx.match(1, 2)
    P = O.Params(channels=1, scales=3, iters=4, radius_q3=12)
    rf, rc, _ = O.match(P, pair.img1, pair.img2, 0, 2)
    rb, _, _ = O.match(P, pair.img2, pair.img1, 1, 2)
    np.testing.assert_array_equal(_host(fwd), rf)
    np.testing.assert_array_equal(_host(cf), rc)
    np.testing.assert_array_equal(_host(ctx.filter(fwd, bwd)), O.filter_mask(rf, rb, 8))
    ctx.close()
