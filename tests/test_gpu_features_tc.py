"""The WHT on the tensor cores.

The precision form (the KITTI-shaped workload): the transform of the FP32
scale-space image (the area average without rounding) with bf16 or fp16
inputs and FP32 accumulation, against an FP64 transform, within the bound
the two formats' rounding allows; and the production path (rounded integer
level images in bf16, exact) through its int8 features and the matching
they feed, bit-exact with the oracle."""
from __future__ import annotations

import numpy as np
import pytest
from scipy import linalg

import oracle as O
from paper_1703_02563_gb300 import ff, workloads

pytestmark = pytest.mark.gpu

# half a unit in the last place of a value below 256: 8 significant bits
# (bf16) leave 0.5, 11 (fp16) leave 1/16
HALF_ULP_BELOW_256 = {"bf16": 0.5, "fp16": 1.0 / 16.0}
# FP32 accumulation of 64 terms whose partial sums stay below 2^14: each
# addition rounds by at most 2^(14 - 24) / 2
FP32_ACC_BOUND = 64 * 2.0 ** -11


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _fp64_scalespace_wht(img: np.ndarray, L: int) -> np.ndarray:
    """FP64: the n x n block mean (replicate border, no rounding), then the
    3 x 3 lowest-sequency Walsh coefficients over the 8 x 8 window at offsets
    -3..+4 (replicate border), from scipy's Hadamard matrix."""
    C, H, W = img.shape
    n = 1 << L
    WL, HL = -(-W // n), -(-H // n)
    pad = np.pad(img.astype(np.float64), ((0, 0), (0, HL * n - H), (0, WL * n - W)), mode="edge")
    D = pad.reshape(C, HL, n, WL, n).mean(axis=(2, 4))
    H8 = linalg.hadamard(8).astype(np.float64)
    changes = [(np.diff(np.sign(r)) != 0).sum() for r in H8]
    w = H8[np.argsort(changes, kind="stable")][:3]
    Dp = np.pad(D, ((0, 0), (3, 4), (3, 4)), mode="edge")
    win = np.lib.stride_tricks.sliding_window_view(Dp, (8, 8), axis=(1, 2))   # C,HL,WL,8,8
    out = np.einsum("chwij,ui,vj->hwcuv", win, w, w)
    return out.reshape(HL, WL, 9 * C)


def _codes(c: np.ndarray) -> np.ndarray:
    q = np.floor(c / 16.0 + 0.5)
    q[..., 0::9] = np.floor(c[..., 0::9] / 64.0 + 0.5) - 128
    return np.clip(q, -128, 127).astype(np.int64)


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
@pytest.mark.parametrize("name", ["kitti1242x375", "sintel1024x436"])
def test_scalespace_wht_within_the_format_bound(name, fmt):
    import torch
    pair, prm = workloads.make_workload(name)
    C, H, W = pair.img1.shape
    img = _dev(pair.img1)
    errs = []
    for L in range(prm["scales"]):
        WL, HL = O.level_dims(W, H, L)
        out = torch.full((HL, WL, 9 * C), float("nan"), dtype=torch.float32, device="cuda")
        ff.ff_wht_coeffs_scalespace_tc(img, W, H, W, C, L, fmt == "fp16", out)
        got = _host(out).astype(np.float64)
        ref = _fp64_scalespace_wht(pair.img1, L)
        assert np.isfinite(got).all()
        err = np.abs(got - ref).max()
        bound = 0.0 if L == 0 else 64 * HALF_ULP_BELOW_256[fmt] + FP32_ACC_BOUND
        assert err <= bound, f"level {L}: max |error| {err} > {bound}"
        errs.append(err)
        flips = int((_codes(got) != _codes(ref)).sum())
        assert 0 <= flips <= got.size
    # the fractional averages of the coarse levels are not all representable
    assert max(errs[1:]) > 0
    assert errs[0] == 0


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
