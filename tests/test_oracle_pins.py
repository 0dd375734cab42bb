"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks one step of the method (arXiv 1703.02563, Sec. 3) against a
closed form, a library routine, brute force on a tiny input, a hand-computed
case or an invariant the paper states, so that a dropped term, a wrong sign,
a wrong index or a transposed operand in ``oracle/ffo.c`` fails here.
"""
from __future__ import annotations

import os
from decimal import Decimal, getcontext

import numpy as np
import pytest
from scipy import linalg, ndimage

import oracle as O
from paper_1703_02563_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name: str) -> dict:
    """Read a ``key = value`` fixture (lines starting with # are the citation)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            out[k.strip()] = v.strip()
    return out


# --------------------------------------------------------------------------
# level images (Sec. 3.6: area downsampling, replicative border)
# --------------------------------------------------------------------------
def test_levels_constant_image():
    img = np.full((3, 37, 53), 201, np.uint8)
    for L in range(4):
        D = O.level_image(img, L)
        assert D.shape == (3, -(-37 // (1 << L)), -(-53 // (1 << L)))
        assert np.all(D == 201)


@pytest.mark.parametrize("C,W,H", [(1, 45, 31), (3, 64, 48), (1, 17, 9)])
def test_levels_block_mean_by_reshape(C, W, H):
    rng = np.random.default_rng(W * H + C)
    img = rng.integers(0, 256, (C, H, W), dtype=np.uint8)
    for L in range(4):
        n = 1 << L
        WL, HL = -(-W // n), -(-H // n)
        pad = np.pad(img.astype(np.int64), ((0, 0), (0, HL * n - H), (0, WL * n - W)), mode="edge")
        sums = pad.reshape(C, HL, n, WL, n).sum(axis=(2, 4))
        expect = np.floor(sums / (n * n) + 0.5).astype(np.uint8)
        np.testing.assert_array_equal(O.level_image(img, L), expect)


def test_levels_checkerboard_rounds_half_up():
    img = np.zeros((1, 8, 8), np.uint8)
    img[0, ::2, ::2] = 255
    img[0, 1::2, 1::2] = 255
    # every 2x2 block holds two 255s: mean 127.5 rounds up to 128
    assert np.all(O.level_image(img, 1) == 128)
    # 4x4 blocks: mean 127.5 again
    assert np.all(O.level_image(img, 2) == 128)


# --------------------------------------------------------------------------
# WHT features (Sec. 3.1: first 9 Walsh-Hadamard bases per channel)
# --------------------------------------------------------------------------
def _sequency_walsh(k: int) -> np.ndarray:
    """The k lowest-sequency rows of the 8x8 Sylvester Hadamard matrix."""
    H8 = linalg.hadamard(8).astype(np.float64)
    changes = [(np.diff(np.sign(r)) != 0).sum() for r in H8]
    return H8[np.argsort(changes, kind="stable")][:k]


@pytest.mark.parametrize("C,W,H", [(1, 23, 19), (3, 16, 12), (1, 5, 3)])
def test_wht_equals_fp64_hadamard_product(C, W, H):
    rng = np.random.default_rng(7 + W)
    D = rng.integers(0, 256, (C, H, W), dtype=np.uint8)
    w = _sequency_walsh(3)
    got = O.wht_coeffs(D)
    P = np.pad(D.astype(np.float64), ((0, 0), (3, 4), (3, 4)), mode="edge")
    for y in range(H):
        for x in range(W):
            for c in range(C):
                win = P[c, y:y + 8, x:x + 8]      # rows y-3..y+4, cols x-3..x+4
                coef = w @ win @ w.T               # [u][v], u along rows
                np.testing.assert_array_equal(got[y, x, 9 * c:9 * c + 9], coef.reshape(9))


def test_wht_constant_image_has_only_dc():
    D = np.full((3, 10, 12), 77, np.uint8)
    coef = O.wht_coeffs(D)
    assert np.all(coef[..., 0::9] == 64 * 77)
    mask = np.ones(27, bool)
    mask[0::9] = False
    assert np.all(coef[..., mask] == 0)
    q = O.wht_features(D)
    assert np.all(q[..., 0::9] == 77 - 128)
    assert np.all(q[..., mask] == 0)


def test_wht_vertical_step_edge_closed_form():
    a, b, x0 = 40, 200, 8
    D = np.full((1, 12, 16), a, np.uint8)
    D[0, :, x0:] = b
    coef = O.wht_coeffs(D)
    # pixel x0-1: the window's left half (cols x0-4..x0-1) is a, right half b
    c = coef[6, x0 - 1]
    assert c[0] == 32 * a + 32 * b          # DC
    assert c[1] == 32 * (a - b)              # u=0, v=1: left half minus right half
    assert c[2] == 0                         # u=0, v=2: ++--|--++ cancels
    assert np.all(c[3:] == 0)                # no variation down the rows
    # pixel x0-2: left half a, right half a,b,b,b  (cols x0-5 .. x0+2)
    c = coef[6, x0 - 2]
    assert c[1] == 8 * (4 * a - (a + 3 * b))
    assert c[2] == 8 * ((a + a) - (a + a) - (a + b) + (b + b))


def test_quantiser_rounding_boundaries():
    # AC terms: round(c / 16) half up, saturated
    assert [O.quantise(c, False) for c in (7, 8, -8, -9, 24, -24, 2032, 2040, 5000, -5000)] == \
        [0, 1, 0, -1, 2, -1, 127, 127, 127, -128]
    assert O.quantise(-2056, False) == -128 and O.quantise(-2055, False) == -128
    assert O.quantise(-2040, False) == -127
    # DC term: round(c / 64) half up, minus 128
    assert [O.quantise(c, True) for c in (0, 31, 32, 64 * 255, 64 * 128, 64 * 128 - 33)] == \
        [-128, -128, -127, 127, 0, -1]


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al. SC'11), the random-search generator
# --------------------------------------------------------------------------
getcontext().prec = 60
_PHI = (Decimal(1) + Decimal(5).sqrt()) / 2
_SQRT3 = Decimal(3).sqrt()


def _frac_bits(x: Decimal, w: int) -> int:
    return int((x - int(x)) * (Decimal(2) ** w))


def _philox(ctr, key, w: int, mult):
    """Philox4xW-10 written from the SC'11 description, for any word size."""
    mask = (1 << w) - 1
    bump = (_frac_bits(_PHI, w), _frac_bits(_SQRT3, w))
    c, k = [int(v) for v in ctr], [int(v) for v in key]
    for r in range(10):
        if r:
            k = [(k[0] + bump[0]) & mask, (k[1] + bump[1]) & mask]
        p0, p1 = mult[0] * c[0], mult[1] * c[2]
        c = [(p1 >> w) ^ c[1] ^ k[0], p1 & mask, (p0 >> w) ^ c[3] ^ k[1], p0 & mask]
    return c


_M64 = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
_M32 = (0xD2511F53, 0xCD9E8D57)


def test_philox_round_structure_matches_numpy_4x64():
    # numpy's Philox bit generator is the 4x64-10 member of the same family;
    # it advances its counter by one before each block
    rng = np.random.default_rng(11)
    for _ in range(6):
        ctr = [int(v) for v in rng.integers(0, 2**63, 4)]
        key = [int(v) for v in rng.integers(0, 2**63, 2)]
        bg = np.random.Philox(counter=ctr, key=key)
        got = [int(v) for v in bg.random_raw(4)]
        ctr1 = list(ctr)
        ctr1[0] += 1
        assert got == _philox(ctr1, key, 64, _M64)


def test_philox_4x32_oracle_agrees_with_independent_impl():
    rng = np.random.default_rng(12)
    cases = [([0, 0, 0, 0], [0, 0]), ([2**32 - 1] * 4, [2**32 - 1] * 2)]
    cases += [(list(rng.integers(0, 2**32, 4)), list(rng.integers(0, 2**32, 2)))
              for _ in range(50)]
    for ctr, key in cases:
        assert [int(v) for v in O.philox4x32_10(ctr, key)] == _philox(ctr, key, 32, _M32)


# --------------------------------------------------------------------------
# flow clamp and matching cost (Sec. 3.1: bilinear interpolation, Sec. 3.6 border)
# --------------------------------------------------------------------------
def test_clamp_flow_closed_form():
    W, H = 20, 10
    assert O.clamp_flow(W, H, 3, 4, 16, -8) == (16, -8)          # inside: unchanged
    assert O.clamp_flow(W, H, 3, 4, -100, 0) == (-24, 0)         # target x -> 0
    assert O.clamp_flow(W, H, 3, 4, 500, 500) == (8 * 16, 8 * 5)  # target -> (19, 9)
    assert O.clamp_flow(W, H, 0, 0, -1, -1) == (0, 0)


def test_cost_zero_at_true_integer_translation():
    pair = workloads.translation_pair(seed=4, with_square=False)
    S = 3
    f1 = O.features_all(pair.img1, S)
    f2 = O.features_all(pair.img2, S)
    W, H = pair.width, pair.height
    off = []
    for py in range(12, H - 12, 3):
        for px in range(12, W - 19, 5):
            assert O.cost(f1[0], f2[0], W, H, 0, px, py, 56, -32) == 0
            off.append(O.cost(f1[0], f2[0], W, H, 0, px, py, 56 + 8, -32))
    # one pixel off the truth costs something except inside flat rectangles
    assert np.mean(np.array(off) > 0) > 0.9


@pytest.mark.parametrize("C", [1, 3])
def test_cost_equals_scipy_bilinear_sad(C):
    rng = np.random.default_rng(21 + C)
    W, H = 37, 29
    for L in range(3):
        n = 1 << L
        WL, HL = -(-W // n), -(-H // n)
        f1 = rng.integers(-128, 128, (HL, WL, 9 * C), dtype=np.int8)
        f2 = rng.integers(-128, 128, (HL, WL, 9 * C), dtype=np.int8)
        for _ in range(60):
            gx, gy = int(rng.integers(0, WL)), int(rng.integers(0, HL))
            px, py = gx * n, gy * n
            Fx, Fy = int(rng.integers(-400, 400)), int(rng.integers(-300, 300))
            Fx, Fy = O.clamp_flow(W, H, px, py, Fx, Fy)
            # level coordinate: target in 1/8 px divided by n, rounded half up
            sx = np.floor((8 * px + Fx) / n + 0.5) / 8.0
            sy = np.floor((8 * py + Fy) / n + 0.5) / 8.0
            interp = np.array([ndimage.map_coordinates(f2[..., d].astype(np.float64),
                                                       [[sy], [sx]], order=1, mode="nearest")[0]
                               for d in range(9 * C)])
            expect = np.abs(64.0 * f1[gy, gx].astype(np.float64) - 64.0 * interp).sum()
            assert O.cost(f1, f2, W, H, L, px, py, Fx, Fy) == int(round(expect))


def test_cost_hand_computed_weights():
    # 2x2 level-0 map, one dim used; target (0.375 px, 0.5 px) -> f=3, g=4
    W = H = 2
    f1 = np.zeros((2, 2, 9), np.int8)
    f2 = np.zeros((2, 2, 9), np.int8)
    f1[0, 0, 0] = 10
    f2[0, 0, 0], f2[0, 1, 0], f2[1, 0, 0], f2[1, 1, 0] = 8, 16, -8, 40
    # weights (8-3)(8-4)=20, 3*4=12, 5*4=20, 3*4=12 for taps (0,0),(1,0),(0,1),(1,1)
    interp = 20 * 8 + 12 * 16 + 20 * (-8) + 12 * 40
    assert O.cost(f1, f2, W, H, 0, 0, 0, 3, 4) == abs(640 - interp)


# --------------------------------------------------------------------------
# seeding (Sec. 3.1 Eq. 1, Sec. 3.2 Eq. 4): exact top-l of squared distances
# --------------------------------------------------------------------------
@pytest.mark.parametrize("C,stride,alphabet", [(1, 1, 256), (3, 1, 256), (1, 2, 256),
                                               (1, 1, 3), (3, 2, 2)])
def test_seed_knn_equals_stable_argsort(C, stride, alphabet):
    rng = np.random.default_rng(31 + C + stride + alphabet)
    W, H, S, leaf = 19, 13, 3, 8
    lo = -alphabet // 2
    f1 = rng.integers(lo, lo + alphabet, (H, W, 9 * C)).astype(np.int8)
    f2 = rng.integers(lo, lo + alphabet, (H, W, 9 * C)).astype(np.int8)
    idx, dist = O.seed_knn(f1, f2, S, leaf, stride)
    N = 1 << (S - 1)
    cand_y, cand_x = np.mgrid[0:H:stride, 0:W:stride]
    cand_idx = (cand_y * W + cand_x).reshape(-1)
    cands = f2[cand_y, cand_x].reshape(-1, 9 * C).astype(np.int64)
    for gy in range(idx.shape[0]):
        for gx in range(idx.shape[1]):
            q = f1[gy * N, gx * N].astype(np.int64)
            d = ((cands - q) ** 2).sum(axis=1)
            order = np.lexsort((cand_idx, d))[:leaf]
            np.testing.assert_array_equal(idx[gy, gx], cand_idx[order])
            np.testing.assert_array_equal(dist[gy, gx], d[order])


# --------------------------------------------------------------------------
# propagation (Sec. 3.1 Eq. 2, directions), random search, coarse to fine
# --------------------------------------------------------------------------
def _stripes(W: int, H: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, 256, H).astype(np.uint8)
    return np.repeat(rows[:, None], W, axis=1)[None]


def test_sweep_prefers_horizontal_then_vertical_on_ties():
    # Horizontal stripes, frame 2 == frame 1: E depends on Fy only, and is 0
    # for Fy = 0.  Row 0 ends as [(0,8), (8,0), (8,0), (0,0)] (the last one
    # clamped); at (1,1) the vertical source (8,0) and the horizontal source
    # (0,0) tie at cost 0 and beat the empty point, and the horizontal one must
    # win (Sec. 4.5: horizontal propagation preferred on identical errors).
    W, H = 4, 3
    img = _stripes(W, H, 5)
    f = O.features_all(img, 1)[0]
    I = O.INVALID
    flow = np.full((H, W, 2), I, np.int16)
    flow[0, 0] = (0, 8)
    flow[0, 1] = (8, 0)
    flow[1, 0] = (0, 0)
    cost = np.full((H, W), O.INVALID_COST, np.int32)
    for y in range(H):
        for x in range(W):
            if flow[y, x, 0] != I:
                cost[y, x] = O.cost(f, f, W, H, 0, x, y, int(flow[y, x, 0]), int(flow[y, x, 1]))
    assert cost[0, 0] > 0 and cost[0, 1] == 0 and cost[1, 0] == 0
    out, oc, _ = O.sweep_level(f, f, W, H, 0, 0, flow, cost)
    np.testing.assert_array_equal(out[0], [[0, 8], [8, 0], [8, 0], [0, 0]])
    np.testing.assert_array_equal(out[1], [[0, 0], [0, 0], [0, 0], [0, 0]])
    assert np.all(oc[1:] == 0)


def test_sweep_current_loses_ties_constant_image():
    # all errors equal: every point takes a processed neighbour's flow, so the
    # whole grid ends with the flow of the sweep's first point (here (0, 0),
    # which needs no clamping anywhere), whatever each point held before
    W, H = 6, 5
    img = np.full((1, H, W), 90, np.uint8)
    f = O.features_all(img, 1)[0]
    rng = np.random.default_rng(3)
    yy, xx = np.mgrid[0:H, 0:W]
    first = {0: (0, 0), 1: (W - 1, H - 1), 2: (W - 1, 0), 3: (0, H - 1)}
    for d, (x0, y0) in first.items():
        flow = np.zeros((H, W, 2), np.int16)
        flow[..., 0] = 8 * (rng.integers(0, W, (H, W)) - xx)
        flow[..., 1] = 8 * (rng.integers(0, H, (H, W)) - yy)
        flow[y0, x0] = (0, 0)
        cost = np.zeros((H, W), np.int32)
        out, oc, ev = O.sweep_level(f, f, W, H, 0, d, flow, cost)
        assert np.all(out == 0) and np.all(oc == 0)
        assert ev == 2 * W * H - W - H


def test_sweep_order_follows_direction():
    # a single valid point at a corner spreads over the whole grid only when
    # the sweep starts there; otherwise it reaches just its own quadrant
    W, H = 5, 4
    img = np.full((1, H, W), 10, np.uint8)
    f = O.features_all(img, 1)[0]
    corners = {0: (0, 0), 1: (W - 1, H - 1), 2: (W - 1, 0), 3: (0, H - 1)}
    for d, (cx, cy) in corners.items():
        for (x0, y0) in corners.values():
            flow = np.full((H, W, 2), O.INVALID, np.int16)
            cost = np.full((H, W), O.INVALID_COST, np.int32)
            flow[y0, x0] = (0, 0)
            cost[y0, x0] = 0
            out, _, _ = O.sweep_level(f, f, W, H, 0, d, flow, cost)
            filled = out[..., 0] != O.INVALID
            if (x0, y0) == (cx, cy):
                assert filled.all()
            else:
                assert not filled.all()
                # filled points lie in the quadrant downstream of the seed
                ys, xs = np.nonzero(filled)
                sx = 1 if d in (0, 3) else -1
                sy = 1 if d in (0, 2) else -1
                assert np.all((xs - x0) * sx >= 0) and np.all((ys - y0) * sy >= 0)


def test_random_search_step_matches_philox_offsets():
    pair = workloads.translation_pair(seed=6)
    W, H = pair.width, pair.height
    f1 = O.features_all(pair.img1, 2)
    f2 = O.features_all(pair.img2, 2)
    L, t, direction, R, seed, pid = 1, 2, 1, 8, 99, 5
    flow, cost, _ = O.match(O.Params(scales=2, iters=3), pair.img1, pair.img2, 0, 0,
                            until_level=1, until_sweeps=1)
    out, oc, ev = O.random_search_level(f1[1], f2[1], W, H, L, t, direction, R, seed, pid,
                                        flow, cost)
    n = 2
    Rn = R * n
    HL, WL = cost.shape
    assert ev == HL * WL
    for gy in range(HL):
        for gx in range(WL):
            px, py = gx * n, gy * n
            r = _philox([py * W + px, t, L, direction], [seed, pid], 32, _M32)
            ox = r[0] % (2 * Rn + 1) - Rn
            oy = r[1] % (2 * Rn + 1) - Rn
            cx, cy = O.clamp_flow(W, H, px, py, int(flow[gy, gx, 0]) + ox,
                                  int(flow[gy, gx, 1]) + oy)
            e = O.cost(f1[1], f2[1], W, H, L, px, py, cx, cy)
            if e < cost[gy, gx]:
                assert tuple(out[gy, gx]) == (cx, cy) and oc[gy, gx] == e
            else:
                assert tuple(out[gy, gx]) == tuple(flow[gy, gx]) and oc[gy, gx] == cost[gy, gx]


def test_first_sweep_fills_every_level():
    pair = workloads.translation_pair(seed=1)
    P = O.Params(scales=3, iters=4)
    for L in range(3):
        flow, cost, _ = O.match(P, pair.img1, pair.img2, 0, 0, until_level=L, until_sweeps=0)
        if L < 2:
            # entering a finer level only the points of the coarser grid are set
            valid = flow[..., 0] != O.INVALID
            yy, xx = np.mgrid[0:valid.shape[0], 0:valid.shape[1]]
            np.testing.assert_array_equal(valid, (xx % 2 == 0) & (yy % 2 == 0))
        flow, cost, _ = O.match(P, pair.img1, pair.img2, 0, 0, until_level=L, until_sweeps=1)
        assert np.all(flow[..., 0] != O.INVALID) and np.all(cost < O.INVALID_COST)


def test_costs_never_increase_and_cache_is_exact():
    pair = workloads.layered_pair(seed=8, width=96, height=64, channels=3, max_disp=20)
    P = O.Params(channels=3, scales=3, iters=5)
    f1 = O.features_all(pair.img1, 3)
    f2 = O.features_all(pair.img2, 3)
    W, H = pair.width, pair.height
    for L in range(3):
        prev = None
        for k in range(1, P.iters + 1):
            flow, cost, _ = O.match(P, pair.img1, pair.img2, 0, 3, until_level=L, until_sweeps=k)
            if prev is not None:
                assert np.all(cost <= prev)
            prev = cost
        n = 1 << L
        for gy in range(0, cost.shape[0], 3):
            for gx in range(0, cost.shape[1], 2):
                e = O.cost(f1[L], f2[L], W, H, L, gx * n, gy * n, int(flow[gy, gx, 0]),
                           int(flow[gy, gx, 1]))
                assert e == cost[gy, gx]


def test_eval_count_closed_form():
    # Sec. 4.3: 4 propagations (2 candidates each) + 3 random searches = 11
    # patch comparisons per point and scale; boundary points lack a source
    g = _golden("patch_comparisons.txt")
    iters, per_point = int(g["iters"]), int(g["comparisons_per_point"])
    assert per_point == 3 * iters - 1
    for (W, H, S, leaf) in [(128, 96, 3, 8), (45, 31, 2, 4), (33, 17, 4, 8)]:
        pair = workloads.random_pair(seed=W, width=W, height=H)
        P = O.Params(scales=S, iters=iters, seed_leaf=leaf)
        _, _, ev = O.match(P, pair.img1, pair.img2, 0, 0)
        dims = [O.level_dims(W, H, L) for L in range(S)]
        expect = leaf * dims[S - 1][0] * dims[S - 1][1]
        for L, (WL, HL) in enumerate(dims):
            expect += per_point * WL * HL - iters * (WL + HL)
            if L < S - 1:
                expect += dims[L + 1][0] * dims[L + 1][1]  # carried points re-evaluated
        assert ev == expect


# --------------------------------------------------------------------------
# whole method: invariants on synthetic pairs with known flow
# --------------------------------------------------------------------------
def _interior(W, H, shift, margin):
    yy, xx = np.mgrid[0:H, 0:W]
    sx, sy = shift
    return ((xx >= margin + max(0, -sx)) & (xx < W - margin - max(0, sx))
            & (yy >= margin + max(0, -sy)) & (yy < H - margin - max(0, sy)))


@pytest.mark.parametrize("seed", [1, 2])
def test_pure_translation_recovered_exactly(seed):
    pair = workloads.translation_pair(seed=seed, with_square=False)
    P = O.Params(scales=3, iters=4)
    W, H = pair.width, pair.height
    fwd, _, _ = O.match(P, pair.img1, pair.img2, 0, seed)
    bwd, _, _ = O.match(P, pair.img2, pair.img1, 1, seed)
    inner = _interior(W, H, (7, -4), 5 * 4)
    assert np.all(fwd[inner] == [56, -32])
    inner_b = _interior(W, H, (-7, 4), 5 * 4)
    assert np.all(bwd[inner_b] == [-56, 32])
    mask = O.filter_mask(fwd, bwd, 8)
    assert np.all(mask[inner] == 1)


def test_filter_on_exact_translation_flows():
    W, H = 40, 30
    fwd = np.zeros((H, W, 2), np.int16)
    fwd[..., 0], fwd[..., 1] = 56, -32
    bwd = -fwd
    yy, xx = np.mgrid[0:H, 0:W]
    visible = (xx + 7 < W) & (yy - 4 >= 0)
    np.testing.assert_array_equal(O.filter_mask(fwd, bwd, 8), visible.astype(np.uint8))


def test_filter_threshold_is_strict():
    W, H = 3, 1
    fwd = np.zeros((H, W, 2), np.int16)
    bwd = np.zeros((H, W, 2), np.int16)
    bwd[0, 0] = (8, 0)      # |d| = 8 = eps -> rejected
    bwd[0, 1] = (7, 3)      # 49 + 9 = 58 < 64 -> kept
    bwd[0, 2] = (0, -8)     # rejected
    np.testing.assert_array_equal(O.filter_mask(fwd, bwd, 8)[0], [0, 1, 0])
    # the backward flow is read at the nearest pixel of p + F (half up)
    fwd[0, 0] = (4, 0)      # 0.5 px -> pixel 1
    bwd[0, 1] = (-4, 0)
    assert O.filter_mask(fwd, bwd, 1)[0, 0] == 1
    fwd[0, 0] = (3, 0)      # 0.375 px -> pixel 0 (bwd (8,0): |3 + 8| >= 1)
    assert O.filter_mask(fwd, bwd, 1)[0, 0] == 0


def test_filter_rejects_invalid_and_outside():
    W, H = 4, 4
    fwd = np.zeros((H, W, 2), np.int16)
    bwd = np.zeros((H, W, 2), np.int16)
    fwd[1, 1] = (O.INVALID, O.INVALID)
    fwd[2, 2] = (8 * 5, 0)
    bwd[0, 3] = (O.INVALID, O.INVALID)
    fwd[0, 0] = (8 * 3, 0)
    m = O.filter_mask(fwd, bwd, 8)
    assert m[1, 1] == 0 and m[2, 2] == 0 and m[0, 0] == 0 and m[3, 3] == 1


def test_seeds_in_replace_search():
    pair = workloads.translation_pair(seed=2, with_square=False)
    P = O.Params(scales=3, iters=4)
    WS, HS = O.level_dims(pair.width, pair.height, 2)
    seeds = np.zeros((HS, WS, 2), np.int16)
    seeds[..., 0], seeds[..., 1] = 56, -32
    flow, _, _ = O.match(P, pair.img1, pair.img2, 0, 0, seeds_in=seeds, until_level=2,
                         until_sweeps=0)
    W, H = pair.width, pair.height
    # seeds are clamped per point, then kept
    for gy in range(HS):
        for gx in range(WS):
            assert tuple(flow[gy, gx]) == O.clamp_flow(W, H, 4 * gx, 4 * gy, 56, -32)
    fwd, _, _ = O.match(P, pair.img1, pair.img2, 0, 0, seeds_in=seeds)
    inner = _interior(W, H, (7, -4), 20)
    assert np.all(fwd[inner] == [56, -32])


# --------------------------------------------------------------------------
# Flow Fields+ schedules (Sec. 3.3, 3.4) and the two-way check (Sec. 3.7)
# --------------------------------------------------------------------------
def test_schedule_counts_match_the_paper():
    g = {k: int(v) for k, v in _golden("schedules.txt").items()}
    P = O.Params(schedule=1, scales=3)
    for L in range(3):
        n = P.sweeps(L)
        assert n == g["plus_sweeps"]
        rs = [t for t in range(n) if O.lib().ffo_schedule_rs_after(1, 4, L, t)]
        assert len(rs) == g["plus_random_searches"]
        wide = [t for t in range(n) if O.lib().ffo_schedule_radius_mult(1, L, t) == 2]
        assert wide == list(range(g["plus_wide_sweeps"]))
        assert all(O.lib().ffo_schedule_radius_mult(1, L, t) in (1, g["plus_wide_radius_factor"])
                   for t in range(n))
        # the 3 random searches of the wide phase follow its first 3 sweeps
        assert [t for t in rs if t < 4] == [0, 1, 2]
    F = O.Params(schedule=2, scales=3)
    assert F.sweeps(0) == g["fast_finest_sweeps"]
    assert sum(O.lib().ffo_schedule_rs_after(2, 4, 0, t) for t in range(4)) == \
        g["fast_finest_random_searches"]
    assert all(O.lib().ffo_schedule_radius_mult(2, 0, t) == 1 for t in range(4))
    assert F.sweeps(1) == g["plus_sweeps"] and F.sweeps(2) == g["plus_sweeps"]


def test_fast_x2_schedule_counts_match_the_paper():
    g = {k: int(v) for k, v in _golden("schedules.txt").items()}
    X = O.Params(schedule=3, scales=4)
    assert X.final_level() == g["x2_final_level"]
    assert 1 << X.final_level() == g["x2_match_region"]
    assert X.sweeps(0) == g["x2_finest_sweeps"]
    assert X.sweeps(1) == g["x2_second_sweeps"]
    assert sum(O.lib().ffo_schedule_rs_after(3, 4, 1, t) for t in range(4)) == \
        g["x2_second_random_searches"]
    assert all(O.lib().ffo_schedule_radius_mult(3, 1, t) == 1 for t in range(4))
    for L in (2, 3):
        assert X.sweeps(L) == g["plus_sweeps"]
        assert [O.lib().ffo_schedule_radius_mult(3, L, t) for t in range(12)] == \
            [O.lib().ffo_schedule_radius_mult(1, L, t) for t in range(12)]
    for sch in (0, 1, 2):
        assert O.Params(schedule=sch).final_level() == 0


@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_schedule_eval_count_closed_form(schedule):
    W, H, S, leaf = 45, 31, 3, 8
    pair = workloads.random_pair(seed=77, width=W, height=H)
    P = O.Params(scales=S, iters=4, seed_leaf=leaf, schedule=schedule)
    _, _, ev = O.match(P, pair.img1, pair.img2, 0, 0)
    dims = [O.level_dims(W, H, L) for L in range(S)]
    expect = leaf * dims[S - 1][0] * dims[S - 1][1]
    for L, (WL, HL) in enumerate(dims):
        if L < P.final_level():
            continue
        n = P.sweeps(L)
        rs = sum(O.lib().ffo_schedule_rs_after(schedule, 4, L, t) for t in range(n))
        expect += n * (2 * WL * HL - WL - HL) + rs * WL * HL
        if L < S - 1:
            expect += dims[L + 1][0] * dims[L + 1][1]
    assert ev == expect


def test_plus_schedule_composes_pinned_steps_with_wide_radius():
    # the first two sweeps of a Flow Fields+ level: sweep 0, search with 2R,
    # sweep 1 -- built from the single-step functions pinned above
    pair = workloads.translation_pair(seed=8, width=64, height=48)
    W, H = pair.width, pair.height
    P = O.Params(scales=2, iters=4, schedule=1, radius_q3=8)
    f1 = O.features_all(pair.img1, 2)
    f2 = O.features_all(pair.img2, 2)
    flow, cost, _ = O.match(P, pair.img1, pair.img2, 0, 4, until_level=1, until_sweeps=0)
    flow, cost, _ = O.sweep_level(f1[1], f2[1], W, H, 1, 0, flow, cost)
    flow, cost, _ = O.random_search_level(f1[1], f2[1], W, H, 1, 0, 0, 16, P.seed, 4, flow, cost)
    flow, cost, _ = O.sweep_level(f1[1], f2[1], W, H, 1, 1, flow, cost)
    rf, rc, _ = O.match(P, pair.img1, pair.img2, 0, 4, until_level=1, until_sweeps=2)
    # until_sweeps=2 includes the search after sweep 1, with 2R as well
    flow, cost, _ = O.random_search_level(f1[1], f2[1], W, H, 1, 1, 0, 16, P.seed, 4, flow, cost)
    np.testing.assert_array_equal(rf, flow)
    np.testing.assert_array_equal(rc, cost)


def test_two_way_filter_needs_both_backward_flows():
    W, H = 4, 1
    fwd = np.zeros((H, W, 2), np.int16)
    b1 = np.zeros((H, W, 2), np.int16)
    b2 = np.zeros((H, W, 2), np.int16)
    b2[0, 1] = (16, 0)         # pixel 1: consistent with b1 only
    b1[0, 2] = (0, 16)         # pixel 2: consistent with b2 only
    b1[0, 3] = (9, 0)          # pixel 3: consistent with neither
    b2[0, 3] = (0, 9)
    np.testing.assert_array_equal(O.filter_mask2(fwd, b1, b2, 8)[0], [1, 0, 0, 0])
    np.testing.assert_array_equal(O.filter_mask2(fwd, b1, b1, 8), O.filter_mask(fwd, b1, 8))


def test_fast_x2_is_flow_fields_plus_cut_short_at_the_second_scale():
    # coarser scales run exactly as Flow Fields+; the 2nd-finest scale is the
    # upsampled state followed by 4 sweeps with R and 3 random searches, made
    # of the single-step functions pinned above; the finest never runs
    pair = workloads.layered_pair(seed=5, width=72, height=52, channels=3, max_disp=10)
    W, H, S = pair.width, pair.height, 3
    X = O.Params(channels=3, scales=S, schedule=3, radius_q3=8, seed_stride=2)
    Pp = O.Params(channels=3, scales=S, schedule=1, radius_q3=8, seed_stride=2)
    for k in (0, 5, 12):
        a = O.match(X, pair.img1, pair.img2, 0, 3, until_level=2, until_sweeps=k)
        b = O.match(Pp, pair.img1, pair.img2, 0, 3, until_level=2, until_sweeps=k)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
    f1 = O.features_all(pair.img1, S)
    f2 = O.features_all(pair.img2, S)
    flow, cost, _ = O.match(X, pair.img1, pair.img2, 0, 3, until_level=1, until_sweeps=0)
    for t in range(4):
        flow, cost, _ = O.sweep_level(f1[1], f2[1], W, H, 1, t, flow, cost)
        if t < 3:
            flow, cost, _ = O.random_search_level(f1[1], f2[1], W, H, 1, t, 0, 8, X.seed, 3,
                                                  flow, cost)
    rf, rc, _ = O.match(X, pair.img1, pair.img2, 0, 3)
    assert rf.shape[:2] == O.level_dims(W, H, 1)[::-1]
    np.testing.assert_array_equal(rf, flow)
    np.testing.assert_array_equal(rc, cost)
    with pytest.raises(ValueError):
        O.match(X, pair.img1, pair.img2, 0, 3, until_level=0, until_sweeps=0)


def test_grid_filter_worked_example():
    # level-1 grid: point (x 2, y 2); a forward flow of exactly 1 px lies half
    # way between grid points 0 and 1 and rounds up to grid point 1
    fwd = np.zeros((1, 4, 2), np.int16)
    bwd = np.zeros((1, 4, 2), np.int16)
    fwd[0, 0] = (8, 0)      # -> grid 1, bwd there (-8, 0): consistent
    fwd[0, 1] = (4, 0)      # -> grid 1 (itself), bwd (-8, 0): |(-4, 0)| < 1 px
    fwd[0, 2] = (-9, 0)     # -> grid 1 (2*2*8 - 9 = 23 Q3 -> 1.44 grid), bwd (-8,0): far
    fwd[0, 3] = (8, 0)      # -> grid 4: outside
    bwd[0, 1] = (-8, 0)
    bwd[0, 2] = (9, 0)
    np.testing.assert_array_equal(O.filter_mask(fwd, bwd, 8, level=1)[0], [1, 1, 0, 0])
    # on the pixel grid point 1 reads pixel 2, whose (9, 0) is inconsistent
    np.testing.assert_array_equal(O.filter_mask(fwd, bwd, 8, level=0)[0], [1, 0, 0, 0])


def test_grid_filter_is_the_pixel_filter_on_block_constant_flows():
    # flows constant on 2x2 blocks with whole 2-px displacements land on even
    # pixels, so the level-1 check is the pixel check subsampled
    rng = np.random.default_rng(4)
    W, H = 30, 22
    blocks = lambda a: np.repeat(np.repeat(a, 2, axis=0), 2, axis=1)[:H, :W]
    fwd = blocks(16 * rng.integers(-3, 4, (H // 2, W // 2, 2))).astype(np.int16)
    bwd = blocks(16 * rng.integers(-3, 4, (H // 2, W // 2, 2))).astype(np.int16)
    bwd[fwd[..., 0] > 16] = -fwd[fwd[..., 0] > 16]
    full = O.filter_mask(fwd, bwd, 12)
    grid = O.filter_mask(fwd[::2, ::2], bwd[::2, ::2], 12, level=1)
    assert 0 < grid.sum() < grid.size
    np.testing.assert_array_equal(grid, full[::2, ::2])


# --------------------------------------------------------------------------
# region filter (Sec. 3.7)
# --------------------------------------------------------------------------
def _region_filter_by_graph(fwd, mask, s):
    """The rule restated with networkx's connected components."""
    nx = pytest.importorskip("networkx")
    H, W, _ = fwd.shape
    f = fwd.astype(np.int64)
    close = lambda a, b: ((f[a] - f[b]) ** 2).sum() < 24 * 24
    g = nx.Graph()
    for y in range(H):
        for x in range(W):
            if mask[y, x]:
                g.add_node((y, x))
    for y in range(H):
        for x in range(W):
            for yy, xx in ((y, x + 1), (y + 1, x)):
                if yy < H and xx < W and mask[y, x] and mask[yy, xx] and close((y, x), (yy, xx)):
                    g.add_edge((y, x), (yy, xx))
    out = mask.copy()
    for comp in nx.connected_components(g):
        if len(comp) >= s:
            continue
        joinable = False
        for (y, x) in comp:
            for yy, xx in ((y, x + 1), (y, x - 1), (y + 1, x), (y - 1, x)):
                if 0 <= yy < H and 0 <= xx < W and not mask[yy, xx] \
                        and fwd[yy, xx, 0] != -32768 and close((y, x), (yy, xx)):
                    joinable = True
        if joinable:
            for (y, x) in comp:
                out[y, x] = 0
    return out


def test_region_filter_worked_examples():
    row = lambda fx: np.array([[[v, 0] for v in fx]], np.int16)
    m = np.array([[1, 1, 1, 1, 1, 0]], np.uint8)
    # pixels 3-4 form a 2-pixel region whose removed neighbour 5 is far: kept
    f = row([0, 0, 0, 100, 100, 0])
    np.testing.assert_array_equal(O.region_filter(f, m, 3), m)
    # the removed neighbour is 2 px away from pixel 4: the region is removed
    f = row([0, 0, 0, 100, 100, 116])
    np.testing.assert_array_equal(O.region_filter(f, m, 3)[0], [1, 1, 1, 0, 0, 0])
    # ... unless it is not smaller than s
    np.testing.assert_array_equal(O.region_filter(f, m, 2), m)
    # exactly 3 px apart is not "below 3 pixels": pixels 3 and 4 split, and
    # only the single pixel 4 joins the outlier
    f = row([0, 0, 0, 100, 124, 140])
    np.testing.assert_array_equal(O.region_filter(f, m, 3)[0], [1, 1, 1, 1, 0, 0])
    # an unset flow joins nothing
    f = row([0, 0, 0, 100, 100, -32768])
    np.testing.assert_array_equal(O.region_filter(f, m, 3), m)
    # diagonal neighbours do not connect: the 1-pixel region at (1, 1) has
    # only a diagonal removed neighbour, and stays
    f = np.zeros((2, 2, 2), np.int16)
    only_11 = np.array([[0, 0], [0, 1]], np.uint8)
    # (0, 1) and (1, 0) are removed 4-neighbours with the same flow: removed
    np.testing.assert_array_equal(O.region_filter(f, only_11, 5), [[0, 0], [0, 0]])
    # with those two unset, only the diagonal (0, 0) remains: kept
    f[0, 1] = f[1, 0] = (-32768, -32768)
    np.testing.assert_array_equal(O.region_filter(f, only_11, 5), only_11)


def test_region_filter_drifting_region_counts_whole():
    # flows rising 2 px per pixel: one region of 10 (neighbours close, ends
    # 18 px apart); with s = 10 it is not small, with s = 11 it is
    f = np.array([[[16 * i, 0] for i in range(10)] + [[16 * 9 + 8, 0]]], np.int16)
    m = np.array([[1] * 10 + [0]], np.uint8)
    np.testing.assert_array_equal(O.region_filter(f, m, 10), m)
    np.testing.assert_array_equal(O.region_filter(f, m, 11)[0], [0] * 11)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_region_filter_equals_connected_components(seed):
    rng = np.random.default_rng(seed)
    H, W = 23, 31
    blocks = rng.integers(-6, 7, (H // 4 + 1, W // 4 + 1, 2)) * 20
    f = np.repeat(np.repeat(blocks, 4, 0), 4, 1)[:H, :W] + rng.integers(-14, 15, (H, W, 2))
    f = f.astype(np.int16)
    f[rng.random((H, W)) < 0.05] = (-32768, -32768)
    m = (rng.random((H, W)) < 0.8).astype(np.uint8)
    m[f[..., 0] == -32768] = 0
    for s in (1, 4, 15, 60):
        got = O.region_filter(f, m, s)
        np.testing.assert_array_equal(got, _region_filter_by_graph(f, m, s), err_msg=f"s {s}")
        assert np.all(got <= m)
    assert (O.region_filter(f, m, 60) != m).any()


# --------------------------------------------------------------------------
# sparsification (Sec. 3.7-3.8)
# --------------------------------------------------------------------------
def test_sparsify_worked_examples():
    fwd = np.zeros((2, 2, 2), np.int16)
    b1 = np.array([[[3, 4], [0, 4]], [[4, 0], [5, 12]]], np.int16)   # errors 5, 4, 4, 13
    m = np.ones((2, 2), np.uint8)
    # smallest error 4 twice: the first in raster order wins
    np.testing.assert_array_equal(O.sparsify(fwd, b1, None, m, 2, 1), [[0, 1], [0, 0]])
    np.testing.assert_array_equal(O.sparsify(fwd, b1, None, m, 2, 4), [[0, 1], [0, 0]])
    np.testing.assert_array_equal(O.sparsify(fwd, b1, None, m, 2, 5), np.zeros((2, 2)))
    # two backward flows: the errors add (5 + 0, 4 + 3, 4 + 5, 13 + 0)
    b2 = np.array([[[0, 0], [3, 0]], [[3, 4], [0, 0]]], np.int16)
    np.testing.assert_array_equal(O.sparsify(fwd, b1, b2, m, 2, 1), [[1, 0], [0, 0]])
    # a rejected point is never chosen
    m2 = m.copy()
    m2[0, 1] = 0
    np.testing.assert_array_equal(O.sparsify(fwd, b1, None, m2, 2, 3), [[0, 0], [1, 0]])
    np.testing.assert_array_equal(O.sparsify(fwd, b1, None, m2, 2, 4), np.zeros((2, 2)))


def test_sparsify_partial_cells_and_trivial_cells():
    rng = np.random.default_rng(5)
    H, W = 7, 11
    fwd = rng.integers(-3, 4, (H, W, 2)).astype(np.int16)
    b1 = rng.integers(-9, 10, (H, W, 2)).astype(np.int16)
    m = (rng.random((H, W)) < 0.7).astype(np.uint8)
    # q = 1, e = 1: every kept point is its own cell
    np.testing.assert_array_equal(O.sparsify(fwd, b1, None, m, 1, 1), m)
    # q = 3: cells of 3 x 3, the last column of cells 2 wide, the last row 1 high
    for e in (1, 3, 5):
        out = O.sparsify(fwd, b1, None, m, 3, e)
        assert np.all(out <= m)
        for cy in range(0, H, 3):
            for cx in range(0, W, 3):
                cell_m = m[cy:cy + 3, cx:cx + 3]
                cell_o = out[cy:cy + 3, cx:cx + 3]
                assert cell_o.sum() == (1 if cell_m.sum() >= e else 0)


def test_sparsify_level1_reads_the_nearest_grid_point():
    # the backward flow is read where the grid consistency check reads it:
    # on the level-1 grid F = (4, 0) stays at point 0 (error |4 + 20|) and
    # F = (-4, 0) at point 1 (error |-4 - 4|); on the pixel grid F = (4, 0)
    # reaches pixel 1 (error |4 - 4| = 0)
    fwd = np.array([[[4, 0], [-4, 0]]], np.int16)
    b1 = np.array([[[20, 0], [-4, 0]]], np.int16)
    m = np.ones((1, 2), np.uint8)
    np.testing.assert_array_equal(O.sparsify(fwd, b1, None, m, 2, 1, level=1), [[0, 1]])
    np.testing.assert_array_equal(O.sparsify(fwd, b1, None, m, 2, 1, level=0), [[1, 0]])


# --------------------------------------------------------------------------
# exhaustive matching (Sec. 4: the exact nearest-neighbour field) and the
# Eq. 1 rerank.  The exhaustive cost table is built here with scipy's bilinear
# interpolation, independently of the oracle's cost function.
# --------------------------------------------------------------------------
def _exhaustive_table(f2L: np.ndarray, W: int, H: int) -> np.ndarray:
    """64 x the bilinear interpolation of level-0 features at every Q3 target
    inside the frame: int32 [8(H-1)+1][8(W-1)+1][D]."""
    ty, tx = np.mgrid[0:8 * (H - 1) + 1, 0:8 * (W - 1) + 1]
    coords = np.stack([ty.ravel() / 8.0, tx.ravel() / 8.0])
    D = f2L.shape[-1]
    out = np.empty(ty.shape + (D,), np.int32)
    for d in range(D):
        v = ndimage.map_coordinates(f2L[..., d].astype(np.float64), coords, order=1,
                                    mode="nearest")
        out[..., d] = np.rint(64.0 * v).reshape(ty.shape).astype(np.int32)
    return out


def _costs_at(table: np.ndarray, f1L: np.ndarray, px: int, py: int) -> np.ndarray:
    """E(p, t) for every Q3 target t of the table: int64 [TY][TX]."""
    q = 64 * f1L[py, px].astype(np.int32)
    return np.abs(table - q).sum(axis=-1, dtype=np.int64)


def _flow_index(px, py, fx, fy):
    return 8 * py + int(fy), 8 * px + int(fx)


@pytest.mark.parametrize("C,W,H,S", [(1, 32, 24, 1), (1, 31, 23, 3), (3, 24, 20, 2),
                                     (3, 32, 24, 3)])
def test_final_costs_against_exhaustive_search(C, W, H, S):
    # every final flow's cached cost is the independently computed E of that
    # flow, and no point ends below the global minimum over all Q3 targets
    pair = workloads.layered_pair(seed=40 + C + S, width=W, height=H, channels=C, max_disp=6.0)
    P = O.Params(channels=C, scales=S, iters=4)
    f1 = O.features_all(pair.img1, S)
    f2 = O.features_all(pair.img2, S)
    flow, cost, _ = O.match_features(P, f1, f2, W, H, 0, 3)
    table = _exhaustive_table(f2[0], W, H)
    for py in range(H):
        for px in range(W):
            E = _costs_at(table, f1[0], px, py)
            fx, fy = flow[py, px]
            assert fx != O.INVALID
            iy, ix = _flow_index(px, py, fx, fy)
            assert 0 <= iy < E.shape[0] and 0 <= ix < E.shape[1]
            assert cost[py, px] == E[iy, ix]
            assert cost[py, px] >= E.min()


@pytest.mark.parametrize("C", [1, 3])
def test_translation_is_the_unique_exhaustive_minimum_and_is_found(C):
    # on smoothed noise under an integer translation the true flow costs 0 and
    # is the only zero of E on the interior: the exact nearest-neighbour field,
    # and the method's result, are that flow
    W, H = 32, 24
    pair = workloads.translation_pair(seed=11, width=W, height=H, shift=(3, -2), rects=0,
                                      with_square=False)
    img1, img2 = pair.img1, pair.img2
    if C == 3:
        rng = np.random.default_rng(5)
        img1 = np.concatenate([img1, img1[:, :, ::-1], rng.permutation(img1.ravel()).reshape(img1.shape)])
        img2 = np.concatenate([img2, img2[:, :, ::-1], np.zeros_like(img2)])
        img2[2] = np.roll(np.roll(img1[2], -2, axis=0), 3, axis=1)   # same shift on channel 3
        img2[1] = np.roll(np.roll(img1[1], -2, axis=0), 3, axis=1)
    S = 2
    P = O.Params(channels=C, scales=S, iters=4)
    f1 = O.features_all(img1, S)
    f2 = O.features_all(img2, S)
    flow, cost, _ = O.match_features(P, f1, f2, W, H, 0, 0)
    table = _exhaustive_table(f2[0], W, H)
    checked = 0
    for py in range(7, H - 7):
        for px in range(7, W - 7):
            E = _costs_at(table, f1[0], px, py)
            zeros = np.argwhere(E == 0)
            assert zeros.tolist() == [[8 * py - 16, 8 * px + 24]]
            assert tuple(flow[py, px]) == (24, -16) and cost[py, px] == 0
            checked += 1
    assert checked >= 100


@pytest.mark.parametrize("C,iters", [(1, 4), (3, 4), (1, 3), (3, 6)])
def test_last_sweep_leaves_a_fixed_point_of_its_sources(C, iters):
    # no random search follows the last sweep, so each final flow is the
    # argmin over [current, vertical source, horizontal source] with the
    # sources' final values, and on equal cost the later candidate
    # (horizontal, then vertical) is the one kept (Sec. 3.1 Eq. 2, Sec. 4.5)
    W, H = 28, 20
    pair = workloads.layered_pair(seed=77 + C, width=W, height=H, channels=C, max_disp=5.0)
    P = O.Params(channels=C, scales=2, iters=iters)
    f1 = O.features_all(pair.img1, 2)
    f2 = O.features_all(pair.img2, 2)
    flow, cost, _ = O.match_features(P, f1, f2, W, H, 0, 1)
    d = (iters - 1) % 4
    dx = 1 if d in (0, 3) else -1
    dy = 1 if d in (0, 2) else -1
    table = _exhaustive_table(f2[0], W, H)
    ties = 0
    for py in range(H):
        for px in range(W):
            E = _costs_at(table, f1[0], px, py)
            here = E[_flow_index(px, py, *flow[py, px])]
            for sx, sy in ((px, py - dy), (px - dx, py)):          # vertical, horizontal
                if not (0 <= sx < W and 0 <= sy < H):
                    continue
                cx, cy = O.clamp_flow(W, H, px, py, *map(int, flow[sy, sx]))
                Ec = E[_flow_index(px, py, cx, cy)]
                assert here <= Ec
            hx, hy = px - dx, py
            if 0 <= hx < W:
                cx, cy = O.clamp_flow(W, H, px, py, *map(int, flow[hy, hx]))
                if E[_flow_index(px, py, cx, cy)] == here:
                    assert tuple(flow[py, px]) == (cx, cy)   # horizontal wins a tie
                    ties += 1
    assert ties > 0


def _rerank_case(cands):
    """Features for a 1-row frame: query pixel 0 is the zero vector; image 2
    holds the given 9-d vectors from pixel 1 on, after a far vector at 0."""
    W = len(cands) + 2
    f1 = np.zeros((1, W, 9), np.int8)
    f2 = np.full((1, W, 9), 60, np.int8)
    f1[0, 1:] = 90
    for i, c in enumerate(cands):
        f2[0, 1 + i] = c
    return f1, f2, W


def test_rerank_takes_a_later_rank_with_lower_cost():
    # Eq. 1: among the seeding candidates the one with the lowest matching
    # error wins, even when it is not the nearest WHT vector
    a = [1] * 9               # |a|^2 = 9,  sum|a| = 9
    b = [3, 1] + [0] * 7      # |b|^2 = 10, sum|b| = 4
    f1, f2, W = _rerank_case([a, b])
    idx, dist = O.seed_knn(f1, f2, 1)
    assert idx[0, 0, 0] == 1 and idx[0, 0, 1] == 2 and dist[0, 0, 0] < dist[0, 0, 1]
    P = O.Params(channels=1, scales=1, iters=1)
    flow, cost, _ = O.match_features(P, [f1], [f2], W, 1, 0, 0, until_level=0, until_sweeps=0)
    assert tuple(flow[0, 0]) == (16, 0) and cost[0, 0] == 64 * 4


def test_rerank_keeps_the_earlier_rank_on_equal_cost():
    # equal matching errors: the nearer WHT vector (the earlier rank) stays,
    # although the other candidate has the smaller pixel index
    a = [2] + [0] * 8         # pixel 1: |a|^2 = 4, sum|a| = 2
    b = [1, 1] + [0] * 7      # pixel 2: |b|^2 = 2, sum|b| = 2
    f1, f2, W = _rerank_case([a, b])
    idx, _ = O.seed_knn(f1, f2, 1)
    assert idx[0, 0, 0] == 2 and idx[0, 0, 1] == 1
    P = O.Params(channels=1, scales=1, iters=1)
    flow, cost, _ = O.match_features(P, [f1], [f2], W, 1, 0, 0, until_level=0, until_sweeps=0)
    assert tuple(flow[0, 0]) == (16, 0) and cost[0, 0] == 64 * 2


def test_repetitive_object_needs_the_coarse_scale():
    # Sec. 4.5: a repetitive pattern is matched flawlessly once the influence
    # area of the coarsest scale is larger than the ambiguous pattern.  A 36 px
    # object with a 12 px period moves on its own: 8 px windows (S = 1) match
    # it at wrong period shifts, the 64 px windows of S = 4 see its outline.
    cases = [(s, sh) for s in (5, 6, 7) for sh in ((11, 6), (-9, 5))]
    exact = {1: 0, 4: 0}
    wrong = {1: 0, 4: 0}
    for seed, shift in cases:
        pair = workloads.periodic_object_pair(seed=seed, shift=shift)
        obj = np.all(pair.flow == shift, axis=2)
        ys, xs = np.nonzero(obj)
        core = np.zeros_like(obj)
        core[ys.min() + 4:ys.max() - 3, xs.min() + 4:xs.max() - 3] = True
        for S in (1, 4):
            P = O.Params(channels=1, scales=S, iters=4)
            flow, _, _ = O.match(P, pair.img1, pair.img2, 0, 0)
            bad = np.any(flow != 8 * np.asarray(shift), axis=2) & core
            exact[S] += int(not bad.any())
            wrong[S] += int(bad.sum())
    assert exact[1] == 0 and exact[4] >= 4
    assert wrong[4] * 4 < wrong[1]
