"""The seeded input generators (CPU): the colour conversion against textbook
CIELab values, and each generator against the ground truth it states.

These are the inputs of every parity test and of the benchmark, so the recipe
the design notes give for them (sizes, motions, displacement bounds,
occlusion) is checked here rather than taken on trust.
"""
import numpy as np
import pytest

from paper_1703_02563_gb300 import workloads

# sRGB (D65) primaries and white/black in CIELab, the values tabulated in the
# usual colour-science references (L*, a*, b*).
_LAB_TEXTBOOK = [
    ((1.0, 1.0, 1.0), (100.0, 0.0, 0.0)),
    ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)),
    ((1.0, 0.0, 0.0), (53.2408, 80.0925, 67.2032)),
    ((0.0, 1.0, 0.0), (87.7347, -86.1827, 83.1793)),
    ((0.0, 0.0, 1.0), (32.2970, 79.1875, -107.8602)),
]


@pytest.mark.parametrize("rgb,lab", _LAB_TEXTBOOK)
def test_lab_textbook_values(rgb, lab):
    # stored as L*·255/100, a*+128, b*+128, rounded and saturated to uint8
    img = np.array(rgb, np.float64).reshape(3, 1, 1)
    got = workloads.rgb_to_lab_u8(img)[:, 0, 0]
    L, a, b = lab
    want = np.clip(np.rint([L * 2.55, a + 128.0, b + 128.0]), 0, 255).astype(np.uint8)
    np.testing.assert_array_equal(got, want)


def test_lab_gray_axis_is_achromatic_and_monotone():
    v = np.linspace(0.0, 1.0, 256)
    img = np.broadcast_to(v, (3, 1, 256)).copy()
    lab = workloads.rgb_to_lab_u8(img)[:, 0, :]
    np.testing.assert_array_equal(lab[1], 128)
    np.testing.assert_array_equal(lab[2], 128)
    assert np.all(np.diff(lab[0].astype(int)) >= 0)
    # sRGB 0.5 has L* = 53.39 (CIE 1976 lightness of Y = 0.2140)
    mid = workloads.rgb_to_lab_u8(np.full((3, 1, 1), 0.5))[0, 0, 0]
    assert mid == round(53.389 * 2.55)


def _constancy_violations(pair):
    """Visible pixels of an integer-flow pair whose frame-2 value differs."""
    H, W = pair.height, pair.width
    yy, xx = np.mgrid[0:H, 0:W]
    fx = pair.flow[..., 0].astype(np.int64)
    fy = pair.flow[..., 1].astype(np.int64)
    vis = ~pair.occ
    tx, ty = xx + fx, yy + fy
    assert np.all((tx[vis] >= 0) & (tx[vis] < W) & (ty[vis] >= 0) & (ty[vis] < H))
    a = pair.img1[:, yy[vis], xx[vis]]
    b = pair.img2[:, ty[vis], tx[vis]]
    return int(np.count_nonzero(np.any(a != b, axis=0))), int(vis.sum())


@pytest.mark.parametrize("seed", [1, 4, 13])
def test_translation_pair_ground_truth(seed):
    pair = workloads.translation_pair(seed=seed)
    assert pair.img1.shape == (1, 96, 128) and pair.img1.dtype == np.uint8
    fl = pair.flow.reshape(-1, 2)
    # global (+7, -4) shift; one 24x24 square moved by (+18, +11)
    assert np.count_nonzero(np.all(fl == (18, 11), axis=1)) == 24 * 24
    assert np.count_nonzero(np.all(fl == (7, -4), axis=1)) == 128 * 96 - 24 * 24
    bad, vis = _constancy_violations(pair)
    assert bad == 0 and vis > 0.8 * 128 * 96
    # the shifted-out strips are occluded, the moved square never is
    sq = np.all(pair.flow == (18, 11), axis=2)
    assert not pair.occ[sq].any()
    assert (pair.occ | sq)[:, -7:].all() and (pair.occ | sq)[:4, :].all()


def test_periodic_pair_ground_truth():
    pair = workloads.periodic_pair()
    bad, vis = _constancy_violations(pair)
    assert bad == 0 and vis > 0
    # the texture repeats with the stated period
    np.testing.assert_array_equal(pair.img1[:, :, :-12], pair.img1[:, :, 12:])
    np.testing.assert_array_equal(pair.img1[:, :-12, :], pair.img1[:, 12:, :])


@pytest.mark.parametrize("seed,shift", [(5, (11, 6)), (6, (-9, 5))])
def test_periodic_object_pair_ground_truth(seed, shift):
    pair = workloads.periodic_object_pair(seed=seed, shift=shift)
    bad, vis = _constancy_violations(pair)
    assert bad == 0 and vis > 0.8 * 95 * 95
    obj = np.all(pair.flow == shift, axis=2)
    assert obj.sum() == 36 * 36 and not pair.occ[obj].any()
    # the object's texture repeats with its period inside the object
    ys, xs = np.nonzero(obj)
    y0, x0 = ys.min(), xs.min()
    inner = pair.img1[0, y0:y0 + 36, x0:x0 + 36]
    np.testing.assert_array_equal(inner[:, :-12], inner[:, 12:])
    np.testing.assert_array_equal(inner[:-12, :], inner[12:, :])


def test_layered_pair_motion_bounds():
    max_disp = 30.0
    pair = workloads.layered_pair(seed=8, width=160, height=96, channels=3, max_disp=max_disp)
    assert pair.img1.shape == (3, 96, 160) and pair.img2.dtype == np.uint8
    mag = np.hypot(pair.flow[..., 0], pair.flow[..., 1])
    # each layer's affine displacement is at most max_disp at the frame corners, and
    # |displacement| is convex in the position, so it is bounded everywhere
    assert mag.max() <= max_disp + 1e-9
    assert mag.max() > 0.2 * max_disp
    # some, but not most, pixels occluded
    assert 0.0 < pair.occ.mean() < 0.5


def test_layered_pair_visible_pixels_keep_their_colour():
    # frame 2 re-samples the moved layers analytically, so a visible pixel's colour
    # reappears at its (sub-pixel) target: compare the pixels whose target is within
    # 0.05 px of a pixel centre against that frame-2 pixel
    pair = workloads.layered_pair(seed=8, width=160, height=96, channels=3, max_disp=30.0)
    H, W = pair.height, pair.width
    yy, xx = np.mgrid[0:H, 0:W]
    tx = xx + pair.flow[..., 0]
    ty = yy + pair.flow[..., 1]
    near = (np.abs(tx - np.rint(tx)) < 0.05) & (np.abs(ty - np.rint(ty)) < 0.05) & ~pair.occ
    assert near.sum() > 50
    txi = np.rint(tx[near]).astype(int)
    tyi = np.rint(ty[near]).astype(int)
    d = np.abs(pair.img1[:, yy[near], xx[near]].astype(int)
               - pair.img2[:, tyi, txi].astype(int)).max(axis=0)
    # most such pixels match within a few codes (polygon edges may not)
    assert np.median(d) <= 3


def test_expansion_pair_displacement_bound():
    max_disp = 60.0
    pair = workloads.expansion_pair(seed=3, width=311, height=94, max_disp=max_disp)
    assert pair.img1.shape == (1, 94, 311)
    mag = np.hypot(pair.flow[..., 0], pair.flow[..., 1])
    # the largest ground displacement (the bottom corner farthest from the focus of
    # expansion) is max_disp; nothing in the frame moves farther
    assert mag.max() <= max_disp + 1e-6
    assert mag.max() >= 0.9 * max_disp
    # expansion: every flow vector points away from one focus
    H, W = pair.height, pair.width
    yy, xx = np.mgrid[0:H, 0:W]
    moving = mag > 1.0
    fx, fy = pair.flow[..., 0][moving], pair.flow[..., 1][moving]
    # the focus lies on every flow line: solve for it by least squares and check residuals
    A = np.stack([fy, -fx], axis=1)
    rhs = fy * xx[moving] - fx * yy[moving]
    foe, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    resid = (A @ foe - rhs) / np.hypot(fx, fy)
    assert np.abs(resid).max() < 1e-6
    assert 0.4 * W < foe[0] < 0.6 * W


@pytest.mark.parametrize("gen,kw", [
    (workloads.translation_pair, dict()),
    (workloads.layered_pair, dict(width=64, height=48, max_disp=10.0)),
    (workloads.random_pair, dict(width=33, height=17, channels=3)),
])
def test_generators_are_seeded(gen, kw):
    a, b, c = gen(seed=5, **kw), gen(seed=5, **kw), gen(seed=6, **kw)
    np.testing.assert_array_equal(a.img1, b.img1)
    np.testing.assert_array_equal(a.img2, b.img2)
    np.testing.assert_array_equal(a.flow, b.flow)
    assert not np.array_equal(a.img1, c.img1)
