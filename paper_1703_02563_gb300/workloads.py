"""Seeded synthetic frame pairs shaped like the paper's evaluation data.

The paper evaluates on MPI-Sintel and KITTI (Sec. 4); neither dataset is
available here, so these generators stand in for them.  They produce uint8
frames plus ground-truth flow and an occlusion mask.  This module holds no
arithmetic of the matching method itself: it only draws textures, moves them
and renders the second frame, so both the CUDA path and the oracle can be fed
the same bytes.

Every generator is a pure function of its seed.  Colour frames are returned
already converted to 8-bit CIELab (the paper matches in CIELab, Sec. 3.1):
L*·255/100, a*+128, b*+128, rounded half-to-even and saturated.  Frames are
planar ``[C][H][W]`` uint8 arrays; flows are float64 ``[H][W][2]`` in pixels
(x, y); ``occ`` is a bool ``[H][W]`` array, True where the pixel's match is
not visible in frame 2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy import ndimage


@dataclass
class FramePair:
    img1: np.ndarray      # uint8 [C][H][W]
    img2: np.ndarray      # uint8 [C][H][W]
    flow: np.ndarray      # float64 [H][W][2], ground truth, pixels
    occ: np.ndarray       # bool [H][W]
    name: str

    @property
    def channels(self) -> int:
        return int(self.img1.shape[0])

    @property
    def width(self) -> int:
        return int(self.img1.shape[2])

    @property
    def height(self) -> int:
        return int(self.img1.shape[1])


# ----------------------------------------------------------------------------
# texture primitives, evaluated at arbitrary (texture-space) coordinates
# ----------------------------------------------------------------------------
class _ValueNoise:
    """Multi-octave value noise on periodic random lattices (smoothstep blend)."""

    def __init__(self, rng: np.random.Generator, channels: int, octaves: int,
                 base_period: float, persistence: float = 0.6, table: int = 1024):
        self.tables = rng.random((octaves, channels, table, table))
        self.periods = [base_period / (2.0 ** o) for o in range(octaves)]
        self.amps = [persistence ** o for o in range(octaves)]
        self.offsets = rng.random((octaves, 2)) * table
        self.table = table

    def __call__(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        t = self.table
        out = 0.0
        norm = 0.0
        for o, (per, amp) in enumerate(zip(self.periods, self.amps)):
            gx = x / per + self.offsets[o, 0]
            gy = y / per + self.offsets[o, 1]
            x0 = np.floor(gx)
            y0 = np.floor(gy)
            fx = gx - x0
            fy = gy - y0
            fx = fx * fx * (3.0 - 2.0 * fx)
            fy = fy * fy * (3.0 - 2.0 * fy)
            ix0 = np.mod(x0.astype(np.int64), t)
            iy0 = np.mod(y0.astype(np.int64), t)
            ix1 = np.mod(ix0 + 1, t)
            iy1 = np.mod(iy0 + 1, t)
            tab = self.tables[o]
            v = (tab[:, iy0, ix0] * (1 - fx) * (1 - fy) + tab[:, iy0, ix1] * fx * (1 - fy)
                 + tab[:, iy1, ix0] * (1 - fx) * fy + tab[:, iy1, ix1] * fx * fy)
            out = out + amp * v
            norm += amp
        return out / norm  # [C][...] in [0,1]


class _StarPolygons:
    """Filled star-shaped polygons with flat colours, drawn in texture space."""

    def __init__(self, rng: np.random.Generator, channels: int, count: int,
                 extent: tuple[float, float, float, float], rmin: float, rmax: float,
                 verts: tuple[int, int] = (5, 9)):
        x0, y0, x1, y1 = extent
        self.polys = []
        for _ in range(count):
            nv = int(rng.integers(verts[0], verts[1] + 1))
            ang = np.sort(rng.random(nv) * 2 * np.pi)
            base = rng.uniform(rmin, rmax)
            rad = base * rng.uniform(0.45, 1.0, nv)
            cx = rng.uniform(x0, x1)
            cy = rng.uniform(y0, y1)
            col = rng.random(channels)
            self.polys.append((cx, cy, ang, rad, col))

    def paint(self, x: np.ndarray, y: np.ndarray, base: np.ndarray) -> np.ndarray:
        out = base.copy()
        for cx, cy, ang, rad, col in self.polys:
            dx = x - cx
            dy = y - cy
            r = np.hypot(dx, dy)
            if not np.any(r < rad.max()):
                continue
            th = np.mod(np.arctan2(dy, dx), 2 * np.pi)
            # radius of the polygon boundary along angle th (linear between vertices)
            a_ext = np.concatenate([ang[-1:] - 2 * np.pi, ang, ang[:1] + 2 * np.pi])
            r_ext = np.concatenate([rad[-1:], rad, rad[:1]])
            rb = np.interp(th, a_ext, r_ext)
            inside = r < rb
            out[:, inside] = col[:, None]
        return out


class _Texture:
    def __init__(self, rng: np.random.Generator, channels: int, extent, polys: int,
                 octaves: int, base_period: float, poly_r=(6.0, 40.0)):
        self.noise = _ValueNoise(rng, channels, octaves, base_period)
        self.polys = _StarPolygons(rng, channels, polys, extent, poly_r[0], poly_r[1])
        self.contrast = rng.uniform(0.7, 1.0)

    def __call__(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        v = self.noise(x, y)
        v = 0.5 + (v - 0.5) * 2.2 * self.contrast
        v = self.polys.paint(x, y, np.clip(v, 0.0, 1.0))
        return v


# ----------------------------------------------------------------------------
# colour
# ----------------------------------------------------------------------------
def rgb_to_lab_u8(rgb01: np.ndarray) -> np.ndarray:
    """sRGB in [0,1], planar [3][H][W] -> 8-bit CIELab (D65), planar uint8."""
    c = np.where(rgb01 <= 0.04045, rgb01 / 12.92, ((rgb01 + 0.055) / 1.055) ** 2.4)
    r, g, b = c[0], c[1], c[2]
    x = 0.4124564 * r + 0.3575761 * g + 0.1804375 * b
    y = 0.2126729 * r + 0.7151522 * g + 0.0721750 * b
    z = 0.0193339 * r + 0.1191920 * g + 0.9503041 * b
    xn, yn, zn = 0.95047, 1.0, 1.08883
    e = 216.0 / 24389.0
    k = 24389.0 / 27.0

    def f(t):
        return np.where(t > e, np.cbrt(t), (k * t + 16.0) / 116.0)

    fx, fy, fz = f(x / xn), f(y / yn), f(z / zn)
    L = 116.0 * fy - 16.0
    a = 500.0 * (fx - fy)
    bb = 200.0 * (fy - fz)
    out = np.stack([L * 255.0 / 100.0, a + 128.0, bb + 128.0])
    return np.clip(np.rint(out), 0, 255).astype(np.uint8)


def _to_u8(v01: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(v01 * 255.0), 0, 255).astype(np.uint8)


# ----------------------------------------------------------------------------
# generators
# ----------------------------------------------------------------------------
def translation_pair(seed: int = 1, width: int = 128, height: int = 96,
                     shift=(7, -4), square: int = 24, square_shift=(18, 11),
                     rects: int = 20, sigma: float = 1.5,
                     with_square: bool = True) -> FramePair:
    """Gray pair: smoothed white noise + rectangles, shifted globally, one square moved.

    Frame 2 satisfies I2(q) = I1(q - shift) wherever q - shift lies inside the
    canvas; strips uncovered by the shift show the canvas beyond frame 1.  A
    ``square``-sized block of frame 1 is pasted into frame 2 displaced by
    ``square_shift``.
    """
    rng = np.random.default_rng(seed)
    sx, sy = shift
    pad = 64
    ch, cw = height + 2 * pad, width + 2 * pad
    noise = ndimage.gaussian_filter(rng.standard_normal((ch, cw)), sigma, mode="wrap")
    noise = (noise - noise.min()) / (noise.max() - noise.min())
    canvas = noise * 255.0
    for _ in range(rects):
        w = int(rng.integers(4, 33))
        h = int(rng.integers(4, 33))
        x0 = int(rng.integers(0, cw - w))
        y0 = int(rng.integers(0, ch - h))
        canvas[y0:y0 + h, x0:x0 + w] = rng.uniform(0, 255)
    canvas = np.clip(np.rint(canvas), 0, 255).astype(np.uint8)
    f1 = canvas[pad:pad + height, pad:pad + width].copy()
    f2 = canvas[pad - sy:pad - sy + height, pad - sx:pad - sx + width].copy()
    flow = np.zeros((height, width, 2))
    flow[..., 0] = sx
    flow[..., 1] = sy
    yy, xx = np.mgrid[0:height, 0:width]
    tx = xx + sx
    ty = yy + sy
    occ = (tx < 0) | (tx >= width) | (ty < 0) | (ty >= height)
    if with_square:
        qx, qy = square_shift
        lo_x, hi_x = max(0, -qx), min(width - square, width - square - qx)
        lo_y, hi_y = max(0, -qy), min(height - square, height - square - qy)
        x0 = int(rng.integers(lo_x, hi_x + 1))
        y0 = int(rng.integers(lo_y, hi_y + 1))
        block = f1[y0:y0 + square, x0:x0 + square].copy()
        f2[y0 + qy:y0 + qy + square, x0 + qx:x0 + qx + square] = block
        in_sq = (xx >= x0) & (xx < x0 + square) & (yy >= y0) & (yy < y0 + square)
        flow[in_sq, 0] = qx
        flow[in_sq, 1] = qy
        covered = ((tx >= x0 + qx) & (tx < x0 + qx + square)
                   & (ty >= y0 + qy) & (ty < y0 + qy + square))
        occ = np.where(in_sq, False, occ | covered)
    return FramePair(f1[None], f2[None], flow, occ, f"translation{width}x{height}")


def _affine(rng, cx, cy, max_disp, width, height):
    """Random rotation (<=10 deg) + scale (0.9..1.1) about (cx, cy) + translation.

    The translation points in a random direction and is made as long as the
    bound allows: the displacement of every frame corner stays <= max_disp.
    """
    corners = np.array([[0, 0], [width, 0], [0, height], [width, height]], float)
    for _ in range(64):
        th = np.deg2rad(rng.uniform(-10, 10))
        s = rng.uniform(0.9, 1.1)
        A = s * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        b0 = np.array([cx, cy]) - A @ np.array([cx, cy])
        d_rs = corners @ A.T + b0 - corners
        if np.max(np.hypot(d_rs[:, 0], d_rs[:, 1])) > 0.8 * max_disp:
            continue
        ang = rng.uniform(0, 2 * np.pi)
        u = np.array([np.cos(ang), np.sin(ang)])
        lo, hi = 0.0, max_disp
        for _ in range(40):
            m = 0.5 * (lo + hi)
            d = d_rs + m * u
            if np.max(np.hypot(d[:, 0], d[:, 1])) <= max_disp:
                lo = m
            else:
                hi = m
        return A, b0 + lo * u
    return np.eye(2), np.zeros(2)


def layered_pair(seed: int = 2, width: int = 1024, height: int = 436, channels: int = 3,
                 layers: int = 4, max_disp: float = 150.0) -> FramePair:
    """Depth-ordered layers with independent affine motions (Sintel-shaped).

    Layer 0 is a full-frame background whose motion reaches max_disp at the
    worst frame corner; layers 1.. are star-polygon regions in front of it,
    each with a random share (0.4..1) of the bound.  Each layer's texture is multi-octave value noise plus 10-30
    flat polygons, defined in layer coordinates and sampled analytically, so
    frame 2 is an exact re-sampling of the moved layers.  Ground truth is the
    motion of the front-most layer at each frame-1 pixel; a pixel is occluded
    when its moved position is outside frame 2 or covered by another layer.
    """
    rng = np.random.default_rng(seed)
    margin = max_disp + 64
    extent = (-margin, -margin, width + margin, height + margin)
    textures, masks, motions = [], [], []
    for k in range(layers):
        textures.append(_Texture(rng, channels, extent, int(rng.integers(10, 31)),
                                 octaves=int(rng.integers(4, 7)),
                                 base_period=float(rng.uniform(48, 128))))
        if k == 0:
            masks.append(None)
        else:
            rmax = 0.22 * min(width, height) + 0.1 * max(width, height)
            masks.append(_StarPolygons(rng, 1, 1,
                                       (0.15 * width, 0.15 * height, 0.85 * width, 0.85 * height),
                                       0.5 * rmax, rmax, verts=(6, 10)))
        cx = rng.uniform(0.3, 0.7) * width
        cy = rng.uniform(0.3, 0.7) * height
        # the full-frame background takes the whole bound (so the far end of
        # the displacement range occurs), the layers in front a random share
        share = rng.uniform(0.4, 1.0)
        motions.append(_affine(rng, cx, cy, max_disp * (1.0 if k == 0 else share), width, height))

    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)

    def layer_mask(k, x, y):
        if masks[k] is None:
            return np.ones(x.shape, bool)
        return masks[k].paint(x, y, np.zeros((1,) + x.shape))[0] > 0.5

    # frame 1: layers at identity (layer coordinates == frame-1 coordinates)
    img1 = np.zeros((channels, height, width))
    top1 = np.zeros((height, width), np.int64)
    for k in range(layers):
        m = layer_mask(k, xx, yy)
        img1[:, m] = textures[k](xx[m], yy[m])
        top1[m] = k
    # frame 2: each layer moved by its affine map; inverse-map the frame-2 pixels
    img2 = np.zeros((channels, height, width))
    top2 = np.full((height, width), -1, np.int64)
    for k in range(layers):
        A, b = motions[k]
        Ai = np.linalg.inv(A)
        px = Ai[0, 0] * (xx - b[0]) + Ai[0, 1] * (yy - b[1])
        py = Ai[1, 0] * (xx - b[0]) + Ai[1, 1] * (yy - b[1])
        m = layer_mask(k, px, py)
        img2[:, m] = textures[k](px[m], py[m])
        top2[m] = k
    flow = np.zeros((height, width, 2))
    for k in range(layers):
        A, b = motions[k]
        sel = top1 == k
        tx = A[0, 0] * xx + A[0, 1] * yy + b[0]
        ty = A[1, 0] * xx + A[1, 1] * yy + b[1]
        flow[sel, 0] = (tx - xx)[sel]
        flow[sel, 1] = (ty - yy)[sel]
    tx = xx + flow[..., 0]
    ty = yy + flow[..., 1]
    inside = (tx >= 0) & (tx <= width - 1) & (ty >= 0) & (ty <= height - 1)
    txi = np.clip(np.rint(tx), 0, width - 1).astype(np.int64)
    tyi = np.clip(np.rint(ty), 0, height - 1).astype(np.int64)
    occ = ~inside | (top2[tyi, txi] != top1)
    if channels == 3:
        i1, i2 = rgb_to_lab_u8(img1), rgb_to_lab_u8(img2)
    else:
        i1, i2 = _to_u8(img1), _to_u8(img2)
    return FramePair(i1, i2, flow, occ, f"layered{width}x{height}c{channels}")


def expansion_pair(seed: int = 3, width: int = 1242, height: int = 375,
                   max_disp: float = 250.0, obstacles: int = 3) -> FramePair:
    """Gray ego-motion pair (KITTI-shaped): ground plane + planar obstacles.

    The camera moves forward, so every surface point moves away from the focus
    of expansion (FOE) by the factor Z/(Z - Tz).  The ground plane's depth
    follows from the image row (Z proportional to 1/(y - horizon)); obstacles
    are fronto-parallel rectangles at fixed depths; above the horizon a far
    wall moves little.  Tz is scaled so the largest ground displacement
    visible in frame 1 equals ``max_disp``.
    """
    rng = np.random.default_rng(seed)
    foe = np.array([width * rng.uniform(0.45, 0.55), height * rng.uniform(0.38, 0.46)])
    horizon = foe[1]
    fh = 1.0  # focal length * camera height (units cancel)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    # ground: Z(y) = fh / (y - horizon); after moving Tz: s = Z / (Z - Tz)
    y_max = height - 1
    dmax_row = y_max - horizon
    # displacement at bottom corner = s*(corner - foe) - (corner - foe); pick Tz
    corner = np.hypot(max(foe[0], width - 1 - foe[0]), dmax_row)
    s_max = (corner + max_disp) / corner
    Z_bot = fh / dmax_row
    Tz = Z_bot * (1 - 1 / s_max)
    wall_Z = 40.0 * Z_bot / 1.0 + Tz * 30
    margin = max_disp + 64
    tex_ground = _Texture(rng, 1, (-4 * width, 0, 5 * width, 8 * width), 400,
                          octaves=6, base_period=96.0, poly_r=(8, 60))
    tex_wall = _Texture(rng, 1, (-margin, -margin, width + margin, height + margin), 20,
                        octaves=5, base_period=80.0)
    obs = []
    for _ in range(obstacles):
        w = rng.uniform(0.06, 0.16) * width
        h = rng.uniform(0.2, 0.45) * height
        cx = rng.uniform(0.1, 0.9) * width
        base = rng.uniform(horizon + 0.25 * dmax_row, height - 1)
        Z = fh / (base - horizon)
        tex = _Texture(rng, 1, (cx - w, base - 2 * h, cx + w, base + h), 12, 5, 40.0)
        obs.append((cx - w / 2, cx + w / 2, base - h, base, Z, tex))
    obs.sort(key=lambda o: -o[4])   # far to near: nearer obstacles painted later

    def ground_coords(x, y):
        dy = np.maximum(y - horizon, 1e-6)
        Z = fh / dy
        X = (x - foe[0]) * Z
        return X * 400.0, Z * 400.0 * 6.0  # texture-space scaling

    def scale_for(Z):
        return Z / (Z - Tz)

    def render(frame2: bool):
        img = np.zeros((height, width))
        zbuf = np.full((height, width), np.inf)
        layer = np.full((height, width), -1, np.int64)
        s_wall = scale_for(wall_Z)
        # far wall (everywhere, lowest priority)
        if frame2:
            wx = foe[0] + (xx - foe[0]) / s_wall
            wy = foe[1] + (yy - foe[1]) / s_wall
        else:
            wx, wy = xx, yy
        img[:] = tex_wall(wx, wy)[0]
        zbuf[:] = wall_Z
        layer[:] = 0
        # ground plane below the horizon
        if frame2:
            # inverse of the ground map: 1/(y-h) = 1/(y'-h) + Tz/fh
            dy2 = yy - horizon
            ok = dy2 > 1e-3
            inv = np.where(ok, 1.0 / np.where(ok, dy2, 1.0) + Tz / fh, np.inf)
            y1 = horizon + 1.0 / inv
            x1 = foe[0] + (xx - foe[0]) * (y1 - horizon) / np.where(ok, dy2, 1.0)
        else:
            ok = (yy - horizon) > 1e-3
            y1, x1 = yy, xx
        Zg = np.where(ok, fh / np.maximum(y1 - horizon, 1e-9), np.inf)
        gnd = ok & (Zg < wall_Z) & (Zg - Tz > 0)
        gx, gz = ground_coords(x1[gnd], y1[gnd])
        img[gnd] = tex_ground(gx, gz)[0]
        zbuf[gnd] = Zg[gnd]
        layer[gnd] = 1
        for i, (ox0, ox1, oy0, oy1, Z, tex) in enumerate(obs):
            s = scale_for(Z) if frame2 else 1.0
            px = foe[0] + (xx - foe[0]) / s
            py = foe[1] + (yy - foe[1]) / s
            m = (px >= ox0) & (px < ox1) & (py >= oy0) & (py < oy1) & (Z < zbuf)
            img[m] = tex(px[m], py[m])[0]
            zbuf[m] = Z
            layer[m] = 2 + i
        return img, layer, zbuf

    img1, layer1, z1 = render(False)
    img2, layer2, _ = render(True)
    s = np.where(np.isfinite(z1), z1 / (z1 - Tz), 1.0)
    flow = np.zeros((height, width, 2))
    flow[..., 0] = (s - 1.0) * (xx - foe[0])
    flow[..., 1] = (s - 1.0) * (yy - foe[1])
    tx = xx + flow[..., 0]
    ty = yy + flow[..., 1]
    inside = (tx >= 0) & (tx <= width - 1) & (ty >= 0) & (ty <= height - 1)
    txi = np.clip(np.rint(tx), 0, width - 1).astype(np.int64)
    tyi = np.clip(np.rint(ty), 0, height - 1).astype(np.int64)
    occ = ~inside | (layer2[tyi, txi] != layer1)
    return FramePair(_to_u8(img1)[None], _to_u8(img2)[None], flow, occ,
                     f"expansion{width}x{height}")


def periodic_pair(seed: int = 5, width: int = 95, height: int = 95, period: int = 12,
                  shift=(3, 2)) -> FramePair:
    """Repetitive texture (period < patch influence area) shifted globally.

    A stand-in for the paper's repetitive-pattern experiment (Sec. 4.5): a
    small random tile repeated over the frame; frame 2 is frame 1 shifted by
    ``shift`` with the canvas continuing the tiling.
    """
    rng = np.random.default_rng(seed)
    tile = ndimage.gaussian_filter(rng.random((period, period)), 1.0, mode="wrap")
    tile = (tile - tile.min()) / (tile.max() - tile.min())
    pad = 32
    reps_y = (height + 2 * pad) // period + 2
    reps_x = (width + 2 * pad) // period + 2
    canvas = np.tile(tile, (reps_y, reps_x))[:height + 2 * pad, :width + 2 * pad]
    canvas = _to_u8(canvas)
    sx, sy = shift
    f1 = canvas[pad:pad + height, pad:pad + width].copy()
    f2 = canvas[pad - sy:pad - sy + height, pad - sx:pad - sx + width].copy()
    flow = np.zeros((height, width, 2))
    flow[..., 0] = sx
    flow[..., 1] = sy
    yy, xx = np.mgrid[0:height, 0:width]
    occ = (xx + sx < 0) | (xx + sx >= width) | (yy + sy < 0) | (yy + sy >= height)
    return FramePair(f1[None], f2[None], flow, occ, f"periodic{width}x{height}")


def periodic_object_pair(seed: int = 5, width: int = 95, height: int = 95, size: int = 36,
                         period: int = 12, shift=(11, 6), bg_shift=(2, 1),
                         sigma: float = 1.5) -> FramePair:
    """A square object with a repetitive texture, moving on its own.

    A stand-in for the paper's repetitive-pattern experiment (Sec. 4.5, 95x95
    frames): the object's texture is a random tile repeated with ``period``,
    so a window smaller than the object matches it at every period shift; the
    object (``size`` x ``size``) is smaller than the coarsest influence area
    of a 4-scale run.  The background is smoothed noise translated by
    ``bg_shift``; the object moves by ``shift`` and covers the background in
    both frames.
    """
    rng = np.random.default_rng(seed)
    pad = 48
    noise = ndimage.gaussian_filter(rng.standard_normal((height + 2 * pad, width + 2 * pad)),
                                    sigma, mode="wrap")
    bg = _to_u8((noise - noise.min()) / (noise.max() - noise.min()))
    tile = ndimage.gaussian_filter(rng.random((period, period)), 1.0, mode="wrap")
    tile = (tile - tile.min()) / (tile.max() - tile.min())
    reps = size // period + 2
    obj = _to_u8(np.tile(tile, (reps, reps))[:size, :size])
    bx, by = bg_shift
    ox, oy = shift
    f1 = bg[pad:pad + height, pad:pad + width].copy()
    f2 = bg[pad - by:pad - by + height, pad - bx:pad - bx + width].copy()
    x0 = (width - size) // 2 - ox // 2
    y0 = (height - size) // 2 - oy // 2
    assert 0 <= x0 and x0 + size + max(ox, 0) <= width and x0 + min(ox, 0) >= 0
    assert 0 <= y0 and y0 + size + max(oy, 0) <= height and y0 + min(oy, 0) >= 0
    f1[y0:y0 + size, x0:x0 + size] = obj
    f2[y0 + oy:y0 + oy + size, x0 + ox:x0 + ox + size] = obj
    yy, xx = np.mgrid[0:height, 0:width]
    inobj = (xx >= x0) & (xx < x0 + size) & (yy >= y0) & (yy < y0 + size)
    flow = np.zeros((height, width, 2))
    flow[..., 0], flow[..., 1] = bx, by
    flow[inobj, 0], flow[inobj, 1] = ox, oy
    tx, ty = xx + flow[..., 0].astype(int), yy + flow[..., 1].astype(int)
    covered = ((tx >= x0 + ox) & (tx < x0 + ox + size) & (ty >= y0 + oy) & (ty < y0 + oy + size))
    occ = (tx < 0) | (tx >= width) | (ty < 0) | (ty >= height) | (~inobj & covered)
    return FramePair(f1[None], f2[None], flow, occ, f"periodic_object{width}x{height}")


def random_pair(seed: int, width: int, height: int, channels: int = 1) -> FramePair:
    """Two independent uniform-noise frames (no meaningful flow); for parity cases."""
    rng = np.random.default_rng(seed)
    i1 = rng.integers(0, 256, (channels, height, width), dtype=np.uint8)
    i2 = rng.integers(0, 256, (channels, height, width), dtype=np.uint8)
    return FramePair(i1, i2, np.zeros((height, width, 2)), np.zeros((height, width), bool),
                     f"random{width}x{height}c{channels}")


# ----------------------------------------------------------------------------
# the named workloads and their matching parameters
# ----------------------------------------------------------------------------
WORKLOADS = {
    # tiny gray pair: 3 scales, 4 propagation iterations, R = 1 px
    "tiny128x96": dict(gen=translation_pair, kw=dict(seed=1), scales=3, iters=4, radius_q3=8),
    # Sintel-shaped 1024x436 Lab pair: 4 scales, 6 iterations, R = 1 px
    "sintel1024x436": dict(gen=layered_pair, kw=dict(seed=2), scales=4, iters=6, radius_q3=8),
    # KITTI-shaped 1242x375 gray pair: 4 scales, 4 iterations, R = 1.5 px
    "kitti1242x375": dict(gen=expansion_pair, kw=dict(seed=3), scales=4, iters=4, radius_q3=12),
}


def make_workload(name: str) -> tuple[FramePair, dict]:
    spec = WORKLOADS[name]
    pair = spec["gen"](**spec["kw"])
    params = dict(scales=spec["scales"], iters=spec["iters"], radius_q3=spec["radius_q3"],
                  channels=pair.channels)
    return pair, params


# ----------------------------------------------------------------------------
# batched workload: many pairs of mixed sizes in one Lab configuration
# ----------------------------------------------------------------------------
BATCH_SIZES = ((320, 240), (640, 480), (1024, 436), (1242, 375))
# matching parameters of the batch (those of the Sintel-shaped pair)
BATCH_PARAMS = dict(channels=3, scales=4, iters=6, radius_q3=8)


def _gray_to_lab(pair: FramePair) -> FramePair:
    """A gray pair as 8-bit CIELab frames (r = g = b = gray): L carries the
    image, a and b sit at their neutral 128."""
    to_lab = lambda g: rgb_to_lab_u8(np.repeat(g.astype(np.float64) / 255.0, 3, axis=0))
    return FramePair(to_lab(pair.img1), to_lab(pair.img2), pair.flow, pair.occ,
                     pair.name + "-lab")


def batch_pair(seed: int, k: int, sizes=BATCH_SIZES, layered_only: bool = False) -> FramePair:
    """Pair k of the mixed batch: a size drawn uniformly from `sizes` and,
    alternately, the layered Sintel-shaped generator (displacement scaled to
    the frame: 150 px at 1024 wide) or the translation generator of the tiny
    workload (a per-pair global shift up to 3 % of the width, promoted to Lab).
    layered_only: every pair from the layered generator."""
    rng = np.random.default_rng([seed, k])
    w, h = sizes[int(rng.integers(0, len(sizes)))]
    if k % 2 == 0 or layered_only:
        return layered_pair(seed=int(rng.integers(1 << 30)), width=w, height=h, channels=3,
                            max_disp=150.0 * w / 1024.0)
    m = max(2, int(0.03 * w))
    shift = (int(rng.integers(-m, m + 1)), int(rng.integers(-m, m + 1)))
    g = translation_pair(seed=int(rng.integers(1 << 30)), width=w, height=h, shift=shift,
                         square=min(24, h // 4, w // 4),
                         square_shift=(min(18, w // 8), min(11, h // 8)),
                         rects=max(20, w * h // 4000))
    return _gray_to_lab(g)


def _batch_pair_args(a):
    return batch_pair(*a)


def make_batch(n: int = 64, seed: int = 4, sizes=BATCH_SIZES, workers: int = 0,
               layered_only: bool = False) -> list[FramePair]:
    """The n pairs of the mixed batch; `workers` > 1 generates them in a
    process pool started with 'spawn' (safe after CUDA has been initialised)."""
    args = [(seed, k, sizes, layered_only) for k in range(n)]
    if workers > 1 and n > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, n)) as pool:
            return pool.map(_batch_pair_args, args)
    return [batch_pair(*a) for a in args]


# ----------------------------------------------------------------------------
# serving workload: requests of sizes 256x256 .. 1920x1080 in 64-px steps
# ----------------------------------------------------------------------------
SERVE_WIDTHS = tuple(range(256, 1921, 64))
SERVE_HEIGHTS = tuple(range(256, 1025, 64)) + (1080,)


def _serving_pair(a) -> FramePair:
    seed, w, h = a
    return layered_pair(seed=seed, width=w, height=h, channels=3, max_disp=300.0 * w / 1920.0)


def serving_pairs(n: int, seed: int = 8, workers: int = 0, widths=SERVE_WIDTHS,
                  heights=SERVE_HEIGHTS) -> list[FramePair]:
    """n independent layered pairs (the Sintel-shaped generator, Lab), each
    with its own size drawn uniformly from widths x heights, its own layers
    and motions, displacements up to 300 px at 1920 wide (scaled with the
    width); `workers` > 1 generates them in a 'spawn' process pool."""
    rng = np.random.default_rng(seed)
    args = [(seed * 100000 + k, int(widths[int(rng.integers(0, len(widths)))]),
             int(heights[int(rng.integers(0, len(heights)))])) for k in range(n)]
    if workers > 1 and n > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, n)) as pool:
            return pool.map(_serving_pair, args)
    return [_serving_pair(a) for a in args]


def serving_pair_requests(n: int, n_pairs: int, seed: int = 9) -> list[dict]:
    """n requests over n_pairs pairs: each names a pair drawn uniformly and
    carries its own pair id (its own random-search stream)."""
    rng = np.random.default_rng(seed)
    return [dict(pair=int(rng.integers(0, n_pairs)), pair_id=k) for k in range(n)]


def _serving_base(seed: int) -> FramePair:
    return layered_pair(seed=seed, width=1920, height=1080, channels=3, max_disp=300.0)


def serving_bases(n: int = 4, seed: int = 6, workers: int = 0) -> list[FramePair]:
    """n full-HD layered pairs (displacements up to 300 px) that requests are
    cut from; `workers` > 1 generates them in a 'spawn' process pool."""
    seeds = [seed * 1000 + k for k in range(n)]
    if workers > 1 and n > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, n)) as pool:
            return pool.map(_serving_base, seeds)
    return [_serving_base(s) for s in seeds]


def serving_requests(n: int, n_bases: int, seed: int = 7, widths=SERVE_WIDTHS,
                     heights=SERVE_HEIGHTS, base_w: int = 1920,
                     base_h: int = 1080) -> list[dict]:
    """n requests: a size drawn uniformly from widths x heights, a base pair
    (base_w x base_h) and a crop offset inside it; cropping both frames at
    the same window keeps the pair's flow (the crop of the ground truth)."""
    assert max(widths) <= base_w and max(heights) <= base_h
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        w = int(widths[int(rng.integers(0, len(widths)))])
        h = int(heights[int(rng.integers(0, len(heights)))])
        out.append(dict(base=int(rng.integers(0, n_bases)), w=w, h=h,
                        x0=int(rng.integers(0, base_w - w + 1)),
                        y0=int(rng.integers(0, base_h - h + 1)), pair_id=k))
    return out
