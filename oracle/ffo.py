"""ctypes view of the C oracle (test infrastructure only).

Thin NumPy wrappers around ``libffo.so``; every array is host memory.  The
arithmetic lives in ``ffo.c``.
"""
from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass

import numpy as np

from . import build as _build

INVALID = -32768
INVALID_COST = 2**31 - 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ct.CDLL(path)
        P = ct.c_void_p
        i = ct.c_int
        L.ffo_level_dims.argtypes = [i, i, i, P, P]
        L.ffo_feature_offset.argtypes = [i, i, i, i]
        L.ffo_feature_offset.restype = ct.c_long
        L.ffo_feature_bytes.argtypes = [i, i, i, i]
        L.ffo_feature_bytes.restype = ct.c_long
        L.ffo_level_image.argtypes = [P, i, i, i, i, P]
        L.ffo_wht_coeffs.argtypes = [P, i, i, i, P]
        L.ffo_quantise.argtypes = [ct.c_int32, i]
        L.ffo_quantise.restype = i
        L.ffo_wht_features.argtypes = [P, i, i, i, P]
        L.ffo_features_all.argtypes = [P, i, i, i, i, P]
        L.ffo_philox4x32_10.argtypes = [P, P, P]
        L.ffo_clamp_flow.argtypes = [i, i, i, i, P, P]
        L.ffo_cost.argtypes = [P, P, i, i, i, i, i, i, ct.c_int32, ct.c_int32]
        L.ffo_cost.restype = ct.c_int32
        L.ffo_seed_knn.argtypes = [P, P, i, i, i, i, i, i, P, P]
        L.ffo_seed_knn.restype = i
        L.ffo_seed_knn_rows.argtypes = [P, P, i, i, i, i, i, i, i, i, P, P]
        L.ffo_seed_knn_rows.restype = i
        L.ffo_match_features.argtypes = [P, P, P, i, i, i, ct.c_uint32, P, i, i, P, P, P]
        L.ffo_match_features.restype = i
        L.ffo_match_features_knn.argtypes = [P, P, P, i, i, i, ct.c_uint32, P, i, i, P, P, P]
        L.ffo_match_features_knn.restype = i
        L.ffo_match.argtypes = [P, P, P, i, i, i, ct.c_uint32, P, i, i, P, P, P]
        L.ffo_match.restype = i
        L.ffo_filter.argtypes = [P, P, i, i, i, P]
        L.ffo_filter_grid.argtypes = [P, P, i, i, i, i, P]
        L.ffo_region_filter.argtypes = [P, P, i, i, i, P]
        L.ffo_region_filter.restype = None
        L.ffo_sparsify.argtypes = [P, P, P, P, i, i, i, i, i, P]
        L.ffo_sparsify.restype = None
        L.ffo_filter2.argtypes = [P, P, P, i, i, i, i, P]
        L.ffo_schedule_final_level.argtypes = [i]
        L.ffo_schedule_final_level.restype = i
        L.ffo_schedule_sweeps.argtypes = [i, i, i]
        L.ffo_schedule_sweeps.restype = i
        L.ffo_schedule_radius_mult.argtypes = [i, i, i]
        L.ffo_schedule_radius_mult.restype = i
        L.ffo_schedule_rs_after.argtypes = [i, i, i, i]
        L.ffo_schedule_rs_after.restype = i
        L.ffo_sweep_level.argtypes = [P, P, i, i, i, i, i, P, P, P]
        L.ffo_random_search_level.argtypes = [P, P, i, i, i, i, i, i, i, ct.c_uint32,
                                              ct.c_uint32, P, P, P]
        _lib = L
    return _lib


class _Params(ct.Structure):
    _fields_ = [("channels", ct.c_int), ("scales", ct.c_int), ("iters", ct.c_int),
                ("radius_q3", ct.c_int), ("seed_leaf", ct.c_int), ("seed_stride", ct.c_int),
                ("seed", ct.c_uint32), ("schedule", ct.c_int)]


@dataclass
class Params:
    channels: int = 1
    scales: int = 3
    iters: int = 4
    radius_q3: int = 8
    seed_leaf: int = 8
    seed_stride: int = 1
    seed: int = 20261203
    schedule: int = 0   # 0 basic, 1 Flow Fields+, 2 Flow Fields+ Fast, 3 Fast x2

    def c(self) -> _Params:
        return _Params(self.channels, self.scales, self.iters, self.radius_q3,
                       self.seed_leaf, self.seed_stride, self.seed, self.schedule)

    def sweeps(self, level: int) -> int:
        return int(lib().ffo_schedule_sweeps(self.schedule, self.iters, level))

    def final_level(self) -> int:
        return int(lib().ffo_schedule_final_level(self.schedule))


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ct.c_void_p)


def level_dims(W: int, H: int, L: int) -> tuple[int, int]:
    n = 1 << L
    return (W + n - 1) // n, (H + n - 1) // n


def level_image(img: np.ndarray, L: int) -> np.ndarray:
    img = np.ascontiguousarray(img, np.uint8)
    C, H, W = img.shape
    WL, HL = level_dims(W, H, L)
    out = np.zeros((C, HL, WL), np.uint8)
    lib().ffo_level_image(_p(img), C, W, H, L, _p(out))
    return out


def wht_coeffs(D: np.ndarray) -> np.ndarray:
    D = np.ascontiguousarray(D, np.uint8)
    C, HL, WL = D.shape
    out = np.zeros((HL, WL, 9 * C), np.int32)
    lib().ffo_wht_coeffs(_p(D), C, WL, HL, _p(out))
    return out


def quantise(c: int, dc: bool) -> int:
    return int(lib().ffo_quantise(int(c), 1 if dc else 0))


def wht_features(D: np.ndarray) -> np.ndarray:
    D = np.ascontiguousarray(D, np.uint8)
    C, HL, WL = D.shape
    out = np.zeros((HL, WL, 9 * C), np.int8)
    lib().ffo_wht_features(_p(D), C, WL, HL, _p(out))
    return out


def features_all(img: np.ndarray, S: int) -> list[np.ndarray]:
    """Features of every level as a list of int8 [HL][WL][9C] arrays."""
    img = np.ascontiguousarray(img, np.uint8)
    C, H, W = img.shape
    nb = lib().ffo_feature_bytes(W, H, C, S)
    flat = np.zeros(nb, np.int8)
    lib().ffo_features_all(_p(img), C, W, H, S, _p(flat))
    out = []
    for L in range(S):
        WL, HL = level_dims(W, H, L)
        off = lib().ffo_feature_offset(W, H, C, L)
        out.append(flat[off:off + WL * HL * 9 * C].reshape(HL, WL, 9 * C))
    return out


def _flat_features(feats: list[np.ndarray]) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([f.reshape(-1) for f in feats]), np.int8)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, np.uint32))
    k = np.ascontiguousarray(np.asarray(key, np.uint32))
    out = np.zeros(4, np.uint32)
    lib().ffo_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def clamp_flow(W: int, H: int, px: int, py: int, Fx: int, Fy: int) -> tuple[int, int]:
    fx = ct.c_int32(Fx)
    fy = ct.c_int32(Fy)
    lib().ffo_clamp_flow(W, H, px, py, ct.byref(fx), ct.byref(fy))
    return fx.value, fy.value


def cost(f1L: np.ndarray, f2L: np.ndarray, W: int, H: int, L: int, px: int, py: int,
         Fx: int, Fy: int) -> int:
    f1L = np.ascontiguousarray(f1L, np.int8)
    f2L = np.ascontiguousarray(f2L, np.int8)
    C = f1L.shape[-1] // 9
    return int(lib().ffo_cost(_p(f1L), _p(f2L), C, W, H, L, px, py, Fx, Fy))


def seed_knn(f1_0: np.ndarray, f2_0: np.ndarray, S: int, leaf: int = 8, stride: int = 1):
    f1_0 = np.ascontiguousarray(f1_0, np.int8)
    f2_0 = np.ascontiguousarray(f2_0, np.int8)
    H, W, D = f1_0.shape
    C = D // 9
    WS, HS = level_dims(W, H, S - 1)
    idx = np.zeros((HS, WS, leaf), np.int32)
    dist = np.zeros((HS, WS, leaf), np.int32)
    lib().ffo_seed_knn(_p(f1_0), _p(f2_0), C, W, H, S, leaf, stride, _p(idx), _p(dist))
    return idx, dist


def seed_knn_rows(f1_0: np.ndarray, f2_0: np.ndarray, S: int, gy0: int, gy1: int,
                  leaf: int = 8, stride: int = 1):
    """Seeding search for coarsest-grid rows gy0..gy1-1 only (others left -1)."""
    f1_0 = np.ascontiguousarray(f1_0, np.int8)
    f2_0 = np.ascontiguousarray(f2_0, np.int8)
    H, W, D = f1_0.shape
    WS, HS = level_dims(W, H, S - 1)
    idx = np.full((HS, WS, leaf), -1, np.int32)
    dist = np.full((HS, WS, leaf), -1, np.int32)
    lib().ffo_seed_knn_rows(_p(f1_0), _p(f2_0), D // 9, W, H, S, leaf, stride, gy0, gy1,
                            _p(idx), _p(dist))
    return idx, dist


def seed_knn_threaded(f1_0: np.ndarray, f2_0: np.ndarray, S: int, leaf: int = 8,
                      stride: int = 1, workers: int | None = None):
    """ffo_seed_knn's lists, computed as independent bands of coarsest-grid
    rows (ffo_seed_knn_rows) on a thread pool; ctypes releases the GIL during
    each call.  The result is the same as seed_knn's: every row is computed
    by the same sequential C code, only different rows run at once."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    f1_0 = np.ascontiguousarray(f1_0, np.int8)
    f2_0 = np.ascontiguousarray(f2_0, np.int8)
    H, W, D = f1_0.shape
    WS, HS = level_dims(W, H, S - 1)
    idx = np.full((HS, WS, leaf), -1, np.int32)
    dist = np.full((HS, WS, leaf), -1, np.int32)
    workers = workers or os.cpu_count() or 1
    bands = [(y, y + 1) for y in range(HS)]

    def run(band):
        gy0, gy1 = band
        bi = np.full((HS, WS, leaf), -1, np.int32)
        bd = np.full((HS, WS, leaf), -1, np.int32)
        lib().ffo_seed_knn_rows(_p(f1_0), _p(f2_0), D // 9, W, H, S, leaf, stride, gy0, gy1,
                                _p(bi), _p(bd))
        return gy0, gy1, bi[gy0:gy1], bd[gy0:gy1]

    with ThreadPoolExecutor(max_workers=workers) as ex:
        for gy0, gy1, bi, bd in ex.map(run, bands):
            idx[gy0:gy1] = bi
            dist[gy0:gy1] = bd
    return idx, dist


def match_features_knn(prm: Params, fsrc: list[np.ndarray], fdst: list[np.ndarray], W: int,
                       H: int, direction: int, pair_id: int, knn_idx: np.ndarray):
    """ffo_match_features with the seeding lists given (the Eq. 1 rerank and
    everything after it run in the oracle).  Returns (flow, cost, evals)."""
    Lf = prm.final_level()
    WL, HL = level_dims(W, H, Lf)
    flow = np.zeros((HL, WL, 2), np.int16)
    cst = np.zeros((HL, WL), np.int32)
    ev = ct.c_int64(0)
    knn = np.ascontiguousarray(knn_idx, np.int32)
    c = prm.c()
    fs, fd = _flat_features(fsrc), _flat_features(fdst)
    rc = lib().ffo_match_features_knn(ct.byref(c), _p(fs), _p(fd), W, H, direction, pair_id,
                                      _p(knn), Lf, prm.sweeps(Lf), _p(flow), _p(cst),
                                      ct.byref(ev))
    if rc != 0:
        raise ValueError("ffo_match_features_knn rejected its arguments")
    return flow, cst, ev.value


def match_features(prm: Params, fsrc: list[np.ndarray], fdst: list[np.ndarray], W: int, H: int,
                   direction: int = 0, pair_id: int = 0, seeds_in: np.ndarray | None = None,
                   until_level: int | None = None, until_sweeps: int | None = None):
    """Returns (flow int16 [HL][WL][2], cost int32 [HL][WL], evals)."""
    if until_level is None:
        until_level = prm.final_level()
    if until_sweeps is None:
        until_sweeps = prm.sweeps(until_level)
    WL, HL = level_dims(W, H, until_level)
    flow = np.zeros((HL, WL, 2), np.int16)
    cst = np.zeros((HL, WL), np.int32)
    ev = ct.c_int64(0)
    s_ptr = None
    if seeds_in is not None:
        seeds_in = np.ascontiguousarray(seeds_in, np.int16)
        s_ptr = _p(seeds_in)
    c = prm.c()
    fs, fd = _flat_features(fsrc), _flat_features(fdst)
    rc = lib().ffo_match_features(ct.byref(c), _p(fs), _p(fd), W, H, direction, pair_id, s_ptr,
                                  until_level, until_sweeps, _p(flow), _p(cst), ct.byref(ev))
    if rc != 0:
        raise ValueError("ffo_match_features rejected its arguments")
    return flow, cst, ev.value


def match(prm: Params, src: np.ndarray, dst: np.ndarray, direction: int = 0, pair_id: int = 0,
          seeds_in: np.ndarray | None = None, until_level: int | None = None,
          until_sweeps: int | None = None):
    """Match image src -> dst.  Returns (flow, cost, evals) at the stop level."""
    src = np.ascontiguousarray(src, np.uint8)
    dst = np.ascontiguousarray(dst, np.uint8)
    C, H, W = src.shape
    assert C == prm.channels and dst.shape == src.shape
    if until_level is None:
        until_level = prm.final_level()
    if until_sweeps is None:
        until_sweeps = prm.sweeps(until_level)
    WL, HL = level_dims(W, H, until_level)
    flow = np.zeros((HL, WL, 2), np.int16)
    cst = np.zeros((HL, WL), np.int32)
    ev = ct.c_int64(0)
    s_ptr = None
    if seeds_in is not None:
        seeds_in = np.ascontiguousarray(seeds_in, np.int16)
        s_ptr = _p(seeds_in)
    c = prm.c()
    rc = lib().ffo_match(ct.byref(c), _p(src), _p(dst), W, H, direction, pair_id, s_ptr,
                         until_level, until_sweeps, _p(flow), _p(cst), ct.byref(ev))
    if rc != 0:
        raise ValueError("ffo_match rejected its arguments")
    return flow, cst, ev.value


def filter_mask(fwd: np.ndarray, bwd: np.ndarray, eps_q3: int, level: int = 0) -> np.ndarray:
    """Consistency mask of flows on the level-`level` grid (0: pixels)."""
    fwd = np.ascontiguousarray(fwd, np.int16)
    bwd = np.ascontiguousarray(bwd, np.int16)
    H, W, _ = fwd.shape
    mask = np.zeros((H, W), np.uint8)
    if level == 0:
        lib().ffo_filter(_p(fwd), _p(bwd), W, H, eps_q3, _p(mask))
    else:
        lib().ffo_filter_grid(_p(fwd), _p(bwd), W, H, level, eps_q3, _p(mask))
    return mask


def sweep_level(f1L, f2L, W: int, H: int, L: int, d: int, flow, cost):
    """One propagation sweep in direction d on a level state (returns copies)."""
    f1L = np.ascontiguousarray(f1L, np.int8)
    f2L = np.ascontiguousarray(f2L, np.int8)
    flow = np.array(flow, np.int16, order="C")
    cost = np.array(cost, np.int32, order="C")
    ev = ct.c_int64(0)
    lib().ffo_sweep_level(_p(f1L), _p(f2L), f1L.shape[-1] // 9, W, H, L, d, _p(flow), _p(cost),
                          ct.byref(ev))
    return flow, cost, ev.value


def random_search_level(f1L, f2L, W: int, H: int, L: int, t: int, direction: int,
                        radius_q3: int, seed: int, pair_id: int, flow, cost):
    """One random-search pass on a level state (returns copies)."""
    f1L = np.ascontiguousarray(f1L, np.int8)
    f2L = np.ascontiguousarray(f2L, np.int8)
    flow = np.array(flow, np.int16, order="C")
    cost = np.array(cost, np.int32, order="C")
    ev = ct.c_int64(0)
    lib().ffo_random_search_level(_p(f1L), _p(f2L), f1L.shape[-1] // 9, W, H, L, t, direction,
                                  radius_q3, seed, pair_id, _p(flow), _p(cost), ct.byref(ev))
    return flow, cost, ev.value


def filter_mask2(fwd: np.ndarray, bwd1: np.ndarray, bwd2: np.ndarray, eps_q3: int,
                 level: int = 0) -> np.ndarray:
    """Two-way check: consistent with both backward flows."""
    fwd = np.ascontiguousarray(fwd, np.int16)
    bwd1 = np.ascontiguousarray(bwd1, np.int16)
    bwd2 = np.ascontiguousarray(bwd2, np.int16)
    H, W, _ = fwd.shape
    mask = np.zeros((H, W), np.uint8)
    lib().ffo_filter2(_p(fwd), _p(bwd1), _p(bwd2), W, H, level, eps_q3, _p(mask))
    return mask


def region_filter(fwd: np.ndarray, mask: np.ndarray, s: int) -> np.ndarray:
    """Region filter (Sec. 3.7) of a consistency mask on the flows' grid."""
    fwd = np.ascontiguousarray(fwd, np.int16)
    mask = np.ascontiguousarray(mask, np.uint8)
    H, W, _ = fwd.shape
    out = np.zeros((H, W), np.uint8)
    lib().ffo_region_filter(_p(fwd), _p(mask), W, H, s, _p(out))
    return out


def sparsify(fwd: np.ndarray, bwd1: np.ndarray, bwd2: np.ndarray | None, mask: np.ndarray,
             q: int, e: int, level: int = 0) -> np.ndarray:
    """Sparsification (Sec. 3.7-3.8): one point per q x q cell of >= e kept points."""
    fwd = np.ascontiguousarray(fwd, np.int16)
    bwd1 = np.ascontiguousarray(bwd1, np.int16)
    b2 = None if bwd2 is None else np.ascontiguousarray(bwd2, np.int16)
    mask = np.ascontiguousarray(mask, np.uint8)
    H, W, _ = fwd.shape
    out = np.zeros((H, W), np.uint8)
    lib().ffo_sparsify(_p(fwd), _p(bwd1), None if b2 is None else _p(b2), _p(mask), W, H, level,
                       q, e, _p(out))
    return out
