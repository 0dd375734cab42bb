"""Python binding of ``libff.so`` (declared in include/ff.h).

Argument marshalling only: every function here passes pointers and sizes to
the C ABI function of the same name; all the work runs in the CUDA kernels.
Device buffers are torch tensors (PyTorch provides device memory and
streams); host buffers are NumPy arrays or pinned torch CPU tensors.

The library is required: importing this module raises if ``libff.so`` cannot
be built or loaded.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass

from . import _build

FF_OK, FF_EINVAL, FF_ENOMEM, FF_ECUDA, FF_ETIMEOUT, FF_ESTATE = range(6)
FF_FWD, FF_BWD, FF_BWD2 = 0, 1, 2
FF_SCHED_BASIC, FF_SCHED_PLUS, FF_SCHED_PLUS_FAST, FF_SCHED_PLUS_FAST_X2 = 0, 1, 2, 3
FF_DEBUG_WAIT_LIMIT_NS, FF_DEBUG_FORCE_TIMEOUT, FF_DEBUG_SWEEP_LANES = 1, 2, 4
FF_DEBUG_SEED_TC = 5
FF_PROFILE_LAUNCHES, FF_PROFILE_SWEEP_RUNS = 1, 2
INVALID = -32768

EXPORTED = ("ff_config_default", "ff_create", "ff_set_stream", "ff_features", "ff_match",
            "ff_match_until", "ff_filter", "ff_filter_2way", "ff_region_filter", "ff_sparsify", "ff_wht_coeffs_tc",
            "ff_wht_coeffs_scalespace_tc",
            "ff_pair_host", "ff_get_features", "ff_seed_knn",
            "ff_seed_knn_static", "ff_measure_peaks", "ff_sync", "ff_debug_set", "ff_profile", "ff_kernel_stats",
            "ff_launch_count", "ff_last_error", "ff_status_string", "ff_destroy",
            "ff_batch_create", "ff_batch_run", "ff_batch_set_stream", "ff_batch_sync",
            "ff_batch_debug_set",
            "ff_batch_launch_count", "ff_batch_last_error", "ff_batch_destroy",
            "ff_slot_bytes", "ff_server_create", "ff_server_slots", "ff_server_submit",
            "ff_server_poll", "ff_server_pending", "ff_server_launch_count",
            "ff_server_last_error", "ff_server_destroy")


class ff_config(ct.Structure):
    _fields_ = [("patch", ct.c_int), ("n_coeffs", ct.c_int), ("channels", ct.c_int),
                ("scales", ct.c_int), ("iters", ct.c_int), ("radius_q3", ct.c_int),
                ("seed_leaf", ct.c_int), ("seed_stride", ct.c_int), ("eps_q3", ct.c_int),
                ("seed", ct.c_uint32), ("max_width", ct.c_int), ("max_height", ct.c_int),
                ("schedule", ct.c_int), ("region_min", ct.c_int),
                ("wht_tensor_cores", ct.c_int)]


class ff_pair_desc(ct.Structure):
    _fields_ = [("img1", ct.c_void_p), ("img2", ct.c_void_p), ("w", ct.c_int), ("h", ct.c_int),
                ("pitch", ct.c_int), ("pair_id", ct.c_uint32), ("flow_fwd", ct.c_void_p),
                ("flow_bwd", ct.c_void_p), ("flow_bwd2", ct.c_void_p), ("mask", ct.c_void_p)]


class ff_host_pair(ct.Structure):
    _fields_ = [("img1", ct.c_void_p), ("img2", ct.c_void_p), ("w", ct.c_int), ("h", ct.c_int),
                ("pitch", ct.c_int), ("plane", ct.c_longlong), ("pair_id", ct.c_uint32),
                ("two_way", ct.c_int), ("flow_fwd", ct.c_void_p), ("flow_bwd", ct.c_void_p),
                ("flow_bwd2", ct.c_void_p), ("mask", ct.c_void_p)]


class ff_peaks(ct.Structure):
    _fields_ = [("sm_count", ct.c_int), ("dp4a_per_s", ct.c_double), ("iadd3_per_s", ct.c_double),
                ("imad_per_s", ct.c_double), ("sad_dims_per_s", ct.c_double),
                ("l2_read_gbs", ct.c_double), ("lat_alu", ct.c_double), ("lat_prmt", ct.c_double),
                ("lat_dp4a", ct.c_double), ("lat_shfl", ct.c_double), ("lat_lds", ct.c_double),
                ("lat_ldg_l1", ct.c_double), ("lat_ldg_l2", ct.c_double)]


class FFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


_lib = None


def lib(build: bool = True) -> ct.CDLL:
    """Load libff.so (building it first when missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build else _build.LIB
        L = ct.CDLL(path)
        P, i, u32 = ct.c_void_p, ct.c_int, ct.c_uint32
        L.ff_config_default.argtypes = [ct.POINTER(ff_config)]
        L.ff_create.argtypes = [ct.POINTER(ff_config), i, P, ct.POINTER(P)]
        L.ff_set_stream.argtypes = [P, P]
        L.ff_features.argtypes = [P, i, P, i, i, i]
        L.ff_match.argtypes = [P, i, u32, P, P, P]
        L.ff_match_until.argtypes = [P, i, u32, P, i, i, P, P]
        L.ff_filter.argtypes = [P, P, P, P]
        L.ff_filter_2way.argtypes = [P, P, P, P, P]
        L.ff_region_filter.argtypes = [P, P, P, i, P]
        L.ff_sparsify.argtypes = [P, P, P, P, P, i, i, P]
        L.ff_wht_coeffs_tc.argtypes = [P, i, i, i, i, i, P, P]
        L.ff_wht_coeffs_scalespace_tc.argtypes = [P, i, i, i, i, i, i, P, P]
        L.ff_pair_host.argtypes = [P, P, P, i, i, u32, P, P, P]
        L.ff_get_features.argtypes = [P, i, i, P]
        L.ff_seed_knn.argtypes = [P, i, P, P]
        L.ff_seed_knn_static.argtypes = [P, P, i, i, i, i, i, i, P, P, P,
                                         ct.POINTER(ct.c_char_p)]
        L.ff_measure_peaks.argtypes = [i, ct.POINTER(ff_peaks)]
        L.ff_sync.argtypes = [P]
        L.ff_debug_set.argtypes = [P, i, ct.c_longlong]
        L.ff_profile.argtypes = [P, i]
        L.ff_kernel_stats.argtypes = [P, ct.c_char_p, ct.POINTER(ct.c_longlong),
                                      ct.POINTER(ct.c_double)]
        L.ff_launch_count.argtypes = [P]
        L.ff_launch_count.restype = ct.c_longlong
        L.ff_last_error.argtypes = [P]
        L.ff_last_error.restype = ct.c_char_p
        L.ff_status_string.argtypes = [i]
        L.ff_status_string.restype = ct.c_char_p
        L.ff_destroy.argtypes = [P]
        L.ff_destroy.restype = None
        L.ff_batch_create.argtypes = [ct.POINTER(ff_config), i, i, P, ct.POINTER(P)]
        L.ff_batch_run.argtypes = [P, i, ct.POINTER(ff_pair_desc), i]
        L.ff_batch_set_stream.argtypes = [P, P]
        L.ff_batch_sync.argtypes = [P]
        L.ff_batch_debug_set.argtypes = [P, i, ct.c_longlong]
        L.ff_batch_launch_count.argtypes = [P]
        L.ff_batch_launch_count.restype = ct.c_longlong
        L.ff_batch_last_error.argtypes = [P]
        L.ff_batch_last_error.restype = ct.c_char_p
        L.ff_batch_destroy.argtypes = [P]
        L.ff_batch_destroy.restype = None
        L.ff_slot_bytes.argtypes = [ct.POINTER(ff_config)]
        L.ff_slot_bytes.restype = ct.c_size_t
        L.ff_server_create.argtypes = [ct.POINTER(ff_config), i, ct.c_size_t, i, ct.POINTER(P)]
        L.ff_server_slots.argtypes = [P]
        L.ff_server_submit.argtypes = [P, ct.POINTER(ff_host_pair), ct.POINTER(ct.c_longlong)]
        L.ff_server_poll.argtypes = [P, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_int), i,
                                     ct.POINTER(ct.c_int)]
        L.ff_server_pending.argtypes = [P]
        L.ff_server_launch_count.argtypes = [P]
        L.ff_server_launch_count.restype = ct.c_longlong
        L.ff_server_last_error.argtypes = [P]
        L.ff_server_last_error.restype = ct.c_char_p
        L.ff_server_destroy.argtypes = [P]
        L.ff_server_destroy.restype = None
        for name in EXPORTED:
            if name not in ("ff_last_error", "ff_status_string", "ff_destroy",
                            "ff_launch_count", "ff_batch_launch_count", "ff_batch_last_error",
                            "ff_batch_destroy", "ff_slot_bytes", "ff_server_launch_count",
                            "ff_server_last_error", "ff_server_destroy"):
                getattr(L, name).restype = ct.c_int
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().ff_status_string(int(s)).decode()


def _ptr(x) -> int | None:
    """Address of a torch tensor, NumPy array, raw int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


@dataclass
class Config:
    channels: int = 1
    scales: int = 4
    iters: int = 4
    radius_q3: int = 8
    seed_leaf: int = 8
    seed_stride: int = 1
    eps_q3: int = 8
    seed: int = 20261203
    max_width: int = 1024
    max_height: int = 1024
    patch: int = 8
    n_coeffs: int = 9
    schedule: int = FF_SCHED_BASIC
    region_min: int = 0
    wht_tensor_cores: int = 0

    def final_level(self) -> int:
        """The grid the schedule's matches come on (1 for Fast x2, else 0)."""
        return 1 if self.schedule == FF_SCHED_PLUS_FAST_X2 else 0

    def sweeps(self, level: int) -> int:
        """Sweeps of `level` under this config's schedule."""
        s = self.schedule
        if s == FF_SCHED_PLUS or (s == FF_SCHED_PLUS_FAST and level > 0) or \
                (s == FF_SCHED_PLUS_FAST_X2 and level > 1):
            return 12
        if level < self.final_level():
            return 0
        return 4 if s in (FF_SCHED_PLUS_FAST, FF_SCHED_PLUS_FAST_X2) else self.iters

    def random_searches(self, level: int) -> int:
        """Random-search passes of `level`: one after every sweep of a phase
        but its last (two phases on Flow Fields+ levels)."""
        n = self.sweeps(level)
        return n - 2 if n == 12 and self.schedule != FF_SCHED_BASIC else max(n - 1, 0)

    def c(self) -> ff_config:
        c = ff_config()
        lib().ff_config_default(ct.byref(c))
        for k, v in self.__dict__.items():
            setattr(c, k, int(v))
        return c


def ff_config_default() -> Config:
    c = ff_config()
    _check(None, lib().ff_config_default(ct.byref(c)))
    return Config(**{k: getattr(c, k) for k, _ in ff_config._fields_})


def _check(ctx, status: int):
    if status != FF_OK:
        msg = lib().ff_last_error(ctx).decode() if ctx else ""
        raise FFError(status, msg)


def ff_create(cfg: Config, device: int = 0, stream=None) -> int:
    out = ct.c_void_p()
    c = cfg.c()
    _check(None, lib().ff_create(ct.byref(c), device, _stream_handle(stream), ct.byref(out)))
    return out.value


def ff_set_stream(ctx: int, stream) -> None:
    _check(ctx, lib().ff_set_stream(ctx, _stream_handle(stream)))


def ff_features(ctx: int, slot: int, img, w: int, h: int, pitch: int) -> None:
    _check(ctx, lib().ff_features(ctx, slot, _ptr(img), w, h, pitch))


def ff_match(ctx: int, direction: int, pair_id: int, seeds_in, flow_out, cost_out=None) -> None:
    _check(ctx, lib().ff_match(ctx, direction, pair_id, _ptr(seeds_in), _ptr(flow_out),
                               _ptr(cost_out)))


def ff_match_until(ctx: int, direction: int, pair_id: int, seeds_in, until_level: int,
                   until_sweeps: int, flow_out, cost_out=None) -> None:
    _check(ctx, lib().ff_match_until(ctx, direction, pair_id, _ptr(seeds_in), until_level,
                                     until_sweeps, _ptr(flow_out), _ptr(cost_out)))


def ff_filter(ctx: int, flow_fwd, flow_bwd, mask_out) -> None:
    _check(ctx, lib().ff_filter(ctx, _ptr(flow_fwd), _ptr(flow_bwd), _ptr(mask_out)))


def ff_filter_2way(ctx: int, flow_fwd, flow_bwd1, flow_bwd2, mask_out) -> None:
    _check(ctx, lib().ff_filter_2way(ctx, _ptr(flow_fwd), _ptr(flow_bwd1), _ptr(flow_bwd2),
                                     _ptr(mask_out)))


def ff_region_filter(ctx: int, flow_fwd, mask_in, min_region: int, mask_out) -> None:
    _check(ctx, lib().ff_region_filter(ctx, _ptr(flow_fwd), _ptr(mask_in), min_region,
                                       _ptr(mask_out)))


def ff_sparsify(ctx: int, flow_fwd, flow_bwd1, flow_bwd2, mask_in, q: int, e: int,
                mask_out) -> None:
    _check(ctx, lib().ff_sparsify(ctx, _ptr(flow_fwd), _ptr(flow_bwd1), _ptr(flow_bwd2),
                                  _ptr(mask_in), q, e, _ptr(mask_out)))


def ff_wht_coeffs_scalespace_tc(img, w: int, h: int, pitch: int, channels: int, level: int,
                                fp16: bool, coeffs_out, stream=None) -> None:
    """WHT of the FP32 scale-space image in bf16 or fp16 on the tensor cores."""
    _check(None, lib().ff_wht_coeffs_scalespace_tc(_ptr(img), w, h, pitch, channels, level,
                                                   int(fp16), _ptr(coeffs_out), _stream_handle(stream)))


def ff_wht_coeffs_tc(img, w: int, h: int, pitch: int, channels: int, level: int, coeffs_out,
                     stream=None) -> None:
    _check(None, lib().ff_wht_coeffs_tc(_ptr(img), w, h, pitch, channels, level,
                                        _ptr(coeffs_out), _stream_handle(stream)))


def ff_pair_host(ctx: int, img1_host, img2_host, w: int, h: int, pair_id: int,
                 flow_fwd_host=None, flow_bwd_host=None, mask_host=None) -> None:
    _check(ctx, lib().ff_pair_host(ctx, _ptr(img1_host), _ptr(img2_host), w, h, pair_id,
                                   _ptr(flow_fwd_host), _ptr(flow_bwd_host), _ptr(mask_host)))


def ff_get_features(ctx: int, slot: int, level: int, dst) -> None:
    _check(ctx, lib().ff_get_features(ctx, slot, level, _ptr(dst)))


def ff_seed_knn(ctx: int, direction: int, idx_out, dist_out) -> None:
    _check(ctx, lib().ff_seed_knn(ctx, direction, _ptr(idx_out), _ptr(dist_out)))


def ff_seed_knn_static(feat_src0, feat_dst0, w: int, h: int, channels: int, scales: int,
                       leaf: int, stride: int, idx_out, dist_out, stream=None) -> None:
    """Allocation-free seeding search (no context; see include/ff.h)."""
    why = ct.c_char_p()
    st = lib().ff_seed_knn_static(_ptr(feat_src0), _ptr(feat_dst0), w, h, channels, scales, leaf,
                                  stride, _ptr(idx_out), _ptr(dist_out), _stream_handle(stream),
                                  ct.byref(why))
    if st != FF_OK:
        raise FFError(st, (why.value or b"").decode())


def ff_sync(ctx: int) -> None:
    _check(ctx, lib().ff_sync(ctx))


def ff_debug_set(ctx: int, key: int, value: int) -> None:
    _check(ctx, lib().ff_debug_set(ctx, key, value))


def ff_measure_peaks(device: int = 0) -> dict:
    """The device's measured ceilings (see include/ff.h): a dict of the
    ff_peaks fields."""
    out = ff_peaks()
    s = lib().ff_measure_peaks(device, ct.byref(out))
    if s != FF_OK:
        raise FFError(s, "ff_measure_peaks failed")
    return {name: getattr(out, name) for name, _ in ff_peaks._fields_}


def ff_profile(ctx: int, mode: int) -> None:
    """0 stops; FF_PROFILE_LAUNCHES (or True) times every launch;
    FF_PROFILE_SWEEP_RUNS times each run of consecutive sweep launches."""
    _check(ctx, lib().ff_profile(ctx, int(mode)))


def ff_kernel_stats(ctx: int, kernel: str) -> tuple[int, float]:
    """(launches, summed device ms) of `kernel` recorded since ff_profile started."""
    n = ct.c_longlong(0)
    ms = ct.c_double(0.0)
    _check(ctx, lib().ff_kernel_stats(ctx, kernel.encode(), ct.byref(n), ct.byref(ms)))
    return int(n.value), float(ms.value)


KERNELS = ("k_features", "k_seed_prep", "k_seed_scan", "k_seed_merge", "k_seed_rerank", "k_seed_given",
           "k_upsample", "k_sweep", "k_export", "k_filter", "k_dense", "k_region",
           "k_sparsify")


def ff_launch_count(ctx: int) -> int:
    return int(lib().ff_launch_count(ctx))


def ff_last_error(ctx: int) -> str:
    return lib().ff_last_error(ctx).decode()


def ff_destroy(ctx: int) -> None:
    lib().ff_destroy(ctx)


# ----------------------------------------------------------------------------
# a small convenience layer over the same calls (torch device tensors)
# ----------------------------------------------------------------------------
def level_dims(w: int, h: int, level: int) -> tuple[int, int]:
    n = 1 << level
    return (w + n - 1) // n, (h + n - 1) // n


class Context:
    """Owns one ff_ctx; frames and outputs are torch CUDA tensors."""

    def __init__(self, cfg: Config, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.ctx = ff_create(cfg, device, stream)
        self.size = None

    def close(self):
        if self.ctx:
            ff_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def features(self, slot: int, img) -> None:
        """img: uint8 CUDA tensor [C][H][W] (contiguous)."""
        assert img.is_cuda and img.dtype == self.torch.uint8 and img.is_contiguous()
        C, H, W = img.shape
        assert C == self.cfg.channels
        ff_features(self.ctx, slot, img, W, H, W)
        self.size = (W, H)

    def match(self, direction: int, pair_id: int = 0, seeds_in=None,
              until_level: int | None = None, until_sweeps: int | None = None,
              with_cost: bool = True):
        torch = self.torch
        W, H = self.size
        Lf = self.cfg.final_level()
        if until_level is None:
            until_level = Lf
        if until_sweeps is None:
            until_sweeps = self.cfg.sweeps(until_level)
        WL, HL = level_dims(W, H, until_level)
        dev = torch.device("cuda", self.device)
        flow = torch.empty((HL, WL, 2), dtype=torch.int16, device=dev)
        cost = torch.empty((HL, WL), dtype=torch.int32, device=dev) if with_cost else None
        if until_level == Lf and until_sweeps == self.cfg.sweeps(Lf):
            ff_match(self.ctx, direction, pair_id, seeds_in, flow, cost)
        else:
            ff_match_until(self.ctx, direction, pair_id, seeds_in, until_level, until_sweeps,
                           flow, cost)
        return flow, cost

    def filter(self, flow_fwd, flow_bwd):
        torch = self.torch
        WL, HL = level_dims(*self.size, self.cfg.final_level())
        mask = torch.empty((HL, WL), dtype=torch.uint8, device=flow_fwd.device)
        ff_filter(self.ctx, flow_fwd, flow_bwd, mask)
        return mask

    def filter_2way(self, flow_fwd, flow_bwd1, flow_bwd2):
        torch = self.torch
        WL, HL = level_dims(*self.size, self.cfg.final_level())
        mask = torch.empty((HL, WL), dtype=torch.uint8, device=flow_fwd.device)
        ff_filter_2way(self.ctx, flow_fwd, flow_bwd1, flow_bwd2, mask)
        return mask

    def region_filter(self, flow_fwd, mask, min_region: int):
        out = self.torch.empty_like(mask)
        ff_region_filter(self.ctx, flow_fwd, mask, min_region, out)
        return out

    def sparsify(self, flow_fwd, flow_bwd1, flow_bwd2, mask, q: int, e: int):
        out = self.torch.empty_like(mask)
        ff_sparsify(self.ctx, flow_fwd, flow_bwd1, flow_bwd2, mask, q, e, out)
        return out

    def features_of(self, slot: int, level: int):
        torch = self.torch
        W, H = self.size
        WL, HL = level_dims(W, H, level)
        out = torch.empty((HL, WL, 9 * self.cfg.channels), dtype=torch.int8,
                          device=torch.device("cuda", self.device))
        ff_get_features(self.ctx, slot, level, out)
        return out

    def seed_knn(self, direction: int):
        torch = self.torch
        W, H = self.size
        WS, HS = level_dims(W, H, self.cfg.scales - 1)
        dev = torch.device("cuda", self.device)
        idx = torch.empty((HS, WS, self.cfg.seed_leaf), dtype=torch.int32, device=dev)
        dist = torch.empty_like(idx)
        ff_seed_knn(self.ctx, direction, idx, dist)
        return idx, dist

    def sync(self):
        ff_sync(self.ctx)


# ---- batched form ----------------------------------------------------------
def _bcheck(b, status: int):
    if status != FF_OK:
        msg = lib().ff_batch_last_error(b).decode() if b else ""
        raise FFError(status, msg)


def ff_batch_create(cfg: Config, device: int = 0, slots: int = 8, stream=None) -> int:
    out = ct.c_void_p()
    c = cfg.c()
    _bcheck(None, lib().ff_batch_create(ct.byref(c), device, slots, _stream_handle(stream),
                                        ct.byref(out)))
    return out.value


def pair_descs(pairs) -> ct.Array:
    """ff_pair_desc array from dicts with keys img1, img2, w, h, pitch (default
    w), pair_id, flow_fwd, flow_bwd, flow_bwd2 (optional), mask (optional)."""
    arr = (ff_pair_desc * max(len(pairs), 1))()
    for k, p in enumerate(pairs):
        arr[k] = ff_pair_desc(_ptr(p["img1"]), _ptr(p["img2"]), p["w"], p["h"],
                              p.get("pitch", p["w"]), p.get("pair_id", 0), _ptr(p["flow_fwd"]),
                              _ptr(p["flow_bwd"]), _ptr(p.get("flow_bwd2")), _ptr(p.get("mask")))
    return arr


def ff_batch_run(b: int, descs, n: int | None = None, use_graph: bool = False) -> None:
    if not isinstance(descs, ct.Array):
        n = len(descs)
        descs = pair_descs(descs)
    _bcheck(b, lib().ff_batch_run(b, len(descs) if n is None else n, descs, int(use_graph)))


def ff_batch_set_stream(b: int, stream) -> None:
    _bcheck(b, lib().ff_batch_set_stream(b, _stream_handle(stream)))


def ff_batch_sync(b: int) -> None:
    _bcheck(b, lib().ff_batch_sync(b))


def ff_batch_debug_set(b: int, key: int, value: int) -> None:
    _bcheck(b, lib().ff_batch_debug_set(b, key, value))


def ff_batch_launch_count(b: int) -> int:
    return int(lib().ff_batch_launch_count(b))


def ff_batch_destroy(b: int) -> None:
    lib().ff_batch_destroy(b)


# ---- serving loop ------------------------------------------------------------
def _scheck(v, status: int):
    if status != FF_OK:
        msg = lib().ff_server_last_error(v).decode() if v else ""
        raise FFError(status, msg)


def ff_slot_bytes(cfg: Config) -> int:
    c = cfg.c()
    return int(lib().ff_slot_bytes(ct.byref(c)))


def ff_server_create(cfg: Config, device: int = 0, mem_budget: int = 8 << 30,
                     max_slots: int = 64) -> int:
    out = ct.c_void_p()
    c = cfg.c()
    _scheck(None, lib().ff_server_create(ct.byref(c), device, mem_budget, max_slots,
                                         ct.byref(out)))
    return out.value


def ff_server_slots(v: int) -> int:
    return int(lib().ff_server_slots(v))


def host_pair(img1, img2, w: int, h: int, pitch: int | None = None, plane: int | None = None,
              pair_id: int = 0, two_way: bool = False, flow_fwd=None, flow_bwd=None,
              flow_bwd2=None, mask=None) -> ff_host_pair:
    pitch = w if pitch is None else pitch
    plane = h * pitch if plane is None else plane
    return ff_host_pair(_ptr(img1), _ptr(img2), w, h, pitch, plane, pair_id, int(two_way),
                        _ptr(flow_fwd), _ptr(flow_bwd), _ptr(flow_bwd2), _ptr(mask))


def ff_server_submit(v: int, req: ff_host_pair) -> int:
    t = ct.c_longlong()
    _scheck(v, lib().ff_server_submit(v, ct.byref(req), ct.byref(t)))
    return t.value


def ff_server_poll(v: int, cap: int = 256) -> list[tuple[int, int]]:
    tickets = (ct.c_longlong * cap)()
    status = (ct.c_int * cap)()
    n = ct.c_int()
    _scheck(v, lib().ff_server_poll(v, tickets, status, cap, ct.byref(n)))
    return [(tickets[k], status[k]) for k in range(n.value)]


def ff_server_pending(v: int) -> int:
    return int(lib().ff_server_pending(v))


def ff_server_launch_count(v: int) -> int:
    return int(lib().ff_server_launch_count(v))


def ff_server_destroy(v: int) -> None:
    lib().ff_server_destroy(v)
