#!/usr/bin/env python3
"""Throughput of the Flow Fields matching loop on GB300.

One step = one frame pair of the Sintel-shaped workload (1024x436, 8-bit
CIELab, 4 scales, 6 sweeps per scale, R = 1 px): features of both frames,
forward and backward matching (on two streams), consistency filter.  Inputs
are resident in device memory when the timed region starts; L2 is flushed
between steps (a 256 MiB write, outside the per-step events).

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead on a
bounded sample of the same workload.  With ``--gpus N`` (torchrun), the N
ranks run independent replicas (the method does not shard within a pair).
``--schedule`` selects Flow Fields+ (Sec. 3.3), Fast or Fast x2 (Sec. 3.4)
instead of the basic schedule; ``--two-way`` adds the second backward flow
and the two-way check of Sec. 3.7 to every step.

``--serve`` instead runs the serving loop (``ff_server_*``) on a Poisson
stream of host-buffer requests over independent layered pairs of sizes
256x256 .. 1920x1080 (64-px steps): capacity (all requests at once), then
p50 / p99 latency at fractions of that rate.

The line's ``batched`` object times the batched form (``ff_batch_run``, one
CUDA graph per step, pairs overlapping in matching slots) on two batches:
32 Sintel-shaped pairs (distinct seeds) and 64 pairs of mixed sizes
(320x240, 640x480, 1024x436, 1242x375).  Its ``serving`` object runs the
serving loop on a shorter stream of the same kind (capacity and one Poisson
load point at 0.8 of it).  ``roofline`` quotes the dominant kernel against
ceilings measured on the running GPU (ff_measure_peaks).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# many streams run concurrently (matching slots, side streams): give them
# more hardware work queues than the default 8 (a per-process setting, read
# when CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "candidate patch evals/s and frame pairs/s (fwd+bwd) at 1024x436; % of int/L2 roofline"
WORKLOAD = "sintel1024x436"


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------
SCHEDULES = {"basic": 0, "plus": 1, "fast": 2, "fast_x2": 3}


def level_dims(W: int, H: int, L: int) -> tuple[int, int]:
    s = 1 << L
    return (W + s - 1) // s, (H + s - 1) // s


def sweep_evals(W: int, H: int, cfg) -> int:
    """Cost evaluations of all propagation sweeps + random searches of one
    direction: per level and sweep 2 candidates per point (one fewer on the
    two incoming borders), per random search 1 candidate per point."""
    n = 0
    for L in range(cfg.scales):
        wl, hl = level_dims(W, H, L)
        n += cfg.sweeps(L) * (2 * wl * hl - wl - hl) + cfg.random_searches(L) * wl * hl
    return n


def eval_count(W: int, H: int, cfg) -> int:
    """Cost evaluations of one direction: seeding rerank (l per coarsest
    point), upsample re-evaluations of carried points, sweeps and searches."""
    S = cfg.scales
    ws, hs = level_dims(W, H, S - 1)
    n = cfg.seed_leaf * ws * hs + sweep_evals(W, H, cfg)
    for L in range(cfg.final_level(), S - 1):
        wl, hl = level_dims(W, H, L + 1)
        n += wl * hl
    return n


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ----------------------------------------------------------------------------
# CPU oracle (the baseline and the reference arm)
# ----------------------------------------------------------------------------
# coarsest-grid query rows of the exact seeding search timed per direction in
# one bounded oracle sample (the same for the CPU baseline and the reference arm)
ORACLE_SEED_ROWS = 3


def cpu_oracle_rate(pair, prm, schedule: int = 0, two_way: bool = False, region: int = 0,
                    budget_rows: int = ORACLE_SEED_ROWS) -> dict:
    """Time the oracle, as it stands, on a bounded sample of one pair.

    Features of both frames, the full propagation of both directions (seeded
    from the ground truth, which performs the same evaluations as any other
    seeds), and the consistency filter run in full; the exact seeding search,
    the slow part, runs for `budget_rows` rows of coarsest-grid queries per
    direction and is scaled to all rows.  Single thread.
    """
    import oracle as O
    C, S, I, R = prm["channels"], prm["scales"], prm["iters"], prm["radius_q3"]
    W, H = pair.width, pair.height
    stride = 2 if schedule == SCHEDULES["fast_x2"] else 1
    P = O.Params(channels=C, scales=S, iters=I, radius_q3=R, schedule=schedule, seed_stride=stride)
    N = 1 << (S - 1)
    WS, HS = O.level_dims(W, H, S - 1)
    gt = np.rint(pair.flow * 8).astype(np.int16)
    t_all = time.perf_counter()
    t0 = time.perf_counter()
    f1 = O.features_all(pair.img1, S)
    f2 = O.features_all(pair.img2, S)
    t_feat = time.perf_counter() - t0
    t_seed = 0.0
    t_prop = 0.0
    rows = min(budget_rows, HS)
    flows = []
    dirs = [(f1, f2, gt), (f2, f1, -gt)] + ([(f2, f1, -gt)] if two_way else [])
    for d, (a, b, g) in enumerate(dirs):
        t0 = time.perf_counter()
        O.seed_knn_rows(a[0], b[0], S, 0, rows, 8, stride)
        t_seed += (time.perf_counter() - t0) * HS / rows
        seeds = np.ascontiguousarray(g[::N, ::N][:HS, :WS])
        t0 = time.perf_counter()
        fl, _, _ = O.match_features(P, a, b, W, H, d, 0, seeds_in=seeds)
        t_prop += time.perf_counter() - t0
        flows.append(fl)
    t0 = time.perf_counter()
    Lf = P.final_level()
    if two_way:
        mask = O.filter_mask2(flows[0], flows[1], flows[2], 8, level=Lf)
    else:
        mask = O.filter_mask(flows[0], flows[1], 8, level=Lf)
    if region:
        O.region_filter(flows[0], mask, region)
    t_filt = time.perf_counter() - t0
    wall = time.perf_counter() - t_all
    per_pair = t_feat + t_seed + t_prop + t_filt
    return {"pairs_per_s": 1.0 / per_pair, "s_per_pair": per_pair, "wall_s": wall,
            "parts_s": {"features": t_feat, "seeding_scaled": t_seed, "propagation": t_prop,
                        "filter": t_filt},
            "sample": (f"one {W}x{H} pair: features, propagation ({len(dirs)} directions) "
                       f"and filter in full; exact seeding on {rows} of {HS} query rows per "
                       f"direction, scaled by {HS}/{rows}"),
            "cores": 1}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_gpu(args, rank: int, world: int, local_rank: int) -> dict:
    import torch

    from paper_1703_02563_gb300 import ff, workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pair, prm = workloads.make_workload(args.workload)
    C, S, I, R = prm["channels"], prm["scales"], prm["iters"], prm["radius_q3"]
    W, H = pair.width, pair.height
    schedule = SCHEDULES[args.schedule]
    cfg = ff.Config(channels=C, scales=S, iters=I, radius_q3=R, max_width=W, max_height=H,
                    schedule=schedule, seed_stride=2 if args.schedule == "fast_x2" else 1,
                    region_min=args.region, wht_tensor_cores=int(args.wht_tc))
    WL, HL = level_dims(W, H, cfg.final_level())
    main = torch.cuda.Stream(dev)
    side = torch.cuda.Stream(dev)
    side2 = torch.cuda.Stream(dev)
    ctx = ff.ff_create(cfg, local_rank, main)
    if args.sweep_lanes:
        ff.ff_debug_set(ctx, ff.FF_DEBUG_SWEEP_LANES, args.sweep_lanes)
    if args.seed_path == "mma":
        ff.ff_debug_set(ctx, ff.FF_DEBUG_SEED_TC, 0)
    peaks = ff.ff_measure_peaks(local_rank)
    img1 = torch.from_numpy(pair.img1).to(dev)
    img2 = torch.from_numpy(pair.img2).to(dev)
    flow_f = torch.empty((HL, WL, 2), dtype=torch.int16, device=dev)
    flow_b = torch.empty((HL, WL, 2), dtype=torch.int16, device=dev)
    flow_b2 = torch.empty((HL, WL, 2), dtype=torch.int16, device=dev)
    mask = torch.empty((HL, WL), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev_fork = torch.cuda.Event()
    ev_join = torch.cuda.Event()
    ev_join2 = torch.cuda.Event()
    ev_feat = torch.cuda.Event()

    def step(pair_id: int, i1=img1, i2=img2):
        # the two frames' features on the main and side streams (each stream
        # then waits for the other's); the backward flow(s) on side streams
        # overlap the forward flow; the filter joins them
        ev_fork.record(main)
        side.wait_event(ev_fork)
        ff.ff_set_stream(ctx, main)
        ff.ff_features(ctx, 0, i1, W, H, W)
        ff.ff_set_stream(ctx, side)
        ff.ff_features(ctx, 1, i2, W, H, W)
        ev_fork.record(main)
        ev_feat.record(side)
        side.wait_event(ev_fork)
        main.wait_event(ev_feat)
        ff.ff_set_stream(ctx, side)
        ff.ff_match(ctx, ff.FF_BWD, pair_id, None, flow_b, None)
        if args.two_way:
            side2.wait_event(ev_fork)
            side2.wait_event(ev_feat)
            ff.ff_set_stream(ctx, side2)
            ff.ff_match(ctx, ff.FF_BWD2, pair_id, None, flow_b2, None)
        ff.ff_set_stream(ctx, main)
        ff.ff_match(ctx, ff.FF_FWD, pair_id, None, flow_f, None)
        ev_join.record(side)
        main.wait_event(ev_join)
        if args.two_way:
            ev_join2.record(side2)
            main.wait_event(ev_join2)
            ff.ff_filter_2way(ctx, flow_f, flow_b, flow_b2, mask)
        else:
            ff.ff_filter(ctx, flow_f, flow_b, mask)
        if args.region:
            ff.ff_region_filter(ctx, flow_f, mask, args.region, mask)

    for i in range(args.warmup):
        step(replica_pair_id(rank, i))
    torch.cuda.synchronize()
    ff.ff_sync(ctx)

    # ---- timed region: device-resident inputs, per-step events, L2 flushed between
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    launches0 = ff.ff_launch_count(ctx)
    # the dominant kernel is timed live: one event pair per run of a level's
    # sweeps (per-launch events would cost ~2% of the step)
    ff.ff_profile(ctx, ff.FF_PROFILE_SWEEP_RUNS)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        with torch.cuda.stream(main):
            flush.fill_(i & 0xff)
        starts[i].record(main)
        step(replica_pair_id(rank, args.warmup + i))
        ends[i].record(main)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ff.ff_sync(ctx)
    ff.ff_profile(ctx, 0)
    launches = ff.ff_launch_count(ctx) - launches0
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    sweep_live = ff.ff_kernel_stats(ctx, "k_sweep")
    # the last timed step's forward flow and mask (for `accuracy`)
    timed_flow, timed_mask = flow_f.cpu().numpy(), mask.cpu().numpy()
    # every kernel's launches timed one by one, over as many steps again right
    # after the timed region: the shares and kernels_ms
    ff.ff_profile(ctx, ff.FF_PROFILE_LAUNCHES)
    for i in range(args.steps):
        with torch.cuda.stream(main):
            flush.fill_(i & 0xff)
        step(replica_pair_id(rank, args.warmup + args.steps + i))
    torch.cuda.synchronize()
    ff.ff_sync(ctx)
    ff.ff_profile(ctx, 0)
    kstats = {k: ff.ff_kernel_stats(ctx, k) for k in ff.KERNELS}

    # ---- end to end from pinned host buffers: ff_pair_host (one backward
    # flow), or the device calls above with the copies around them (two)
    h1 = torch.from_numpy(pair.img1.copy()).pin_memory()
    h2 = torch.from_numpy(pair.img2.copy()).pin_memory()
    hf = torch.empty((HL, WL, 2), dtype=torch.int16).pin_memory()
    hb = torch.empty((HL, WL, 2), dtype=torch.int16).pin_memory()
    hb2 = torch.empty((HL, WL, 2), dtype=torch.int16).pin_memory()
    hm = torch.empty((HL, WL), dtype=torch.uint8).pin_memory()
    d1, d2 = torch.empty_like(img1), torch.empty_like(img2)

    def host_step(pair_id: int):
        if not args.two_way:
            ff.ff_pair_host(ctx, h1, h2, W, H, pair_id, hf, hb, hm)
            return
        with torch.cuda.stream(main):
            d1.copy_(h1, non_blocking=True)
            d2.copy_(h2, non_blocking=True)
        step(pair_id, d1, d2)
        with torch.cuda.stream(main):
            for dst, src in ((hf, flow_f), (hb, flow_b), (hb2, flow_b2), (hm, mask)):
                dst.copy_(src, non_blocking=True)
        main.synchronize()
        ff.ff_sync(ctx)

    ff.ff_set_stream(ctx, main)
    for i in range(2):
        host_step(replica_pair_id(rank, i))
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        host_step(replica_pair_id(rank, i))
    e2e_s = time.perf_counter() - t0
    n_out = 3 if args.two_way else 2
    e2e_bytes = (2 * C * W * H, n_out * 4 * WL * HL + WL * HL)
    accuracy = flow_accuracy(timed_flow, timed_mask, pair, cfg.final_level())
    ff.ff_destroy(ctx)
    return {"total_ms": total_ms, "step_ms": step_ms, "kstats": kstats, "sweep_live": sweep_live,
            "launches": launches,
            "peaks": peaks,
            "accuracy": accuracy,
            "clocks": clocks, "e2e_s": e2e_s, "e2e_bytes": e2e_bytes, "W": W, "H": H, "C": C,
            "S": S, "I": I, "cfg": cfg, "prm": prm, "pair": pair, "workload": args.workload}


# Algorithmic integer operations of the matching error per feature dimension:
# the bilinear interpolation's 4 multiply-adds (2 ops each), the subtraction
# of 64 q, the absolute value and the accumulation.
OPS_PER_DIM = 11


def sweep_diagonals(W: int, H: int, cfg) -> int:
    """Anti-diagonals of every propagation sweep of one direction: the
    sequential steps the raster order leaves (a point waits for its left and
    upper neighbours), U_L + V_L - 1 per sweep of level L."""
    n = 0
    for L in range(cfg.scales):
        wl, hl = level_dims(W, H, L)
        n += cfg.sweeps(L) * (wl + hl - 1)
    return n


def step_floor_cycles(peaks: dict) -> float:
    """Dependent latency of one wavefront step of the sweep, from measured
    instruction latencies: the row above's decision arrives by a shuffle;
    selecting and clamping the candidate (4 ALU), its tap address (9 ALU:
    sign extension, rounding to the level, column and row offsets, 64-bit
    address), one L1-hit load, the byte transpose (2 permutes), one dp4a,
    absolute value and accumulation (3 ALU), the two-level shuffle exchange
    of the costs (2 shuffles, 1 add) and the argmin over [current, vertical,
    horizontal] into the next step's horizontal source (7 ALU)."""
    return (3 * peaks["lat_shfl"] + peaks["lat_ldg_l1"] + 2 * peaks["lat_prmt"]
            + peaks["lat_dp4a"] + 24 * peaks["lat_alu"])


# ----------------------------------------------------------------------------
# replicas (--gpus N): every rank matches its own pairs; no data-path exchange
# ----------------------------------------------------------------------------
def flow_accuracy(flow_q3: np.ndarray, mask: np.ndarray, pair, level: int = 0) -> dict:
    """End-point error of a forward flow (1/8 px, on the level-`level` grid)
    against the generator's ground truth, over all points, the visible ones
    (not occluded) and the ones the filter kept; and the kept fraction."""
    n = 1 << level
    gt = pair.flow[::n, ::n][:flow_q3.shape[0], :flow_q3.shape[1]]
    occ = pair.occ[::n, ::n][:flow_q3.shape[0], :flow_q3.shape[1]]
    valid = flow_q3[..., 0] != -32768
    f = flow_q3.astype(np.float64) / 8.0
    err = np.hypot(f[..., 0] - gt[..., 0], f[..., 1] - gt[..., 1])
    kept = (mask != 0) & valid
    vis = valid & ~occ
    mean = lambda m: float(err[m].mean()) if m.any() else None
    return {"epe_all": mean(valid), "epe_visible": mean(vis), "epe_kept": mean(kept),
            "kept_fraction": float(kept.mean()),
            "outliers_3px_visible": float((err[vis] > 3.0).mean()) if vis.any() else None,
            "outliers_3px_kept": float((err[kept] > 3.0).mean()) if kept.any() else None}


def replica_pair_id(rank: int, k: int) -> int:
    """Random-search key word of the k-th pair of a rank: ranks never share one."""
    return rank * 1_000_000 + k


def replica_times(times: list[float], world: int, device: str) -> list[float]:
    """Each timing's maximum over the ranks: the job is as slow as its slowest
    replica.  Needs an initialised process group when world > 1."""
    if world == 1:
        return list(times)
    import torch
    t = torch.tensor(times, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def replica_throughput(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the units of all ranks over the slowest rank's time."""
    return units_per_rank * world / seconds


def run_batched(pairs, prm, slots: int, steps: int, warmup: int, local_rank: int,
                sweep_lanes: int = 0, autotune: bool = False, peak_tops: float | None = None) -> dict:
    """Throughput of the batched form on `pairs` (inputs resident, L2
    flushed between steps, one graph launch per step timed with CUDA events
    on the batch's stream)."""
    import torch

    from paper_1703_02563_gb300 import ff

    dev = torch.device("cuda", local_rank)
    W = max(p.width for p in pairs)
    H = max(p.height for p in pairs)
    cfg = ff.Config(channels=prm["channels"], scales=prm["scales"], iters=prm["iters"],
                    radius_q3=prm["radius_q3"], max_width=W, max_height=H)
    stream = torch.cuda.Stream(dev)
    imgs = [(torch.from_numpy(p.img1).to(dev), torch.from_numpy(p.img2).to(dev)) for p in pairs]
    outs = [tuple(torch.empty(s, dtype=t, device=dev)
                  for s, t in (((p.height, p.width, 2), torch.int16),
                               ((p.height, p.width, 2), torch.int16),
                               ((p.height, p.width), torch.uint8))) for p in pairs]
    descs = ff.pair_descs([dict(img1=i1, img2=i2, w=p.width, h=p.height, pair_id=k,
                                flow_fwd=o[0], flow_bwd=o[1], mask=o[2])
                           for k, (p, (i1, i2), o) in enumerate(zip(pairs, imgs, outs))])
    tuned = None
    if autotune:
        from paper_1703_02563_gb300 import autotune as at
        tuned = at.tune(cfg, descs, len(pairs), local_rank)
        slots, sweep_lanes = tuned["slots"], tuned["lanes"]
    b = ff.ff_batch_create(cfg, local_rank, slots=slots, stream=stream)
    if sweep_lanes:
        ff.ff_batch_debug_set(b, ff.FF_DEBUG_SWEEP_LANES, sweep_lanes)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(warmup):
        ff.ff_batch_run(b, descs, use_graph=True)
    ff.ff_batch_sync(b)
    n0 = ff.ff_batch_launch_count(b)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        ff.ff_batch_run(b, descs, use_graph=True)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ff.ff_batch_sync(b)
    launches = ff.ff_batch_launch_count(b) - n0
    ff.ff_batch_destroy(b)
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_s = sum(ms) / 1e3
    evals = sum(2 * eval_count(p.width, p.height, cfg) for p in pairs) * steps
    sweep_ops = sum(2 * sweep_evals(p.width, p.height, cfg) for p in pairs) * steps \
        * 9 * prm["channels"] * OPS_PER_DIM
    return {"value": len(pairs) * steps / total_s, "unit": "pairs/s", "pairs": len(pairs),
            "slots": slots, "steps": steps, "ms_per_batch": total_s * 1e3 / steps,
            "evals_per_s": evals / total_s, "gpu_launches": launches,
            # a lower bound on k_sweep's fraction of the measured per-dimension
            # arithmetic peak: all of the step's time charged to the sweeps
            "sweep_alu_frac_of_step": (sweep_ops / total_s / 1e12 / peak_tops)
            if peak_tops else None,
            "sizes": sorted({f"{p.width}x{p.height}" for p in pairs}),
            **({"autotune": tuned} if tuned else {})}


def code_hash(paths: list[str]) -> str:
    """SHA-256 of C/CUDA sources with comments removed and whitespace runs
    collapsed (string literals kept as they are): a change to the code changes
    it, a change to a comment does not."""
    import hashlib
    import re
    tok = re.compile(r'"(?:\\.|[^"\\])*"|//[^\n]*|/\*.*?\*/', re.S)
    parts = []
    for p in paths:
        text = open(os.path.join(ROOT, p), encoding="utf-8").read()
        text = tok.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", text)
        parts.append(" ".join(text.split()))
    return hashlib.sha256("\n".join(parts).encode()).hexdigest()


def recorded_counters(kernel: str, workload: str) -> dict | None:
    """Per-launch counters of a kernel from the committed ncu summary, if they
    were taken on this workload and the kernel's code is unchanged since."""
    try:
        with open(os.path.join(ROOT, "profiles", f"{kernel}_counters.json")) as f:
            rec = json.load(f)
        if code_hash(rec["sources"]) != rec["code_sha256"] or rec["workload"] != workload:
            return None
        return rec
    except (OSError, KeyError, ValueError):
        return None


def roofline(res: dict, steps: int, n_dirs: int) -> dict:
    """Roofline of the kernel with the largest share of device time.

    k_sweep (propagation + random search) is integer-ALU work on a serial
    wavefront.  Its algorithmic work is OPS_PER_DIM integer operations per
    feature dimension per evaluation (evaluations per launch from
    sweep_evals); the peak is the same arithmetic's measured throughput
    (ff_measure_peaks: sad_dims_per_s x OPS_PER_DIM), with the dp4a
    instruction peak (8 ops per dp4a) beside it.  Its L2 fraction is the L2
    traffic of one launch (ncu record) over the launch time, against the
    measured L2 read bandwidth.  Its critical path is the cycles per
    anti-diagonal (device time x SM clock over the sweeps' anti-diagonals)
    against the dependent latency of one step (step_floor_cycles).
    k_seed_scan (the tensor-core seeding) is a dense contraction: 2 flops per
    multiply-add of (queries x candidates x K), against the measured bf16
    tensor peak.
    """
    ks = res["kstats"]
    peaks = res["peaks"]
    tot = {k: v[1] for k, v in ks.items()}
    dom = max(tot, key=lambda k: tot[k])
    n_launch, ms = ks[dom]
    W, H, C, S, I = res["W"], res["H"], res["C"], res["S"], res["I"]
    share = ms / sum(tot.values())
    timing = "per-launch events in a profiled pass of the same steps after the timed region"
    if dom == "k_sweep" and res.get("sweep_live") and res["sweep_live"][0]:
        # live: CUDA events over the timed region, one pair per run of
        # consecutive sweeps on a stream (the run includes its launch gaps)
        n_launch, ms = res["sweep_live"]
        timing = ("CUDA events over the timed region on the launching streams, one pair per run "
                  "of a level's sweeps (launch gaps inside a run included)")
    avg_ms = ms / max(n_launch, 1)
    if dom == "k_sweep":
        dims = n_dirs * steps * sweep_evals(W, H, res["cfg"]) * 9 * C / max(n_launch, 1)
        achieved = dims * OPS_PER_DIM / (avg_ms / 1e3) / 1e12
        peak = peaks["sad_dims_per_s"] * OPS_PER_DIM / 1e12
        dp4a_peak = peaks["dp4a_per_s"] * 8 / 1e12
        rec = recorded_counters(dom, res["workload"])
        l2 = None
        traffic = None
        if rec:
            traffic = rec["dram_bytes_per_launch"]
            l2_gbs = rec["l2_bytes_per_launch"] / (avg_ms / 1e3) / 1e9
            l2 = {"achieved": l2_gbs, "peak": peaks["l2_read_gbs"], "unit": "GB/s",
                  "frac": l2_gbs / peaks["l2_read_gbs"],
                  "l2_bytes_per_launch": rec["l2_bytes_per_launch"],
                  "source": "ncu lts__t_bytes.sum per launch (profiles/k_sweep_counters.json) "
                            "over the live launch time; peak measured by ff_measure_peaks"}
        clk = res["clocks"].get("sm_mhz") or 2070.0
        diags = n_dirs * steps * sweep_diagonals(W, H, res["cfg"])
        cyc = ms / 1e3 * clk * 1e6 / diags
        floor = step_floor_cycles(peaks)
        return {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Tops/s", "frac": achieved / peak, "traffic": traffic,
                "launches": n_launch, "avg_launch_ms": avg_ms, "share": share, "timing": timing,
                "share_source": "per-launch events in a profiled pass of the same steps after "
                                "the timed region",
                "peak_source": "measured (ff_measure_peaks): the matching error's per-dimension "
                               f"arithmetic at full occupancy, {OPS_PER_DIM} ops per dimension",
                "dp4a_peak": dp4a_peak, "frac_of_dp4a_peak": achieved / dp4a_peak,
                "l2": l2,
                "critical_path": {"cycles_per_step": cyc, "floor_cycles": floor,
                                  "frac": floor / cyc, "sm_mhz": clk,
                                  "steps": "anti-diagonals U_L + V_L - 1 of every sweep",
                                  "floor": "dependent latency of one step from measured "
                                           "instruction latencies (step_floor_cycles)"}}
    if dom == "k_seed_scan":
        N = 1 << (S - 1)
        nq = ((W + N - 1) // N) * ((H + N - 1) // N)
        K = 16 if C == 1 else 32
        ncand = ((W + 1) // 2) * ((H + 1) // 2) if res["cfg"].seed_stride == 2 else W * H
        flops = n_dirs * steps * 2 * nq * ncand * K * 2 * (1 + 1 / 16) / max(n_launch, 1)
        peak = measured_peaks().get("bf16_tflops", 1900.0)
        achieved = flops / (avg_ms / 1e3) / 1e12
        return {"kernel": dom, "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "launches": n_launch, "avg_launch_ms": avg_ms, "share": share, "timing": timing,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (measured)"}
    return {"kernel": dom, "bound": "alu", "achieved": None, "peak": None,
            "unit": "Tops/s", "frac": None, "traffic": None, "launches": n_launch,
            "avg_launch_ms": avg_ms, "share": share}


def _fp64_scalespace_wht(img: np.ndarray, L: int) -> np.ndarray:
    """FP64 WHT of the scale-space image (the n x n block mean without
    rounding, replicate border): separable +-1 sums over the 8 x 8 window at
    offsets -3..+4, rows (u) then columns (v); [HL][WL][9C], dim c*9 + 3u + v."""
    C, H, W = img.shape
    n = 1 << L
    WL, HL = -(-W // n), -(-H // n)
    pad = np.pad(img.astype(np.float64), ((0, 0), (0, HL * n - H), (0, WL * n - W)), mode="edge")
    D = np.pad(pad.reshape(C, HL, n, WL, n).mean(axis=(2, 4)), ((0, 0), (3, 4), (3, 4)),
               mode="edge")
    walsh = np.array([[1] * 8, [1] * 4 + [-1] * 4, [1, 1, -1, -1, -1, -1, 1, 1]], np.float64)
    out = np.zeros((HL, WL, C, 3, 3))
    for u in range(3):
        rows = sum(walsh[u, i] * D[:, i:i + HL, :] for i in range(8))        # C, HL, WL+7
        for v in range(3):
            out[:, :, :, u, v] = np.moveaxis(
                sum(walsh[v, j] * rows[:, :, j:j + WL] for j in range(8)), 0, -1)
    return out.reshape(HL, WL, 9 * C)


def precision_form(pair, scales: int, local_rank: int) -> dict:
    """The precision form: the WHT of the FP32 scale-space image on the
    tensor cores in bf16 and fp16 (FP32 accumulation) against FP64, per
    level: max |coefficient error|, the bound the format's rounding allows,
    and the int8 codes that differ from the FP64 coefficients' codes."""
    import torch

    from paper_1703_02563_gb300 import ff

    C, H, W = pair.img1.shape
    img = torch.from_numpy(pair.img1).cuda(local_rank)
    half_ulp = {"bf16": 0.5, "fp16": 1.0 / 16.0}

    def codes(c):
        q = np.floor(c / 16.0 + 0.5)
        q[..., 0::9] = np.floor(c[..., 0::9] / 64.0 + 0.5) - 128
        return np.clip(q, -128, 127)

    out = {}
    for fmt in ("bf16", "fp16"):
        levels = []
        for L in range(scales):
            WL, HL = level_dims(W, H, L)
            t = torch.empty((HL, WL, 9 * C), dtype=torch.float32, device=img.device)
            ff.ff_wht_coeffs_scalespace_tc(img, W, H, W, C, L, fmt == "fp16", t)
            got = t.cpu().numpy().astype(np.float64)
            ref = _fp64_scalespace_wht(pair.img1, L)
            flips = int((codes(got) != codes(ref)).sum())
            levels.append({"level": L, "max_abs_err": float(np.abs(got - ref).max()),
                           "bound": 0.0 if L == 0 else 64 * half_ulp[fmt] + 64 * 2.0 ** -11,
                           "int8_flips": flips, "codes": int(got.size)})
        out[fmt] = {"levels": levels,
                    "max_abs_err": max(x["max_abs_err"] for x in levels),
                    "int8_flips": sum(x["int8_flips"] for x in levels),
                    "codes": sum(x["codes"] for x in levels)}
    out["note"] = ("FP32 scale-space image (area average without rounding) in bf16/fp16 on the "
                   "tensor cores, FP32 accumulation, against an FP64 transform; matching uses "
                   "the rounded integer level image and stays bit-exact")
    return out


def run_serving(pairs, reqs, fracs, budget_gb: float, region: int, local_rank: int) -> dict:
    """Capacity and latency of the serving loop, host buffers end to end:
    all requests submitted at once (capacity), then a Poisson stream at each
    fraction of that rate; latency runs from a request's arrival to the poll
    that retires it."""
    import torch

    from paper_1703_02563_gb300 import ff, serving, workloads

    prm = workloads.BATCH_PARAMS
    maxw = max(p.width for p in pairs)
    maxh = max(p.height for p in pairs)
    cfg = ff.Config(channels=3, scales=prm["scales"], iters=prm["iters"],
                    radius_q3=prm["radius_q3"], max_width=maxw, max_height=maxh,
                    region_min=region)
    torch.cuda.set_device(local_rank)
    srv = ff.ff_server_create(cfg, local_rank, mem_budget=int(budget_gb * (1 << 30)),
                              max_slots=256)
    slots = ff.ff_server_slots(srv)
    frames = serving.HostPairs(pairs)
    pool = serving.OutputPool(slots + 64, maxw, maxh)
    sampler = ClockSampler(local_rank)
    serving.run(srv, frames, reqs[:2 * slots], None, pool)          # warm-up
    sampler.start()
    n0 = ff.ff_server_launch_count(srv)
    cap = serving.run(srv, frames, reqs, None, pool)
    points = []
    for frac in fracs:
        points.append(dict(serving.run(srv, frames, reqs, frac * cap["pairs_per_s"], pool,
                                       seed=int(frac * 1000)), load=frac))
    launches = ff.ff_server_launch_count(srv) - n0
    clocks = sampler.stop()
    ff.ff_server_destroy(srv)
    return {"slots": slots, "slot_bytes": ff.ff_slot_bytes(cfg), "capacity": cap,
            "latency": points, "clocks": clocks, "gpu_launches": launches,
            "pairs": len(pairs), "requests": len(reqs), "memory_budget_gb": budget_gb,
            "sizes": "256..1920 x 256..1024 (and 1080) in 64-px steps, one per pair",
            "generator": "independent layered pairs (Lab), displacement up to 300 px at "
                         "1920 wide, scaled with the width; each request names a pair and "
                         "carries its own random stream"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", choices=sorted(SCHEDULES), default="basic",
                    help="sweep schedule: basic (Sec. 3.1-3.2), plus (Flow Fields+), fast, "
                         "fast_x2 (Sec. 3.3-3.4)")
    ap.add_argument("--two-way", action="store_true",
                    help="second backward flow and two-way check (Sec. 3.7)")
    ap.add_argument("--region", type=int, default=0,
                    help="region filter s (Sec. 3.7) after the consistency check; 0 = off")
    ap.add_argument("--wht-tc", action="store_true",
                    help="features on the bf16 tensor cores (the precision form)")
    ap.add_argument("--serve", action="store_true",
                    help="run the serving loop on a Poisson request stream instead")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-pairs", type=int, default=128,
                    help="distinct layered pairs the --serve stream draws its requests from")
    ap.add_argument("--serving-leg", type=int, default=480,
                    help="requests of the default line's serving leg (0 = skip it)")
    ap.add_argument("--serve-budget-gb", type=float, default=48.0)
    ap.add_argument("--serve-fracs", type=float, nargs="*", default=[0.5, 0.8, 0.95])
    ap.add_argument("--batch-slots", type=int, default=64,
                    help="matching slots of the batched legs (0 = skip them)")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--autotune", action="store_true",
                    help="choose each batched leg's slots and sweep lane layout by timing "
                         "(autotune.py; the choice is cached)")
    ap.add_argument("--seed-path", choices=["tc", "mma"], default="tc",
                    help="seeding full pass on tcgen05 (default) or mma.sync")
    ap.add_argument("--sweep-lanes", type=int, default=0,
                    help="sweep lanes per grid point (2, 4; 0 = library default)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        from paper_1703_02563_gb300 import workloads
        pair, prm = workloads.make_workload(args.workload)
        sched = SCHEDULES[args.schedule]
        # every step (warm-up included) times one bounded sample of the pair,
        # the same sample cpu_baseline takes
        for _ in range(args.warmup):
            cpu_oracle_rate(pair, prm, sched, args.two_way, args.region)
        rates, walls = [], []
        sample = None
        t_all = time.perf_counter()
        for _ in range(max(1, args.steps)):
            r = cpu_oracle_rate(pair, prm, sched, args.two_way, args.region)
            rates.append(r["pairs_per_s"])
            walls.append(r["wall_s"])
            sample = r["sample"]
        wall = time.perf_counter() - t_all
        v = statistics.median(rates)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s",
                "n_gpus": args.gpus, "steps": len(rates), "warmup": args.warmup,
                "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int8", "data": "synthetic",
                "config": {"workload": args.workload, "frame": f"{pair.width}x{pair.height}",
                           "channels": prm["channels"], "scales": prm["scales"],
                           "iters": prm["iters"], "radius_q3": prm["radius_q3"],
                           "schedule": args.schedule,
                           "backward_flows": 2 if args.two_way else 1},
                "timing": {"samples_timed": len(rates), "sample_wall_s": statistics.mean(walls),
                           "timed_wall_s": wall,
                           "note": "each step is one bounded sample (wall time sample_wall_s); "
                                   "ms_per_step is the time of a whole pair that the sample "
                                   "extrapolates to (the seeding search scaled from its rows)"},
                "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.serve:
        if rank != 0:
            return
        from paper_1703_02563_gb300 import workloads
        pairs = workloads.serving_pairs(args.serve_pairs, workers=min(16, os.cpu_count() or 1))
        reqs = workloads.serving_pair_requests(args.serve_requests, len(pairs))
        res = run_serving(pairs, reqs, args.serve_fracs, args.serve_budget_gb, args.region,
                          local_rank)
        cap = res["capacity"]
        print(json.dumps({
            "metric": METRIC, "value": cap["pairs_per_s"], "unit": "pairs/s", "n_gpus": 1,
            "steps": cap["requests"], "warmup": 2 * res["slots"],
            "ms_per_step": 1e3 / cap["pairs_per_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": "serving: Poisson stream over independent layered pairs, "
                                   "256x256..1920x1080 in 64-px steps (flow up to 300 px)",
                       "channels": 3, "scales": 4, "iters": 6, "radius_q3": 8,
                       "region_min": args.region, "slots": res["slots"],
                       "slot_bytes": res["slot_bytes"], "pairs": res["pairs"],
                       "memory_budget_gb": args.serve_budget_gb,
                       "io": "host buffers: frames in, forward flow and mask out"},
            "clocks": res["clocks"], "gpu_launches": res["gpu_launches"],
            "e2e": {"value": cap["pairs_per_s"], "unit": "pairs/s",
                    "note": "the serving loop is end to end (host buffers)"},
            "serving": {"capacity": cap, "latency": res["latency"]}}))
        return

    batches = {}
    if args.batch_slots and args.schedule == "basic" and not args.two_way and world == 1:
        # generated before CUDA starts, in a spawn pool
        from paper_1703_02563_gb300 import workloads
        workers = min(16, os.cpu_count() or 1)
        batches["sintel1024x436_x32"] = (workloads.make_batch(
            32, seed=2, sizes=((1024, 436),), workers=workers, layered_only=True),
            workloads.BATCH_PARAMS)
        batches["mixed64"] = (workloads.make_batch(64, seed=4, workers=workers),
                              workloads.BATCH_PARAMS)
    serve_pairs = None
    if args.serving_leg and args.schedule == "basic" and not args.two_way and world == 1:
        from paper_1703_02563_gb300 import workloads
        serve_pairs = workloads.serving_pairs(48, workers=min(16, os.cpu_count() or 1))
    if world > 1:
        import torch
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.distributed.init_process_group("nccl")
    res = run_gpu(args, rank, world, local_rank)
    peak_tops = res["peaks"]["sad_dims_per_s"] * OPS_PER_DIM / 1e12
    batched = {name: run_batched(pairs, prm, args.batch_slots, args.batch_steps, 3, local_rank,
                                 args.sweep_lanes, args.autotune, peak_tops)
               for name, (pairs, prm) in batches.items()}
    precision = None
    if args.schedule == "basic" and not args.two_way and world == 1:
        from paper_1703_02563_gb300 import workloads
        kpair, kprm = workloads.make_workload("kitti1242x375")
        precision = dict(precision_form(kpair, kprm["scales"], local_rank),
                         workload="kitti1242x375")
    serving_leg = None
    if serve_pairs:
        from paper_1703_02563_gb300 import workloads
        reqs = workloads.serving_pair_requests(args.serving_leg, len(serve_pairs))
        serving_leg = run_serving(serve_pairs, reqs, [0.8], args.serve_budget_gb, 0, local_rank)
    total_s, e2e_s = replica_times([res["total_ms"] / 1e3, res["e2e_s"]], world, "cuda")
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    K = args.steps
    pairs = K * world
    value = replica_throughput(K, world, total_s)
    W, H, C, S, I = res["W"], res["H"], res["C"], res["S"], res["I"]
    n_dirs = 3 if args.two_way else 2
    evals_pair = n_dirs * eval_count(W, H, res["cfg"])
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": res["total_ms"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "evals_per_s": evals_pair * pairs / total_s,
        "config": {"workload": args.workload, "frame": f"{W}x{H}", "channels": C, "scales": S,
                   "iters": I, "radius_q3": res["prm"]["radius_q3"], "seed_leaf": 8,
                   "schedule": args.schedule, "seed_stride": res["cfg"].seed_stride,
                   "backward_flows": n_dirs - 1, "region_min": args.region,
                   "wht": "bf16 tensor cores, FP32 accumulation" if args.wht_tc else "int32 ALU",
                   "l2": "flushed between steps (256 MiB write outside the step events)",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "clocks": res["clocks"],
        "gpu_launches": res["launches"],
        "e2e": {"value": replica_throughput(K, world, e2e_s), "unit": "pairs/s",
                "h2d_bytes_per_step": res["e2e_bytes"][0],
                "d2h_bytes_per_step": res["e2e_bytes"][1]},
        "roofline": roofline(res, K, n_dirs),
        "peaks_measured": {k: (round(v, 3) if isinstance(v, float) else v)
                           for k, v in res["peaks"].items()},
        "kernels_ms": {k: round(v[1], 4) for k, v in res["kstats"].items() if v[0]},
        "accuracy": res["accuracy"],
    }
    if batched:
        line["batched"] = batched
    if precision:
        line["precision"] = precision
    if serving_leg:
        line["serving"] = {k: serving_leg[k] for k in (
            "capacity", "latency", "slots", "slot_bytes", "pairs", "requests",
            "memory_budget_gb", "sizes", "generator", "gpu_launches", "clocks")}
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    if not args.no_cpu_baseline and world == 1:
        r = cpu_oracle_rate(res["pair"], res["prm"], SCHEDULES[args.schedule], args.two_way,
                            args.region)
        line["cpu_baseline"] = {"value": r["pairs_per_s"], "unit": "pairs/s",
                                "cores": r["cores"], "kind": "oracle", "sample": r["sample"],
                                "wall_s": round(r["wall_s"], 2)}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
