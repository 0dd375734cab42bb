"""Tuning of the batched form: matching-slot count and sweep lane layout.

For a configuration and a sample batch (device inputs and outputs already
allocated), times every candidate (slots, sweep lanes per grid point) through
``ff_batch_run`` graphs with CUDA events and keeps the fastest in a JSON
cache keyed by the device, channel count, scales, schedule and the batch's
largest frame.  Every candidate computes the same results (the lane layout
and the slot count change only how the work is spread over the GPU); the
tuner chooses between them by time alone.
"""
from __future__ import annotations

import json
import os

from . import ff

DEFAULT_CACHE = os.environ.get(
    "FF_TUNE_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json"))


def _key(cfg: ff.Config, device_name: str) -> str:
    return (f"{device_name}|C{cfg.channels}|S{cfg.scales}|I{cfg.iters}|sched{cfg.schedule}|"
            f"{cfg.max_width}x{cfg.max_height}")


def candidates(cfg: ff.Config, max_slots: int) -> list[tuple[int, int]]:
    lanes = (4, 2)
    slots = [s for s in (8, 16, 32, 48, 64) if s <= max_slots]
    return [(s, w) for s in slots for w in lanes]


def lookup(cfg: ff.Config, device: int = 0, path: str = DEFAULT_CACHE) -> dict | None:
    import torch
    try:
        with open(path) as f:
            return json.load(f).get(_key(cfg, torch.cuda.get_device_name(device)))
    except (OSError, ValueError):
        return None


def tune(cfg: ff.Config, descs, n: int, device: int = 0, max_slots: int = 64, steps: int = 2,
         path: str | None = DEFAULT_CACHE) -> dict:
    """Times each candidate on the batch `descs` (n pairs); returns
    {"slots", "lanes", "ms", "trials"} and stores it in the cache at `path`."""
    import torch
    stream = torch.cuda.Stream(device)
    trials = []
    for slots, lanes in candidates(cfg, max_slots):
        b = ff.ff_batch_create(cfg, device, slots=slots, stream=stream)
        try:
            ff.ff_batch_debug_set(b, ff.FF_DEBUG_SWEEP_LANES, lanes)
            ff.ff_batch_run(b, descs, n, use_graph=True)      # capture + first run
            ff.ff_batch_sync(b)
            times = []
            for _ in range(steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ff.ff_batch_run(b, descs, n, use_graph=True)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            ff.ff_batch_sync(b)
        finally:
            ff.ff_batch_destroy(b)
        trials.append({"slots": slots, "lanes": lanes, "ms": min(times)})
    best = min(trials, key=lambda t: t["ms"])
    result = dict(best, trials=trials)
    if path:
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        cache[_key(cfg, torch.cuda.get_device_name(device))] = result
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return result
