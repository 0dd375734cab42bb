"""Open-loop load generator for the serving loop (``ff_server_*``).

Requests arrive as a Poisson stream at a given rate; each is submitted at
its arrival time (or, if all host output buffers are taken, as soon as one
is free), and its latency runs from the arrival time to the poll that sees
it retired with its results on the host.  All matching runs in the
library's kernels; this module only schedules submissions and records times.
"""
from __future__ import annotations

import time

import numpy as np

from . import ff


class HostFrames:
    """Pinned copies of the base pairs, addressed by crop."""

    def __init__(self, bases):
        import torch
        self.frames = [(torch.from_numpy(np.ascontiguousarray(b.img1)).pin_memory(),
                        torch.from_numpy(np.ascontiguousarray(b.img2)).pin_memory()) for b in bases]

    def pixels(self, r: dict) -> int:
        return r["w"] * r["h"]

    def request(self, r: dict, two_way: bool, out: dict | None) -> ff.ff_host_pair:
        i1, i2 = self.frames[r["base"]]
        C, H, W = i1.shape
        off = r["y0"] * W + r["x0"]
        out = out or {}
        return ff.ff_host_pair(i1.data_ptr() + off, i2.data_ptr() + off, r["w"], r["h"], W, H * W,
                               r["pair_id"], int(two_way), ff._ptr(out.get("fwd")),
                               ff._ptr(out.get("bwd")), ff._ptr(out.get("bwd2")),
                               ff._ptr(out.get("mask")))


class HostPairs:
    """Pinned copies of independent pairs; a request names one of them."""

    def __init__(self, pairs):
        import torch
        self.frames = [(torch.from_numpy(np.ascontiguousarray(p.img1)).pin_memory(),
                        torch.from_numpy(np.ascontiguousarray(p.img2)).pin_memory()) for p in pairs]

    def request(self, r: dict, two_way: bool, out: dict | None) -> ff.ff_host_pair:
        i1, i2 = self.frames[r["pair"]]
        C, H, W = i1.shape
        out = out or {}
        return ff.ff_host_pair(i1.data_ptr(), i2.data_ptr(), W, H, W, H * W, r["pair_id"],
                               int(two_way), ff._ptr(out.get("fwd")), ff._ptr(out.get("bwd")),
                               ff._ptr(out.get("bwd2")), ff._ptr(out.get("mask")))

    def pixels(self, r: dict) -> int:
        _, H, W = self.frames[r["pair"]][0].shape
        return W * H


class OutputPool:
    """Pinned host buffers for the forward flow and the mask of in-flight
    requests, each large enough for the largest frame."""

    def __init__(self, n: int, max_w: int, max_h: int):
        import torch
        self.free = [dict(fwd=torch.empty(max_h * max_w * 2, dtype=torch.int16).pin_memory(),
                          mask=torch.empty(max_h * max_w, dtype=torch.uint8).pin_memory())
                     for _ in range(n)]


def run(srv: int, frames: HostFrames, reqs: list[dict], rate: float | None, pool: OutputPool,
        two_way: bool = False, seed: int = 0, timeout_s: float = 600.0) -> dict:
    """Serves `reqs`; rate None submits them all at once (capacity)."""
    n = len(reqs)
    rng = np.random.default_rng(seed)
    if rate is None:
        arrival = np.zeros(n)
    else:
        arrival = np.cumsum(rng.exponential(1.0 / rate, n))
    lat = np.full(n, np.nan)
    ticket_of, busy = {}, {}
    nxt, done, failures = 0, 0, 0
    t0 = time.perf_counter()
    first_done = last_done = None
    while done < n:
        now = time.perf_counter() - t0
        if now > timeout_s:
            raise TimeoutError(f"serving {n} requests took over {timeout_s} s")
        while nxt < n and arrival[nxt] <= now and pool.free:
            out = pool.free.pop()
            t = ff.ff_server_submit(srv, frames.request(reqs[nxt], two_way, out))
            ticket_of[t] = nxt
            busy[t] = out
            nxt += 1
        for t, st in ff.ff_server_poll(srv):
            now = time.perf_counter() - t0
            k = ticket_of.pop(t)
            lat[k] = now - arrival[k]
            pool.free.append(busy.pop(t))
            failures += st != ff.FF_OK
            done += 1
            first_done = now if first_done is None else first_done
            last_done = now
    span = last_done - (arrival[0] if rate is not None else 0.0)
    pixels = sum(frames.pixels(r) for r in reqs)
    return {"requests": n, "rate_per_s": rate, "pairs_per_s": n / span,
            "mpix_per_s": pixels / span / 1e6,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_ms": float(np.max(lat) * 1e3), "failures": failures}
