"""The serving loop: requests admitted as slots free up, overlapping on the
device; every result equals the same pair matched alone (and the oracle)."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle as O
from paper_1703_02563_gb300 import ff, serving, workloads

pytestmark = pytest.mark.gpu


def _crop(img, r):
    return np.ascontiguousarray(img[:, r["y0"]:r["y0"] + r["h"], r["x0"]:r["x0"] + r["w"]])


def test_server_results_same_alone_and_in_the_mix():
    import torch
    bases = [workloads.layered_pair(seed=40 + k, width=220, height=170, channels=3, max_disp=25)
             for k in range(2)]
    reqs = workloads.serving_requests(9, 2, seed=3, widths=(64, 100, 150, 200),
                                      heights=(48, 90, 160), base_w=220, base_h=170)
    two_way = [k % 3 == 2 for k in range(len(reqs))]
    cfg = ff.Config(channels=3, scales=3, iters=4, max_width=200, max_height=160, region_min=30)
    srv = ff.ff_server_create(cfg, 0, mem_budget=3 * ff.ff_slot_bytes(cfg), max_slots=8)
    assert ff.ff_server_slots(srv) == 3
    frames = serving.HostFrames(bases)
    outs = [dict(fwd=torch.full((r["h"], r["w"], 2), 5, dtype=torch.int16).pin_memory(),
                 bwd=torch.full((r["h"], r["w"], 2), 5, dtype=torch.int16).pin_memory(),
                 bwd2=torch.full((r["h"], r["w"], 2), 5, dtype=torch.int16).pin_memory(),
                 mask=torch.full((r["h"], r["w"]), 5, dtype=torch.uint8).pin_memory())
            for r in reqs]
    tickets = [ff.ff_server_submit(srv, frames.request(r, tw, o))
               for r, tw, o in zip(reqs, two_way, outs)]
    assert tickets == list(range(len(reqs)))
    assert ff.ff_server_pending(srv) == len(reqs)
    retired = {}
    while len(retired) < len(reqs):
        for t, st in ff.ff_server_poll(srv):
            assert t not in retired
            retired[t] = st
    assert all(st == ff.FF_OK for st in retired.values())
    assert ff.ff_server_pending(srv) == 0
    # alone: one context, one pair at a time, device calls
    ctx = ff.Context(cfg)
    for k, (r, tw, o) in enumerate(zip(reqs, two_way, outs)):
        a, b = _crop(bases[r["base"]].img1, r), _crop(bases[r["base"]].img2, r)
        ctx.features(0, torch.from_numpy(a).cuda())
        ctx.features(1, torch.from_numpy(b).cuda())
        f, _ = ctx.match(ff.FF_FWD, r["pair_id"], with_cost=False)
        bw, _ = ctx.match(ff.FF_BWD, r["pair_id"], with_cost=False)
        if tw:
            b2, _ = ctx.match(ff.FF_BWD2, r["pair_id"], with_cost=False)
            m = ctx.filter_2way(f, bw, b2)
            assert torch.equal(o["bwd2"], b2.cpu()), f"request {k}"
        else:
            m = ctx.filter(f, bw)
        m = ctx.region_filter(f, m, 30)
        assert torch.equal(o["fwd"], f.cpu()), f"request {k}"
        assert torch.equal(o["bwd"], bw.cpu()), f"request {k}"
        assert torch.equal(o["mask"], m.cpu()), f"request {k}"
    ctx.close()
    # and the oracle, for two of them
    P = O.Params(channels=3, scales=3, iters=4)
    for k in (0, 2):
        r = reqs[k]
        a, b = _crop(bases[r["base"]].img1, r), _crop(bases[r["base"]].img2, r)
        rf, _, _ = O.match(P, a, b, 0, r["pair_id"])
        np.testing.assert_array_equal(outs[k]["fwd"].numpy(), rf)
    ff.ff_server_destroy(srv)


def test_open_loop_run_retires_every_request():
    base = [workloads.layered_pair(seed=50, width=256, height=192, channels=3, max_disp=30)]
    reqs = workloads.serving_requests(24, 1, seed=4, widths=(64, 128, 192, 256),
                                      heights=(64, 128, 192), base_w=256, base_h=192)
    cfg = ff.Config(channels=3, scales=3, iters=4, max_width=256, max_height=192)
    srv = ff.ff_server_create(cfg, 0, mem_budget=4 * ff.ff_slot_bytes(cfg), max_slots=4)
    pool = serving.OutputPool(6, 256, 192)
    res = serving.run(srv, serving.HostFrames(base), reqs, 2000.0, pool, timeout_s=120)
    assert res["requests"] == 24 and res["failures"] == 0
    assert res["p99_ms"] >= res["p50_ms"] > 0
    assert len(pool.free) == 6
    ff.ff_server_destroy(srv)


def test_independent_pairs_served_equal_the_pairs_alone():
    # the benchmark's stream: independent pairs of their own sizes, each
    # request naming one pair with its own random stream
    import torch
    pairs = workloads.serving_pairs(4, seed=12, widths=(64, 128, 192), heights=(64, 96, 128))
    reqs = workloads.serving_pair_requests(10, len(pairs), seed=2)
    maxw = max(p.width for p in pairs)
    maxh = max(p.height for p in pairs)
    cfg = ff.Config(channels=3, scales=3, iters=4, max_width=maxw, max_height=maxh)
    srv = ff.ff_server_create(cfg, 0, mem_budget=3 * ff.ff_slot_bytes(cfg), max_slots=3)
    frames = serving.HostPairs(pairs)
    pool = serving.OutputPool(len(reqs), maxw, maxh)
    outs = list(pool.free)
    res = serving.run(srv, frames, reqs, None, pool, timeout_s=120)
    assert res["requests"] == len(reqs) and res["failures"] == 0
    assert res["mpix_per_s"] > 0
    ff.ff_server_destroy(srv)
    # every buffer came back; which buffer served which request is the pool's
    # business, so check each request alone against the oracle instead
    P = O.Params(channels=3, scales=3, iters=4)
    srv = ff.ff_server_create(cfg, 0, mem_budget=3 * ff.ff_slot_bytes(cfg), max_slots=3)
    for r in reqs[:4]:
        p = pairs[r["pair"]]
        out = dict(fwd=torch.full((p.height * p.width * 2,), 3, dtype=torch.int16).pin_memory(),
                   mask=torch.full((p.height * p.width,), 3, dtype=torch.uint8).pin_memory())
        t = ff.ff_server_submit(srv, frames.request(r, False, out))
        done = []
        t0 = time.perf_counter()
        while not done and time.perf_counter() - t0 < 60:
            done = ff.ff_server_poll(srv)
        assert done == [(t, ff.FF_OK)]
        rf, _, _ = O.match(P, p.img1, p.img2, 0, r["pair_id"])
        np.testing.assert_array_equal(out["fwd"].numpy().reshape(rf.shape), rf)
    ff.ff_server_destroy(srv)
    assert len(outs) == len(reqs)


def test_slot_bytes_match_what_a_context_allocates():
    # admission by device memory is only as good as this estimate
    import torch
    cfg = ff.Config(channels=3, scales=4, iters=6, max_width=1024, max_height=436)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ctx = ff.ff_create(cfg, 0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    est = ff.ff_slot_bytes(cfg)
    ff.ff_destroy(ctx)
    assert abs(used - est) <= 0.05 * est + (8 << 20), (used, est)
