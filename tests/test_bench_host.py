"""bench.py's host-side arithmetic (CPU): the evaluation count behind
``evals_per_s`` and the sweep roofline, and the roofline record itself.

The count is a restatement in the benchmark of how many matching-error
evaluations one direction performs; here it must equal the number the oracle
counts while it runs the method, for every schedule and for frames with
ragged coarse levels.
"""
from __future__ import annotations

import os
import sys

import pytest

import oracle as O
from paper_1703_02563_gb300 import ff, workloads

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("schedule", [0, 1, 2, 3])
@pytest.mark.parametrize("W,H,S,iters,leaf,stride", [
    (45, 31, 3, 4, 8, 1),
    (33, 17, 4, 6, 4, 1),
    (40, 26, 3, 5, 8, 2),
])
def test_eval_count_equals_the_oracles_count(schedule, W, H, S, iters, leaf, stride):
    if schedule == 3 and S < 3:
        pytest.skip("Fast x2 needs three scales")
    pair = workloads.random_pair(seed=W * H + schedule, width=W, height=H)
    P = O.Params(scales=S, iters=iters, seed_leaf=leaf, seed_stride=stride, schedule=schedule)
    _, _, counted = O.match(P, pair.img1, pair.img2, 0, 0)
    cfg = ff.Config(channels=1, scales=S, iters=iters, seed_leaf=leaf, seed_stride=stride,
                    schedule=schedule)
    assert bench.eval_count(W, H, cfg) == counted


def test_sweep_roofline_arithmetic():
    # one direction's sweeps on a 64x48 frame, timed as 10 launches of 2 ms
    cfg = ff.Config(channels=3, scales=2, iters=5)
    W, H = 64, 48
    peaks = {"sad_dims_per_s": 5e12, "dp4a_per_s": 2e13, "l2_read_gbs": 2e4,
             "lat_shfl": 20.0, "lat_ldg_l1": 40.0, "lat_prmt": 5.0, "lat_dp4a": 6.0,
             "lat_alu": 4.0}
    res = {"kstats": {"k_sweep": (10, 20.0), "k_features": (2, 0.5)},
           "W": W, "H": H, "C": 3, "S": 2, "I": 5, "cfg": cfg, "workload": "none",
           "peaks": peaks, "clocks": {"sm_mhz": 2000.0}}
    r = bench.roofline(res, steps=1, n_dirs=1)
    evals = bench.sweep_evals(W, H, cfg)
    # by hand: level 0 64x48, level 1 32x24; 5 sweeps (2 candidates per point, one
    # fewer per incoming border point) and 4 random searches per level
    by_hand = sum(5 * (2 * w * h - w - h) + 4 * w * h for w, h in ((64, 48), (32, 24)))
    assert evals == by_hand
    # 27 dimensions, 11 operations each (4 multiply-adds, subtract, abs, add)
    ops_per_launch = evals * 27 * 11 / 10
    assert r["kernel"] == "k_sweep" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(ops_per_launch / 2e-3 / 1e12)
    assert r["peak"] == pytest.approx(5e12 * 11 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["frac_of_dp4a_peak"] == pytest.approx(r["achieved"] / (2e13 * 8 / 1e12))
    assert r["share"] == pytest.approx(20.0 / 20.5)
    assert r["traffic"] is None and r["l2"] is None   # no recorded capture for this workload
    # critical path: 5 sweeps per level of (64 + 48 - 1) and (32 + 24 - 1) anti-diagonals
    diags = 5 * (64 + 48 - 1) + 5 * (32 + 24 - 1)
    cp = r["critical_path"]
    assert cp["cycles_per_step"] == pytest.approx(20.0e-3 * 2000e6 / diags)
    assert cp["floor_cycles"] == pytest.approx(3 * 20 + 40 + 2 * 5 + 6 + 24 * 4)
    assert cp["frac"] == pytest.approx(cp["floor_cycles"] / cp["cycles_per_step"])
    # the live sweep runs of the timed region (10 launches in 18 ms) take over the
    # launch time and the critical path; the share stays the per-launch pass's
    res["sweep_live"] = (10, 18.0)
    r2 = bench.roofline(res, steps=1, n_dirs=1)
    assert r2["avg_launch_ms"] == pytest.approx(1.8)
    assert r2["achieved"] == pytest.approx(ops_per_launch / 1.8e-3 / 1e12)
    assert r2["critical_path"]["cycles_per_step"] == pytest.approx(18.0e-3 * 2000e6 / diags)
    assert r2["share"] == pytest.approx(20.0 / 20.5)
    assert "timed region" in r2["timing"] and "profiled pass" in r["timing"]


def test_code_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    # the recorded ncu counters stay valid across comment edits only
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "a.cuh").write_text('int f(int x) {  // add one\n    return x + 1; /* done */\n}\n'
                                    'const char *s = "// kept";\n')
    h0 = bench.code_hash(["a.cuh"])
    (tmp_path / "a.cuh").write_text('// a new header comment\nint f(int x) {\n  return x + 1;\n}\n'
                                    'const char *s = "// kept";\n')
    assert bench.code_hash(["a.cuh"]) == h0
    (tmp_path / "a.cuh").write_text('int f(int x) {\n  return x + 2;\n}\nconst char *s = "// kept";\n')
    assert bench.code_hash(["a.cuh"]) != h0
    (tmp_path / "a.cuh").write_text('int f(int x) {\n  return x + 1;\n}\nconst char *s = "// gone";\n')
    assert bench.code_hash(["a.cuh"]) != h0
