"""bench.py's replica logic on two CPU ranks (gloo): the timings are the
maxima over the ranks and the throughput counts every rank's pairs.  The
method does not shard within a pair, so ranks exchange nothing but these
timings."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out_dir: str):
    import json
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    # rank r took (r + 1) s for its timed steps and 10 (r + 1) s end to end
    times = bench.replica_times([rank + 1.0, 10.0 * (rank + 1)], world, "cpu")
    ids = [bench.replica_pair_id(rank, k) for k in range(5)]
    gathered = [None] * world
    dist.all_gather_object(gathered, ids)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"times": times, "ids": gathered,
                   "value": bench.replica_throughput(20, world, times[0])}, f)


def test_two_replicas_report_the_slowest_rank_and_all_pairs(tmp_path):
    import json
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        res = json.load(open(tmp_path / f"rank{r}.json"))
        assert res["times"] == [2.0, 20.0]           # the maximum over the ranks
        assert res["value"] == 20 * 2 / 2.0          # both ranks' pairs / slowest time
        ids = res["ids"]
        assert len(set(ids[0]) | set(ids[1])) == 10  # no pair id used by two ranks


def test_one_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.replica_times([1.5, 3.0], 1, "cpu") == [1.5, 3.0]
    assert bench.replica_throughput(20, 1, 2.0) == 10.0
