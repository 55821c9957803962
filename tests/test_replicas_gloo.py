"""The N > 1 path of bench.py on CPU: two replica processes over gloo.

bench.py runs one replica per GPU with no data collective; the process group only
brackets the timed region with barriers and takes the slowest rank's time.  These
checks run the same helpers (dist_setup, barrier, max_over_ranks, aggregate_rate) in
two spawned processes on the host."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_setup(None, backend="gloo")
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    # each replica times its own steps; the job is as slow as its slowest rank
    my_ms = 100.0 * (rank + 1)
    slowest = bench.max_over_ranks(my_ms, w)
    rate = bench.aggregate_rate(w, 5, slowest)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "rate": rate}, f)


def test_two_replicas_take_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for g in got:
        assert g["slowest"] == pytest.approx(200.0)
        # 2 replicas x 5 steps in 0.2 s of the slowest rank
        assert g["rate"] == pytest.approx(50.0)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    os.environ.pop("WORLD_SIZE", None)
    assert bench.dist_setup(None) == (1, 0, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_rate(1, 4, 2000.0) == pytest.approx(2.0)
