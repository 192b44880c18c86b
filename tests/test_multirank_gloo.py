"""Multi-GPU host logic on CPU: two gloo ranks (world size 2) run the bench's rank aggregation.

Each rank runs its own full step (independent problems, weak scaling, no collective on the data
path); the job's time is the slowest rank's, taken by an all-reduce MAX, and the job throughput
counts every rank's flops.  Rendezvous on 127.0.0.1.
"""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ms_per_rank, out_dir):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mx = bench.max_over_ranks(ms_per_rank[rank], dist, "cpu")
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(repr(mx))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp

    ms = [12.5, 17.25]
    mp.start_processes(_rank_main, args=(2, _free_port(), ms, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = [float(open(tmp_path / f"rank{r}.txt").read()) for r in range(2)]
    assert got == [17.25, 17.25]


def test_job_throughput_counts_every_rank():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    one = bench.job_throughput(1, 2.0e12, 50.0)
    assert abs(one - 40.0) < 1e-12
    assert abs(bench.job_throughput(4, 2.0e12, 50.0) - 4 * one) < 1e-12
