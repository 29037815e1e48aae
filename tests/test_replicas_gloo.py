"""Multi-GPU runs are replicas (one full frame per rank, no data-path collective): the job's time is the
slowest rank's and its throughput counts every rank's points. The rank logic of bench.py is exercised here
with two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [3.0, 5.5][rank]                      # per-rank frame times
    slowest = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.job_rate(100_000_000, world, slowest)
    dist.barrier()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{slowest} {rate}")
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        slowest, rate = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert slowest == 5.5
        assert rate == pytest.approx(2 * 100_000_000 / 5.5e-3)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(4.25) == 4.25
    assert bench.job_rate(10, 1, 2.0) == pytest.approx(5000.0)
