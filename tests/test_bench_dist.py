"""The replica path of bench.py on CPU: two gloo ranks on 127.0.0.1 (no GPU). Each rank times its
own replica; the job's time is the slowest rank's and its throughput counts every rank's work."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (world, rank, rank)
        ms = [2.0 + rank, 10.0 - rank]                 # rank 1 is slower on the first value
        got = bench.max_over_ranks(dist, ms, torch.device("cpu"))
        out[rank] = got + [bench.whole_job_gbps(world, 1e9, got[0])]
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_the_work():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        assert out[r][:2] == [3.0, 10.0]
        assert out[r][2] == pytest.approx(world * 1e9 / 3e-3 / 1e9)


def test_single_process_passes_values_through():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(None, [1.5, 2], torch.device("cpu")) == [1.5, 2.0]
    assert bench.whole_job_gbps(1, 2e9, 1.0) == pytest.approx(2000.0)
