"""Host logic of bench.py with several ranks (one replica of the workload per
GPU): the job's step time is the slowest rank's, and the job's throughput
counts every rank's queries.  Two gloo ranks on the CPU."""
import os
import socket

import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.slowest_rank_ms(2.0 + 3.0 * rank, device="cpu")   # rank 1 is slower
        out[rank] = (ms, bench.job_value(1000, world, ms))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_job_value_over_two_gloo_ranks():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        ms, value = out[rank]
        assert ms == 5.0
        assert abs(value - 2 * 1000 / 5e-3) < 1e-6


def test_single_rank_keeps_its_own_time():
    assert bench.slowest_rank_ms(3.5, device="cpu") == 3.5
    assert bench.job_value(10, 1, 2.0) == 10 / 2e-3
