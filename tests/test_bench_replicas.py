"""Replica timing of bench.py on the CPU: two gloo ranks, no GPU.

The benchmark runs one independent replica of the workload per GPU (the path has no exchange
step); the whole-job value divides all ranks' states by the slowest rank's time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        ms_all = bench.max_over_ranks(ms)
        out[rank] = (ms_all, bench.replica_value(3.0e9, ms_all, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms_all, value = res[0]
    assert ms_all == 150.0
    assert abs(value - 2 * 3.0e9 / 0.150 / 1e9) < 1e-9


def test_single_process_is_its_own_maximum():
    import bench

    assert bench.max_over_ranks(12.5) == 12.5
    assert abs(bench.replica_value(1e9, 1000.0, 1) - 1.0) < 1e-12
