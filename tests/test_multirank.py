"""The N>1 host path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank runs its own copy of the workload (independent units, no collective
on the data path); the job's time is the slowest rank's and the throughput
counts every rank's units.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank           # rank 1 is the slower one
        total = bench.max_over_ranks(local_ms, world, "cpu")
        value = bench.job_throughput(1000, world, total)
        seeds = bench.rank_seed(rank)
        dist.barrier()
        out[rank] = (total, value, seeds["philox_seed"], seeds["instances_seed_offset"])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_units():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    assert res[0][1] == pytest.approx(2 * 1000 / 0.150)
    # distinct seeds and instances per rank
    assert res[0][2] != res[1][2] and res[0][3] != res[1][3]


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_throughput(10, 1, 1000.0) == 10.0
