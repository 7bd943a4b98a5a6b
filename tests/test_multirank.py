"""The N>1 host path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank runs its own copy of the workload (independent units, no collective
on the data path); the job's time is the slowest rank's and the throughput
counts every rank's units.
"""
import os
import socket

import numpy as np
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


class _FakeColony:
    """Stands in for a colony on the CPU: a best tour and the offer rule."""

    def __init__(self, tour, length):
        self.tour, self.length = np.asarray(tour, np.int32), length
        self.offered = []

    def best(self, b=0):
        return self.tour.copy(), self.length

    def offer_best(self, tour, b=0):
        self.offered.append(np.asarray(tour).copy())
        # the rule of acs_offer_best_tour: lengths are faked by tour[0] here
        L = 100 + int(tour[0])
        if L < self.length:
            self.tour, self.length = np.asarray(tour, np.int32), L


def _exchange_worker(rank, world, port, out):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_1605_02669_gb300 import multicolony

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r holds the tour [r, ...] of length 100 + r, except rank 2 the shortest
        lengths = {0: 105, 1: 101, 2: 100}
        first = {0: 5, 1: 1, 2: 0}
        tour = [first[rank]] + [i for i in range(6) if i != first[rank]]
        col = _FakeColony(tour, lengths[rank])
        src, L = multicolony.exchange_ranks(col)
        out[rank] = (src, L, col.length, [t.tolist() for t in col.offered])
    finally:
        dist.destroy_process_group()


def test_exchange_over_three_gloo_ranks_offers_the_shortest_tour():
    import numpy as np  # noqa: F401

    world = 3
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_exchange_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        src, L, mine, offered = res[r]
        assert src == 2 and L == 100 and mine == 100
        if r == 2:
            assert offered == []          # the winner keeps its own
        else:
            assert offered == [[0, 1, 2, 3, 4, 5]]
