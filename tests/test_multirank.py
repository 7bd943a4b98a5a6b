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


def _shard_worker(rank, world, port, out):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        for wl in ("batch256", "large16"):
            bench.select_workload(wl)
            ids, xy, off, sizes, seed, job_sizes, scaling = bench.rank_share(rank, world)
            # every rank learns every share over the process group (host only)
            shares = [None] * world
            dist.all_gather_object(shares, list(ids))
            res[wl] = (shares, sizes, job_sizes, scaling, seed, int(off[-1]), xy.shape[0])
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_batched_workloads_shard_by_instance_over_gloo_ranks(world):
    import bench

    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for wl in ("batch256", "large16"):
        bench.select_workload(wl)
        all_sizes = list(bench.SIZES)
        work = [bench.M * (n - 1) for n in all_sizes]
        shares = res[0][wl][0]
        for r in range(world):
            assert res[r][wl][0] == shares          # every rank agrees on the split
            _, sizes, job_sizes, scaling, seed, nodes, rows = res[r][wl]
            assert scaling == "strong" and job_sizes == all_sizes and seed == 1
            assert sizes == [all_sizes[b] for b in shares[r]]
            assert nodes == rows == sum(sizes)
        flat = sorted(b for sh in shares for b in sh)
        assert flat == list(range(len(all_sizes)))  # each instance exactly once
        loads = [sum(work[b] for b in sh) for sh in shares]
        assert max(loads) - min(loads) <= max(work)  # LPT: within one instance


def test_lpt_partition_small_cases():
    from paper_1605_02669_gb300 import shard

    assert shard.lpt_partition([10, 10, 10], 1, 1) == [[0, 1, 2]]
    # decreasing work, ties to the lower id and the lower rank
    # work 8, 16, 16, 4: 1 -> r0, 2 -> r1, 0 -> r0 (tie), 3 -> r1
    assert shard.lpt_partition([5, 9, 9, 3], 2, 2) == [[0, 1], [2, 3]]
    assert shard.lpt_partition([4], 1, 3) == [[0], [], []]
    with pytest.raises(ValueError):
        shard.lpt_partition([4], 1, 0)
