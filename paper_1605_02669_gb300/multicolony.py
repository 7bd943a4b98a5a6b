"""Multi-colony ACS with a periodic best-tour exchange (the paper's related
work, Sec. 2): independent colonies on the same instance, one per rank (or
several replicas in one batched context), share their best-so-far tour every
few iterations. The shortest tour (ties -> lowest rank or replica) is offered
to every colony, which keeps it only if strictly shorter than its own
(acs_offer_best_tour), so that its next global update deposits on it.

The exchange is one all-gather of the lengths and one broadcast of the
winning tour; everything else is local. Host logic only: the colonies' work
stays in libacs.
"""
import numpy as np


def exchange_ranks(col, b=0, group=None):
    """One exchange over a torch.distributed process group. `col` offers
    best(b) -> (tour, length) and offer_best(tour, b). Returns the winning
    (rank, length)."""
    import torch
    import torch.distributed as dist

    tour, L = col.best(b)
    world = dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    mine = torch.tensor([L], dtype=torch.int64, device=dev)
    lens = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(lens, mine, group=group)
    vals = [int(x.item()) for x in lens]
    src = min(range(world), key=lambda r: (vals[r], r))
    buf = torch.from_numpy(np.ascontiguousarray(tour, np.int32)).to(dev)
    dist.broadcast(buf, src=src, group=group)
    if dist.get_rank(group) != src:
        col.offer_best(buf.cpu().numpy(), b)
    return src, vals[src]


def exchange_replicas(col, replicas):
    """One exchange among the instances `replicas` of one batched context,
    which hold the same coordinates. Returns the winning (instance, length)."""
    best = [(col.best(b)[1], b) for b in replicas]
    L, win = min(best)
    tour, _ = col.best(win)
    for b in replicas:
        if b != win:
            col.offer_best(tour, b)
    return win, L


def run(col, iters, period, exchange):
    """Run `iters` iterations with an exchange every `period` iterations
    (exchange() is one of the functions above, bound to its arguments)."""
    done = 0
    while done < iters:
        k = min(period, iters - done)
        col.run(k)
        done += k
        exchange()
    return done
