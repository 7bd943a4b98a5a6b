"""Partition of a batch of independent instances across GPUs (one rank each).

Instances of a batch share nothing (each has its own pheromone memory and
random stream, keyed by its instance id), so a batch shards by instance with
no collective on the data path: every rank builds a context of its share with
acs_create_batch_ids and the instances' global ids, and returns its own best
tours. The paper names multiple GPUs as further work (Sec. 5); this is the
instance split for batched runs. A single instance does not shard: its every
step reads the whole pheromone state.

The split is longest-processing-time-first on the work of an iteration,
m*(n-1) ant-steps per instance: instances in decreasing work (ties to the
lower id) each go to the rank with the least work so far (ties to the lower
rank). The heaviest rank then exceeds the lightest by at most one instance's
work.
"""
import numpy as np


def lpt_partition(sizes, m, world):
    """Instance ids of each rank: a list of `world` sorted int lists."""
    sizes = [int(n) for n in sizes]
    if world < 1:
        raise ValueError("world must be >= 1")
    work = [m * (n - 1) for n in sizes]
    order = sorted(range(len(sizes)), key=lambda b: (-work[b], b))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(b)
        load[r] += work[b]
    return [sorted(p) for p in parts]


def shard_of(coords, rank, world, m):
    """This rank's share of a batch given as a list of per-instance coordinate
    arrays: (ids, concatenated coords, offsets)."""
    ids = lpt_partition([c.shape[0] for c in coords], m, world)[rank]
    if not ids:
        return ids, np.zeros((0, 2), np.int32), np.zeros(1, np.int64)
    xy = np.concatenate([coords[b] for b in ids]).astype(np.int32)
    off = np.zeros(len(ids) + 1, np.int64)
    off[1:] = np.cumsum([coords[b].shape[0] for b in ids])
    return ids, xy, off
