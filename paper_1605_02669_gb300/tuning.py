"""Cache of autotuned launch shapes, keyed by workload shape (host logic only).

acs_autotune times every (threads per ant, cluster size[, SPM record
placement]) that can launch and keeps the fastest. Its choice depends on the
shape of the batch, not on the coordinates, so it is cached in a JSON file
keyed by: memory, number of instances, ants, SPM slots, and the instance
sizes bucketed by powers of two. A cached shape is applied directly; a miss
runs the autotuner and stores its choice.
"""
import json
import os

from . import acs


def shape_key(sizes, p):
    """Key of a batch: memory, instances, m, s and the sorted size buckets."""
    buckets = sorted({max(1, int(n)).bit_length() for n in sizes})
    return "mem%d-B%d-m%d-s%d-n%s" % (p.memory, len(sizes), p.m,
                                      p.spm_slots if p.memory == acs.ACS_MEM_SPM else 0,
                                      ".".join(str(b) for b in buckets))


def load_cache(path):
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path, cache):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(col, path, trial_iters=2):
    """Apply the cached launch shape of `col`'s batch, or autotune and cache it.
    Returns (entry, hit)."""
    cache = load_cache(path)
    key = shape_key(col.sizes, col.p)
    ent = cache.get(key)
    if ent is not None:
        try:
            if col.p.memory == acs.ACS_MEM_SPM:
                col.set_spm_resident(ent["resident"])
            col.set_cluster_size(ent["cluster_size"])
            col.set_threads_per_ant(ent["threads_per_ant"])
            return ent, True
        except (acs.AcsError, KeyError, TypeError):
            pass   # stale or foreign entry: tune again
    tpa, cs = col.autotune(trial_iters)
    ent = {"threads_per_ant": tpa, "cluster_size": cs,
           "resident": 1 if col.kernel_mode != 1 else 0}
    cache[key] = ent
    save_cache(path, cache)
    return ent, False
