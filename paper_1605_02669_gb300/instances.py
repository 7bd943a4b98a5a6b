"""Seeded synthetic TSP instances (integer coordinates).

This module only draws coordinates; it holds none of the colony's arithmetic,
so both the CUDA path and the CPU oracle can be fed from it.

The paper measures on TSPLIB instances (d198, pr1002, pr2392, ...; Sec. 4)
that are not available here; these generators stand in for them:
    uniform    integer points uniform in [0, side]^2
    clustered  Gaussian clusters (centres uniform in [0, side]^2, sigma per
               axis), rounded to integers, points outside the square rejected
Duplicate points are rejected in both, so every distance between distinct
nodes is at least 1.
"""
import numpy as np

COORD_LIMIT = 1 << 20  # the library accepts coordinates in [0, 2^20)


def _rng(seed, stream=0):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


def _dedupe_fill(rng, n, draw):
    pts = np.empty((0, 2), np.int64)
    seen = set()
    while pts.shape[0] < n:
        cand = draw(rng, 2 * (n - pts.shape[0]) + 16)
        keep = []
        for x, y in cand:
            key = (int(x), int(y))
            if key in seen:
                continue
            seen.add(key)
            keep.append(key)
            if pts.shape[0] + len(keep) == n:
                break
        if keep:
            pts = np.concatenate([pts, np.asarray(keep, np.int64)])
    return pts.astype(np.int32)


def uniform(n, side=10000, seed=1, stream=0):
    """n distinct integer points uniform in [0, side]^2."""
    if side + 1 > COORD_LIMIT:
        raise ValueError("side too large")
    if (side + 1) ** 2 < n:
        raise ValueError("not enough distinct points")
    rng = _rng(seed, stream)
    return _dedupe_fill(rng, n, lambda r, k: r.integers(0, side + 1, size=(k, 2)))


def clustered(n, clusters=20, sigma=300.0, side=10000, seed=1, stream=0):
    """n distinct integer points from Gaussian clusters in [0, side]^2."""
    rng = _rng(seed, stream)
    centres = rng.uniform(0.0, side, size=(clusters, 2))

    def draw(r, k):
        c = centres[r.integers(0, clusters, size=k)]
        p = np.rint(c + r.normal(0.0, sigma, size=(k, 2))).astype(np.int64)
        ok = (p >= 0).all(axis=1) & (p <= side).all(axis=1)
        return p[ok]

    return _dedupe_fill(rng, n, draw)


def batch(sizes, kinds, side=10000, seed=1):
    """Concatenated coordinates and offsets for a batch of instances.

    sizes: list of n_b; kinds: list of 'uniform' / 'clustered'.
    Returns (xy int32 [sum n, 2], offsets int64 [B+1]).
    """
    parts = []
    for b, (n, kind) in enumerate(zip(sizes, kinds)):
        if kind == "uniform":
            parts.append(uniform(n, side=side, seed=seed, stream=1000 + b))
        else:
            parts.append(clustered(n, side=side, seed=seed, stream=1000 + b))
    offsets = np.zeros(len(sizes) + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    return np.concatenate(parts).astype(np.int32), offsets


def mixed_batch(B, n_lo, n_hi, side=10000, seed=1):
    """B instances with n uniform in [n_lo, n_hi]; even b uniform, odd b clustered."""
    rng = _rng(seed, 7)
    sizes = [int(x) for x in rng.integers(n_lo, n_hi + 1, size=B)]
    kinds = ["uniform" if b % 2 == 0 else "clustered" for b in range(B)]
    xy, off = batch(sizes, kinds, side=side, seed=seed)
    return xy, off, sizes, kinds
