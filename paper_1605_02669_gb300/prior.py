"""Learned edge prior over the candidate lists (include/acs_prior.h).

Pipeline, every arithmetic step in libacs kernels (torch holds the buffers):
  1. labels   plain ACS (Alg. 1 with Alg. 2) on a batch of generated
              instances, R seeded runs; the label of candidate edge (i, j) is
              the fraction of the R best-so-far tours that contain {i, j}.
  2. features 8 per candidate edge, BF16 [rows][8] (acs_prior_features).
  3. training mean BCE, Adam, mini-batches drawn through an affine
              permutation of the rows (acs_mlp_train_batch / acs_mlp_adam).
  4. scoring  p = MLP(features) and acs_apply_prior: keep the `keep` best
              candidates of every list, w' = w * p; the full-scan fallback of
              Alg. 2 keeps the plain heuristic.

The parameter vector is FP32 [4801]: W1 [8][64], b1, W2 [64][64] (W2[in][out]),
b2, w3, b3 (offsets in LAYOUT).
"""
import math

import numpy as np
import torch

from . import acs, instances

N_PARAMS = acs.ACS_MLP_PARAMS
LAYOUT = {
    "W1": (0, (8, 64)),
    "b1": (512, (64,)),
    "W2": (576, (64, 64)),
    "b2": (4672, (64,)),
    "w3": (4736, (64,)),
    "b3": (4800, (1,)),
}


def pack(P):
    """dict of arrays -> FP32 parameter vector."""
    v = np.zeros(N_PARAMS, np.float32)
    for k, (o, shp) in LAYOUT.items():
        v[o:o + int(np.prod(shp))] = np.asarray(P[k], np.float32).reshape(-1)
    return v


def unpack(v):
    """FP32 parameter vector (numpy or tensor) -> dict of FP64 arrays."""
    if isinstance(v, torch.Tensor):
        v = v.detach().cpu().numpy()
    v = np.asarray(v, np.float64)
    return {k: v[o:o + int(np.prod(shp))].reshape(shp) for k, (o, shp) in LAYOUT.items()}


def init_params(seed=0):
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    return pack({
        "W1": rng.uniform(-1, 1, (8, 64)) / math.sqrt(8),
        "b1": np.zeros(64),
        "W2": rng.uniform(-1, 1, (64, 64)) / 8.0,
        "b2": np.zeros(64),
        "w3": rng.uniform(-1, 1, 64) / 8.0,
        "b3": np.zeros(1),
    })


def bf16_to_float(t):
    """BF16 bit patterns (int16 tensor or uint16 array) -> FP32 numpy."""
    if isinstance(t, torch.Tensor):
        t = t.cpu().numpy()
    u = np.asarray(t).view(np.uint16).astype(np.uint32) << 16
    return u.view(np.float32)


def _stream():
    return torch.cuda.current_stream()


def colony_features(col, b=0, out=None):
    """BF16 features [n*32, 8] (int16 tensor) of instance b of a Colony."""
    n = col.sizes[b]
    if out is None:
        out = torch.empty((n * 32, 8), dtype=torch.int16, device="cuda")
    acs.acs_prior_features(col.ctx, b, out, _stream())
    return out


def batch_features(col):
    """Features of every instance of a batched Colony, concatenated [32*sum(n), 8]."""
    rows = 32 * sum(col.sizes)
    out = torch.empty((rows, 8), dtype=torch.int16, device="cuda")
    r = 0
    for b, n in enumerate(col.sizes):
        colony_features(col, b, out[r:r + 32 * n])
        r += 32 * n
    return out


def edge_labels(xy, off, runs=8, iters=200, m=64, seed=1, tune=True):
    """Fraction of `runs` plain-ACS best-so-far tours (seeds seed..seed+runs-1,
    `iters` iterations each) that contain each candidate edge, [32*sum(n)]."""
    sizes = np.diff(np.asarray(off, np.int64))
    count = torch.zeros(32 * int(sizes.sum()), dtype=torch.float32, device="cuda")
    for r in range(runs):
        col = acs.Colony(xy, acs.params(m=m, cl=32, seed=seed + r), offsets=off)
        if tune:
            col.autotune(1)
        col.run(iters)
        row = 0
        for b, n in enumerate(sizes):
            acs.acs_prior_count_best_edges(col.ctx, b, count[row:row + 32 * int(n)], _stream())
            row += 32 * int(n)
        torch.cuda.synchronize()
        col.close()
    return count / runs


def _coprime(total, rng):
    while True:
        a = int(rng.integers(1, max(total, 2)))
        if math.gcd(a, total) == 1:
            return a


class Trainer:
    """Adam on the device parameter vector with the library's kernels."""

    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.params = torch.as_tensor(np.asarray(params, np.float32)).cuda()
        self.m = torch.zeros(N_PARAMS, dtype=torch.float32, device="cuda")
        self.v = torch.zeros(N_PARAMS, dtype=torch.float32, device="cuda")
        self.grad = torch.zeros(N_PARAMS, dtype=torch.float32, device="cuda")
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.lr, self.beta1, self.beta2, self.eps = lr, beta1, beta2, eps
        self.step = 0

    def batch(self, feat, label, first, batch, perm_a, perm_c):
        """Gradient of one mini-batch and one Adam step; returns the loss tensor."""
        total = feat.shape[0]
        acs.acs_mlp_train_batch(self.params, feat, label, total, first, batch, perm_a, perm_c,
                                self.grad, self.loss, _stream())
        self.step += 1
        acs.acs_mlp_adam(self.params, self.grad, self.m, self.v, self.step, self.lr, self.beta1,
                         self.beta2, self.eps, _stream())
        return self.loss

    def epoch(self, feat, label, batch=4096, rng=None):
        """One pass over all rows in a fresh affine order; returns the mean loss."""
        rng = rng if rng is not None else np.random.default_rng(0)
        total = feat.shape[0]
        a, c = _coprime(total, rng), int(rng.integers(0, total))
        acc = torch.zeros(1, dtype=torch.float32, device="cuda")
        nb = 0
        for first in range(0, total, batch):
            acc += self.batch(feat, label, first, min(batch, total - first), a, c)
            nb += 1
        # raises if a tensor-core wait of this epoch gave up (incomplete gradients)
        acs.acs_mlp_sync(_stream())
        return float(acc.item()) / nb


def score(params, feat):
    """p = MLP(features) for every row, FP32 tensor."""
    p = torch.empty(feat.shape[0], dtype=torch.float32, device="cuda")
    acs.acs_mlp_forward(params, feat, feat.shape[0], p, _stream())
    return p


def apply(col, params, keep=16):
    """Score every instance of a Colony on its plain lists and prune/reweight them."""
    for b in range(len(col.sizes)):
        feat = colony_features(col, b)
        p = score(params, feat)
        acs.acs_apply_prior(col.ctx, b, p, keep, _stream())


def train(n_instances=2000, n_lo=200, n_hi=1000, runs=8, iters=200, m=64, epochs=4,
          batch=4096, lr=1e-3, seed=11, log=None):
    """Generate instances, label them with plain ACS, train the MLP. Returns
    (params tensor, per-epoch losses)."""
    xy, off, _, _ = instances.mixed_batch(n_instances, n_lo, n_hi, seed=seed)
    label = edge_labels(xy, off, runs=runs, iters=iters, m=m, seed=seed)
    # a one-ant SPM context only to hold the candidate lists for the features
    col = acs.Colony(xy, acs.params(m=1, cl=32, memory=acs.ACS_MEM_SPM, seed=seed), offsets=off)
    feat = batch_features(col)
    col.close()
    tr = Trainer(init_params(seed), lr=lr)
    rng = np.random.default_rng(seed)
    losses = []
    for e in range(epochs):
        losses.append(tr.epoch(feat, label, batch, rng))
        if log:
            log("epoch %d loss %.5f" % (e, losses[-1]))
    return tr.params, losses


def main(argv=None):
    """Train the prior on generated instances and save the parameter vector."""
    import argparse
    import time

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--instances", type=int, default=2000)
    ap.add_argument("--n-lo", type=int, default=200)
    ap.add_argument("--n-hi", type=int, default=1000)
    ap.add_argument("--runs", type=int, default=8, help="plain-ACS runs per instance for labels")
    ap.add_argument("--iters", type=int, default=200, help="iterations of each labelling run")
    ap.add_argument("--m", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--out", default="prior_params.npy")
    ap.add_argument("--apply-n", type=int, default=0,
                    help="then score and prune a generated clustered instance of this size "
                         "and run it for a few iterations (0: skip)")
    a = ap.parse_args(argv)
    from . import build

    build.build()
    t0 = time.time()
    params, _ = train(a.instances, a.n_lo, a.n_hi, a.runs, a.iters, a.m, a.epochs, a.batch, a.lr,
                      a.seed, log=print)
    np.save(a.out, params.cpu().numpy())
    print("trained in %.1f s -> %s" % (time.time() - t0, a.out))
    if a.apply_n:
        xy = instances.clustered(a.apply_n, seed=a.seed + 1)
        col = acs.Colony(xy, acs.params(m=128, cl=32, seed=a.seed))
        apply(col, params, keep=16)
        col.run(3)
        print("prior-pruned colony, n=%d: best %d after 3 iterations" % (a.apply_n, col.best(0)[1]))
        col.close()


if __name__ == "__main__":
    main()
