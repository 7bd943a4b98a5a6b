"""FP64 oracle of the learned edge prior (test infrastructure only).

The edge prior is not part of the paper; it scores the candidate edges of the
ACS candidate lists (Alg. 2) with a small MLP and is checked here in FP64:

    features  8 per candidate edge (i, k), j = nn[i][k]
    forward   h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), z = h2 w3 + b3,
              p = sigmoid(z)
    loss      mean binary cross-entropy against soft labels y in [0, 1]
    backward  the analytic gradients of that loss
    adam      one Adam step (Kingma & Ba, 2015) with bias correction

Only tests/, smoke() and the CPU legs of bench.py use this module.
"""
import numpy as np

CL = 32
N_FEAT = 8
HIDDEN = 64


def _dist(xy, i, j):
    d = xy[i].astype(np.float64) - xy[j].astype(np.float64)
    return np.floor(np.sqrt((d * d).sum(-1)) + 0.5)


def features(xy, nn):
    """Features [n, cl, 8] of every candidate edge, in FP64.

    (1) rank / cl; (2) d_ij / mean candidate distance of i; (3) d_ij / d_i,last;
    (4) (x_j - x_i) / d_i,last; (5) (y_j - y_i) / d_i,last; (6) rank of i in
    j's list / cl, or 1 when absent; (7) d_ij / d_j,last; (8) in-degree of j in
    the candidate graph / cl. d_i,last is the distance to i's last candidate
    (at least 1), the mean distance is also taken at least 1.
    """
    xy = np.asarray(xy, np.int64)
    nn = np.asarray(nn, np.int64)
    n, cl = nn.shape
    ii = np.repeat(np.arange(n), cl).reshape(n, cl)
    d = _dist(xy, ii, nn)                                  # [n, cl]
    dmean = np.maximum(d.mean(1), 1.0)
    dlast = np.maximum(d[:, cl - 1], 1.0)
    indeg = np.bincount(nn.reshape(-1), minlength=n).astype(np.float64)
    f = np.zeros((n, cl, N_FEAT))
    f[:, :, 0] = np.arange(cl)[None, :] / cl
    f[:, :, 1] = d / dmean[:, None]
    f[:, :, 2] = d / dlast[:, None]
    f[:, :, 3] = (xy[nn, 0] - xy[ii, 0]) / dlast[:, None]
    f[:, :, 4] = (xy[nn, 1] - xy[ii, 1]) / dlast[:, None]
    rev = np.ones((n, cl))
    for i in range(n):
        for k in range(cl):
            hit = np.where(nn[nn[i, k]] == i)[0]
            if len(hit):
                rev[i, k] = hit[0] / cl
    f[:, :, 5] = rev
    f[:, :, 6] = d / dlast[nn]
    f[:, :, 7] = indeg[nn] / cl
    return f


def init_params(seed=0):
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases, as a dict of FP64 arrays."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.uniform(-1, 1, (N_FEAT, HIDDEN)) / np.sqrt(N_FEAT),
        "b1": np.zeros(HIDDEN),
        "W2": rng.uniform(-1, 1, (HIDDEN, HIDDEN)) / np.sqrt(HIDDEN),
        "b2": np.zeros(HIDDEN),
        "w3": rng.uniform(-1, 1, HIDDEN) / np.sqrt(HIDDEN),
        "b3": np.zeros(1),
    }


def forward(P, x):
    """x [E, 8] -> dict with h1, h2, z, p (FP64)."""
    a1 = x @ P["W1"] + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"] + P["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ P["w3"] + P["b3"][0]
    p = 1.0 / (1.0 + np.exp(-z))
    return {"a1": a1, "h1": h1, "a2": a2, "h2": h2, "z": z, "p": p}


def bce(z, y):
    """Mean binary cross-entropy with logits z against labels y."""
    return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def backward(P, x, y):
    """Loss and gradients of the mean BCE (dict keyed like the parameters)."""
    f = forward(P, x)
    E = x.shape[0]
    dz = (f["p"] - y) / E                          # [E]
    g = {"w3": f["h2"].T @ dz, "b3": np.array([dz.sum()])}
    dh2 = np.outer(dz, P["w3"]) * (f["a2"] > 0)
    g["W2"] = f["h1"].T @ dh2
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ P["W2"].T) * (f["a1"] > 0)
    g["W1"] = x.T @ dh1
    g["b1"] = dh1.sum(0)
    return bce(f["z"], y), g


def adam(P, g, state, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place; state holds the moments m, v per parameter."""
    for k in P:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[:] = b1 * m + (1 - b1) * g[k]
        v[:] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** step)
        vh = v / (1 - b2 ** step)
        P[k] -= lr * mh / (np.sqrt(vh) + eps)


def select_prior(nn, w, p, keep):
    """Prune each candidate row to its `keep` highest scores (ties -> lower
    rank) and reweight them: w' = w * p in FP32. Returns (nn', w') [n, keep]
    in the original rank order of the kept candidates."""
    nn = np.asarray(nn)
    w = np.asarray(w, np.float32)
    p = np.asarray(p, np.float32)
    n, cl = nn.shape
    keep = min(keep, cl)
    out_nn = np.zeros((n, keep), np.int32)
    out_w = np.zeros((n, keep), np.float32)
    for i in range(n):
        order = sorted(range(cl), key=lambda k: (-float(p[i, k]), k))[:keep]
        order.sort()
        out_nn[i] = nn[i, order]
        out_w[i] = (w[i, order] * p[i, order]).astype(np.float32)
    return out_nn, out_w
