"""Pins of the FP64 learned-prior oracle (oracle/mlp.py).

Each expectation comes from outside the oracle's own code: central finite
differences, closed forms of the network in its linear and constant regimes,
the textbook cross-entropy, Adam's first steps in closed form, invariances of
the features under translation and reflection, per-edge brute force on a tiny
instance, and hand-worked pruning tables.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1605_02669_gb300 import instances


def _rand_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    P = mlp.init_params(seed)
    P["b1"] = rng.normal(0, 0.3 * scale, 64)
    P["b2"] = rng.normal(0, 0.3 * scale, 64)
    P["b3"] = rng.normal(0, 0.3 * scale, 1)
    return P


def _flat(g):
    return np.concatenate([np.ravel(g[k]) for k in ("W1", "b1", "W2", "b2", "w3", "b3")])


def test_backward_matches_central_finite_differences():
    rng = np.random.default_rng(3)
    P = _rand_params(4)
    x = rng.normal(0, 1, (16, 8))
    y = rng.uniform(0, 1, 16)
    loss, g = mlp.backward(P, x, y)
    h = 1e-6
    num = {}
    for k in P:
        num[k] = np.zeros_like(P[k])
        it = np.nditer(P[k], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = P[k][idx]
            P[k][idx] = old + h
            lp = mlp.bce(mlp.forward(P, x)["z"], y)
            P[k][idx] = old - h
            lm = mlp.bce(mlp.forward(P, x)["z"], y)
            P[k][idx] = old
            num[k][idx] = (lp - lm) / (2 * h)
    a, n = _flat(g), _flat(num)
    assert np.linalg.norm(a - n) <= 1e-6 * np.linalg.norm(n)
    for k in P:   # every parameter group receives gradient
        assert np.linalg.norm(g[k]) > 0


def test_bce_is_textbook_cross_entropy():
    z = np.array([-3.0, -0.5, 0.0, 0.7, 2.5])
    y = np.array([0.0, 0.25, 1.0, 0.5, 1.0])
    s = 1 / (1 + np.exp(-z))
    ref = -np.mean(y * np.log(s) + (1 - y) * np.log(1 - s))
    assert mlp.bce(z, y) == pytest.approx(ref, rel=1e-13)
    # large logits stay finite (log-sum-exp form)
    assert math.isfinite(mlp.bce(np.array([800.0, -800.0]), np.array([0.0, 1.0])))


def test_constant_network_closed_form():
    # W1 = W2 = 0: h1 = relu(b1), h2 = relu(b2), z = relu(b2).w3 + b3 for every row
    rng = np.random.default_rng(5)
    P = _rand_params(6)
    P["W1"][:] = 0
    P["W2"][:] = 0
    x = rng.normal(0, 1, (10, 8))
    y = rng.uniform(0, 1, 10)
    z0 = np.maximum(P["b2"], 0) @ P["w3"] + P["b3"][0]
    f = mlp.forward(P, x)
    assert np.allclose(f["z"], z0, rtol=0, atol=1e-14)
    assert np.allclose(f["p"], 1 / (1 + math.exp(-z0)), rtol=0, atol=1e-15)
    _, g = mlp.backward(P, x, y)
    mean_dz = np.mean(1 / (1 + math.exp(-z0)) - y)
    assert g["b3"][0] == pytest.approx(mean_dz, rel=1e-12)
    assert np.allclose(g["w3"], np.maximum(P["b2"], 0) * mean_dz, rtol=1e-12, atol=1e-15)
    assert np.allclose(g["b2"], P["w3"] * (P["b2"] > 0) * mean_dz, rtol=1e-12, atol=1e-15)
    # dW2[in][out] = relu(b1)[in] * dh2[out]: an outer product, not its transpose
    assert np.allclose(g["W2"], np.outer(np.maximum(P["b1"], 0), P["w3"] * (P["b2"] > 0) * mean_dz),
                       rtol=1e-12, atol=1e-15)


def test_linear_regime_closed_form():
    # all pre-activations positive: z = x (W1 W2 w3) + (b1 W2 w3 + b2 w3 + b3)
    rng = np.random.default_rng(7)
    P = {
        "W1": rng.uniform(0.1, 1.0, (8, 64)),
        "b1": rng.uniform(0.1, 1.0, 64),
        "W2": rng.uniform(0.1, 1.0, (64, 64)),
        "b2": rng.uniform(0.1, 1.0, 64),
        "w3": rng.uniform(-0.1, 0.1, 64),
        "b3": np.array([0.05]),
    }
    x = rng.uniform(0.0, 1.0, (12, 8))
    y = rng.uniform(0, 1, 12)
    u = P["W2"] @ P["w3"]                 # effective weight of h1
    v = P["W1"] @ u                       # effective weight of x
    c = P["b1"] @ u + P["b2"] @ P["w3"] + P["b3"][0]
    f = mlp.forward(P, x)
    assert np.allclose(f["z"], x @ v + c, rtol=1e-12, atol=1e-12)
    _, g = mlp.backward(P, x, y)
    dz = (1 / (1 + np.exp(-(x @ v + c))) - y) / len(y)
    assert np.allclose(g["W1"], np.outer(x.T @ dz, u), rtol=1e-10, atol=1e-14)
    assert np.allclose(g["b1"], u * dz.sum(), rtol=1e-10, atol=1e-14)
    h1 = x @ P["W1"] + P["b1"]
    assert np.allclose(g["W2"], np.outer(h1.T @ dz, P["w3"]), rtol=1e-10, atol=1e-14)


def test_adam_first_steps_closed_form():
    P = {"a": np.array([1.0, -2.0, 0.5]), "b": np.array([[3.0]])}
    g = {"a": np.array([0.3, -4.0, 1e-3]), "b": np.array([[-2.0]])}
    st = {}
    mlp.adam(P, g, st, step=1, lr=0.01, eps=1e-8)
    # bias-corrected first step: mhat = g, vhat = g^2 -> lr * g / (|g| + eps)
    for k, p0 in (("a", np.array([1.0, -2.0, 0.5])), ("b", np.array([[3.0]]))):
        assert np.allclose(P[k], p0 - 0.01 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-14)
    # a constant gradient keeps mhat = g and vhat = g^2 on every later step
    before = P["a"].copy()
    mlp.adam(P, g, st, step=2, lr=0.01, eps=1e-8)
    assert np.allclose(P["a"], before - 0.01 * g["a"] / (np.abs(g["a"]) + 1e-8), rtol=1e-12)


def test_features_brute_force_tiny(oracle_mod):
    xy = instances.uniform(14, side=200, seed=9)
    cl = 5
    nn = oracle.knn(xy, cl)
    f = mlp.features(xy, nn)
    n = xy.shape[0]

    def d(a, b):
        return math.floor(math.hypot(int(xy[a][0]) - int(xy[b][0]), int(xy[a][1]) - int(xy[b][1])) + 0.5)

    for i in range(n):
        row = [d(i, int(nn[i][k])) for k in range(cl)]
        dl_i = max(row[-1], 1)
        mean_i = max(sum(row) / cl, 1)
        for k in range(cl):
            j = int(nn[i][k])
            dl_j = max(d(j, int(nn[j][cl - 1])), 1)
            back = [q for q in range(cl) if int(nn[j][q]) == i]
            indeg = sum(1 for a in range(n) for q in range(cl) if int(nn[a][q]) == j)
            want = [k / cl, row[k] / mean_i, row[k] / dl_i,
                    (int(xy[j][0]) - int(xy[i][0])) / dl_i, (int(xy[j][1]) - int(xy[i][1])) / dl_i,
                    back[0] / cl if back else 1.0, row[k] / dl_j, indeg / cl]
            assert np.allclose(f[i, k], want, rtol=1e-14, atol=0), (i, k)


def test_features_invariances(oracle_mod):
    xy = instances.clustered(300, seed=4)
    nn = oracle.knn(xy, 32)
    f = mlp.features(xy, nn)
    n = xy.shape[0]
    # translation leaves every feature unchanged
    assert np.array_equal(mlp.features(xy + np.array([123, 45]), nn), f)
    # reflection x -> -x flips the sign of (4) only
    r = xy.copy()
    r[:, 0] = -r[:, 0]
    fr = mlp.features(r, nn)
    assert np.array_equal(fr[:, :, 3], -f[:, :, 3])
    keep = [0, 1, 2, 4, 5, 6, 7]
    assert np.array_equal(fr[:, :, keep], f[:, :, keep])
    # (1) = k/cl; (3) = 1 at the last rank; (2) averages to 1 over a row
    assert np.array_equal(f[:, :, 0], np.tile(np.arange(32) / 32, (n, 1)))
    assert np.all(f[:, 31, 2] == 1.0)
    assert np.allclose(f[:, :, 1].mean(1), 1.0, rtol=1e-12)
    # in-degrees sum to n*cl over nodes; (6) < 1 exactly on mutual candidate pairs
    indeg = np.bincount(nn.reshape(-1), minlength=n)
    assert indeg.sum() == n * 32
    assert np.array_equal(f[:, :, 7], indeg[nn] / 32)
    mutual = np.array([[i in set(nn[nn[i, k]]) for k in range(32)] for i in range(n)])
    assert np.array_equal(f[:, :, 5] < 1.0, mutual)


def test_select_prior_hand_table():
    nn = np.array([[4, 7, 1, 9, 2], [3, 0, 6, 8, 5]], np.int32)
    w = np.array([[1.0, 0.5, 0.25, 2.0, 4.0], [1.0, 1.0, 1.0, 1.0, 1.0]], np.float32)
    p = np.array([[0.2, 0.9, 0.2, 0.7, 0.1],
                  [0.5, 0.5, 0.5, 0.5, 0.5]], np.float32)
    onn, ow = mlp.select_prior(nn, w, p, 3)
    # row 0: best 0.9 (rank 1), 0.7 (rank 3), then the tie 0.2 goes to rank 0
    assert onn[0].tolist() == [4, 7, 9]
    assert ow[0].tolist() == [np.float32(1.0) * np.float32(0.2), np.float32(0.5) * np.float32(0.9),
                              np.float32(2.0) * np.float32(0.7)]
    # row 1: all tied -> the first three ranks
    assert onn[1].tolist() == [3, 0, 6]
    # keep = cl: same lists, w * p
    onn, ow = mlp.select_prior(nn, w, p, 5)
    assert np.array_equal(onn, nn) and np.array_equal(ow, w * p)
