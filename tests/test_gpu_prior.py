"""Learned-prior kernels against the FP64 oracle (oracle/mlp.py) and the ACS oracle.

Features, scores and gradients are BF16/FP32 on the GPU and FP64 here: the
bounds are the ones the arithmetic allows (one BF16 rounding of each feature;
2e-2 absolute on scores; 2e-2 relative on gradient norms). Pruned tables and
the ACS runs on them are integer/FP32 decisions and compare bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1605_02669_gb300 import acs, instances

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _prior():
    from paper_1605_02669_gb300 import prior

    return prior


def _bf16_bits(x):
    """Round to BF16 (nearest-even) as input preparation; returns uint16 bits."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def _bits_to_f64(b):
    return (np.asarray(b, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _params64(seed):
    """Oracle parameters, rounded to FP32 (what the device vector holds)."""
    rng = np.random.default_rng(seed + 100)
    P = mlp.init_params(seed)
    P["b1"] = rng.normal(0, 0.2, 64)
    P["b2"] = rng.normal(0, 0.2, 64)
    P["b3"] = rng.normal(-1.0, 0.2, 1)
    return {k: np.asarray(v, np.float32).astype(np.float64) for k, v in P.items()}


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


def _edge_rows(xy, cl=32):
    nn = oracle.knn(xy, min(cl, xy.shape[0] - 1))
    return mlp.features(xy, nn).reshape(-1, 8)


def _assert_same(gpu, ref, memory, b=0):
    tg, lg = gpu.tours(b)
    tr, lr = ref.tours()
    assert np.array_equal(tg, tr) and np.array_equal(lg, lr)
    assert gpu.best(b)[1] == ref.best()[1]
    if memory == 0:
        assert np.array_equal(gpu.pheromone(b).view(np.uint32), ref.pheromone().view(np.uint32))
    else:
        gv, gi, gt = gpu.pheromone(b)
        rv, ri, rt = ref.pheromone()
        assert np.array_equal(gi, ri) and np.array_equal(gt, rt)
        assert np.array_equal(gv.view(np.uint32), rv.view(np.uint32))


# ------------------------------------------------------------------ features
@pytest.mark.parametrize("kind,n", [("uniform", 300), ("clustered", 1002), ("uniform", 20),
                                    ("clustered", 4)])
def test_features_match_fp64(oracle_mod, kind, n):
    prior = _prior()
    xy = instances.uniform(n, seed=21) if kind == "uniform" else instances.clustered(n, seed=21)
    col = acs.Colony(xy, acs.params(m=4, cl=32, seed=1))
    g = prior.bf16_to_float(prior.colony_features(col)).reshape(n, 32, 8).astype(np.float64)
    cl = min(32, n - 1)
    ref = mlp.features(xy, oracle.knn(xy, cl))
    assert np.all(g[:, cl:, :] == 0)
    # one BF16 rounding of an FP32 value that is within a few ulps of the FP64 one
    err = np.abs(g[:, :cl] - ref)
    assert np.all(err <= 2.0 ** -8 * np.abs(ref)), float(err.max())
    col.close()


# ------------------------------------------------------------------ forward
@pytest.mark.parametrize("rows", [0, 1, 17, 1007, 32064])
def test_forward_matches_fp64(oracle_mod, rows):
    prior = _prior()
    x = _edge_rows(instances.clustered(1002, seed=3))[:rows]
    bits = _bf16_bits(x)
    P = _params64(5)
    feat = _dev(bits.view(np.int16).reshape(rows, 8))
    params = _dev(prior.pack(P))
    p = prior.score(params, feat).cpu().numpy()
    if rows == 0:
        assert p.shape == (0,)
        return
    ref = mlp.forward(P, _bits_to_f64(bits))["p"]
    assert np.max(np.abs(p - ref)) <= 2e-2
    assert np.all((p > 0) & (p < 1))


def _forward_bf16_points(P, bits):
    """The forward with the kernel's rounding points: W1, W2 and h1 rounded to
    BF16 (nearest-even), everything else FP64. Differs from the kernel only by
    FP32 accumulation order and, rarely, a BF16 rounding of h1 that an FP32
    sum puts on the other side of a rounding boundary."""
    def bf(a):
        return _bits_to_f64(_bf16_bits(np.asarray(a, np.float32)))

    x = _bits_to_f64(bits)
    h1 = bf(np.maximum(x @ bf(P["W1"]) + P["b1"], 0.0))
    h2 = np.maximum(h1 @ bf(P["W2"]) + P["b2"], 0.0)
    z = h2 @ P["w3"].reshape(-1) + P["b3"][0]
    return 1.0 / (1.0 + np.exp(-z))


@pytest.mark.parametrize("rows", [128, 129, 32064, 50000, 76544, 120000, 200000])
def test_forward_matches_bf16_rounding_points(oracle_mod, rows):
    """Tight check of the tensor-core layers: every tile row, every hidden
    unit and both K halves of layer 2 must land in the right place, so a
    transposed operand or a misplaced core matrix fails by far more than
    the bound. Sizes span one full tile, a ragged second tile, CTAs of
    2, 3, 4 and 7 tile groups, and more tiles than the persistent grid
    has groups."""
    prior = _prior()
    base = _edge_rows(instances.clustered(1002, seed=3))
    x = np.tile(base, (rows // base.shape[0] + 1, 1))[:rows]
    x = x * np.random.default_rng(rows).uniform(0.5, 1.5, x.shape)
    bits = _bf16_bits(x)
    P = _params64(7)
    p = prior.score(_dev(prior.pack(P)), _dev(bits.view(np.int16).reshape(rows, 8))).cpu().numpy()
    err = np.abs(p.astype(np.float64) - _forward_bf16_points(P, bits))
    assert np.quantile(err, 0.99) <= 1e-5, float(np.quantile(err, 0.99))
    assert err.max() <= 5e-3, float(err.max())


def test_forward_zero_weights_is_sigmoid_of_bias():
    prior = _prior()
    v = np.zeros(acs.ACS_MLP_PARAMS, np.float32)
    v[4800] = 0.75
    feat = _dev(_bf16_bits(np.random.default_rng(1).normal(0, 1, (100, 8))).view(np.int16))
    p = prior.score(_dev(v), feat).cpu().numpy()
    assert np.all(p == np.float32(1 / (1 + math.exp(-0.75))))


# ------------------------------------------------------------------ backward
def _labels(rows, seed):
    # mostly zeros like the best-tour frequencies (about 2 of 32 candidates)
    rng = np.random.default_rng(seed)
    y = (rng.uniform(size=rows) < 0.08).astype(np.float32)
    y[rng.uniform(size=rows) < 0.05] = 0.5
    return y


def _check_grad(g_gpu, g_ref, loss_gpu, loss_ref):
    prior = _prior()
    G = prior.unpack(g_gpu)
    for k in g_ref:
        num = np.linalg.norm(G[k] - g_ref[k])
        den = np.linalg.norm(g_ref[k])
        assert num <= 2e-2 * den, (k, num / den)
    assert abs(loss_gpu - loss_ref) <= 2e-2 * loss_ref


@pytest.mark.parametrize("rows", [16, 1000, 4096])
def test_train_batch_gradient_matches_fp64(oracle_mod, rows):
    prior = _prior()
    x = _edge_rows(instances.clustered(700, seed=6))[:rows]
    bits = _bf16_bits(x)
    y = _labels(rows, 2)
    P = _params64(8)
    grad = torch.full((acs.ACS_MLP_PARAMS,), 7.0, device="cuda")   # overwritten
    loss = torch.full((1,), 7.0, device="cuda")
    acs.acs_mlp_train_batch(_dev(prior.pack(P)), _dev(bits.view(np.int16)), _dev(y), rows, 0,
                            rows, 1, 0, grad, loss, torch.cuda.current_stream())
    ref_loss, ref_g = mlp.backward(P, _bits_to_f64(bits), y.astype(np.float64))
    _check_grad(grad.cpu().numpy(), ref_g, float(loss.item()), ref_loss)


def test_train_batch_gradient_many_tiles_per_cta(oracle_mod):
    # the grid is at most one CTA per SM, so beyond 128 x SMs rows every CTA
    # walks several tiles and accumulates their weight gradients in TMEM (the
    # accumulate flag after the first tile, operand tiles reused): this size
    # gives every CTA two or three tiles and a ragged last tile
    prior = _prior()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rows = 50001
    assert rows > 2 * 128 * sms
    x = _edge_rows(instances.clustered(1600, seed=16))[:rows]
    bits = _bf16_bits(x)
    y = _labels(rows, 12)
    P = _params64(18)
    grad = torch.full((acs.ACS_MLP_PARAMS,), 7.0, device="cuda")
    loss = torch.full((1,), 7.0, device="cuda")
    acs.acs_mlp_train_batch(_dev(prior.pack(P)), _dev(bits.view(np.int16)), _dev(y), rows, 0,
                            rows, 1, 0, grad, loss, torch.cuda.current_stream())
    ref_loss, ref_g = mlp.backward(P, _bits_to_f64(bits), y.astype(np.float64))
    _check_grad(grad.cpu().numpy(), ref_g, float(loss.item()), ref_loss)


_TIMEOUT_CHILD = r"""
import json, sys
sys.path.insert(0, ROOT)
import numpy as np, torch
from paper_1605_02669_gb300 import acs, instances
L = acs.load()
s = torch.cuda.current_stream()
params = (torch.randn(acs.ACS_MLP_PARAMS, device="cuda") * 0.2).float()
rows = 5000
feat = torch.randn(rows, 8, device="cuda").to(torch.bfloat16).view(torch.int16)
out = []
if KIND == "forward":
    p = torch.empty(rows, device="cuda")
    acs.acs_mlp_forward(params, feat, rows, p, s)
    out.append(L.acs_mlp_sync(None))                  # a normal launch: 0
    ok_scores = bool(torch.isfinite(p).all())
    col = acs.Colony(instances.uniform(200, seed=1), acs.params(m=8, cl=32))
    out.append(L.acs_mlp_test_wait_hook(1000000, 1))  # 1 ms, phantom barrier
    p2 = torch.zeros(rows, device="cuda")
    acs.acs_mlp_forward(params, feat, rows, p2, s)    # the launch itself succeeds
    torch.cuda.synchronize()
    nan_rows = bool(torch.isnan(p2).all())
    sc = torch.full((200 * 32,), 0.5, device="cuda")
    out.append(L.acs_apply_prior(col.ctx, 0, acs._dev(sc), 16, None))   # ETIMEOUT, poisons ctx
    out.append(L.acs_run_iterations(col.ctx, 1))                        # ESTATE
    out.append(L.acs_mlp_sync(None))                                     # ESTATE
    out.append(L.acs_mlp_forward(acs._dev(params), acs._dev(feat), rows, acs._dev(p2), None))
    print("RESULT " + json.dumps({"codes": out, "first_ok": ok_scores, "nan": nan_rows}))
else:
    y = torch.zeros(rows, device="cuda")
    grad = torch.zeros(acs.ACS_MLP_PARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    out.append(L.acs_mlp_test_wait_hook(1000000, 1))
    acs.acs_mlp_train_batch(params, feat, y, rows, 0, rows, 1, 0, grad, loss, s)
    torch.cuda.synchronize()
    nan_loss = bool(torch.isnan(loss).all())
    out.append(L.acs_mlp_sync(None))                                     # ETIMEOUT
    out.append(L.acs_mlp_train_batch(acs._dev(params), acs._dev(feat), acs._dev(y), rows, 0, rows,
                                     1, 0, acs._dev(grad), acs._dev(loss), None))   # ESTATE
    out.append(L.acs_mlp_adam(acs._dev(params), acs._dev(grad), acs._dev(grad), acs._dev(grad),
                              1, 1e-3, 0.9, 0.999, 1e-8, None))                    # ESTATE
    print("RESULT " + json.dumps({"codes": out, "first_ok": True, "nan": nan_loss}))
"""


@pytest.mark.parametrize("kind", ["forward", "train"])
def test_tensor_core_wait_give_up_reports_etimeout(kind):
    # the bounded mbarrier wait of the tcgen05 kernels is driven to its limit by
    # the test hook (a second barrier that nothing arrives on; the real MMA
    # still completes and is drained before tensor memory is freed). The give-up
    # must reach the caller as ACS_ETIMEOUT and close the tensor-core path.
    # A child process: the closed path would otherwise stay closed for the
    # tests that follow.
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = "ROOT = %r\nKIND = %r\n" % (root, kind) + _TIMEOUT_CHILD
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    import json

    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    codes, ok_first, nan_out = res["codes"], res["first_ok"], res["nan"]
    E = acs
    if kind == "forward":
        assert codes == [E.ACS_OK, E.ACS_OK, E.ACS_ETIMEOUT, E.ACS_ESTATE, E.ACS_ESTATE, E.ACS_ESTATE]
        assert ok_first and nan_out
    else:
        assert codes == [E.ACS_OK, E.ACS_ETIMEOUT, E.ACS_ESTATE, E.ACS_ESTATE]
        assert nan_out


def test_train_batch_reads_the_affine_permutation(oracle_mod):
    prior = _prior()
    x = _edge_rows(instances.uniform(300, seed=7))     # 9600 rows
    total = x.shape[0]
    bits = _bf16_bits(x)
    y = _labels(total, 3)
    P = _params64(9)
    a, c, first, batch = 7, 123, 1000, 600
    assert math.gcd(a, total) == 1
    grad = torch.zeros(acs.ACS_MLP_PARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    acs.acs_mlp_train_batch(_dev(prior.pack(P)), _dev(bits.view(np.int16)), _dev(y), total, first,
                            batch, a, c, grad, loss, torch.cuda.current_stream())
    idx = (a * (first + np.arange(batch)) + c) % total
    ref_loss, ref_g = mlp.backward(P, _bits_to_f64(bits[idx]), y[idx].astype(np.float64))
    _check_grad(grad.cpu().numpy(), ref_g, float(loss.item()), ref_loss)


def test_adam_matches_fp64():
    rng = np.random.default_rng(4)
    n = acs.ACS_MLP_PARAMS
    p = rng.normal(0, 0.5, n).astype(np.float32)
    g = rng.normal(0, 1e-2, n).astype(np.float32)
    m = rng.normal(0, 1e-2, n).astype(np.float32)
    v = rng.uniform(0, 1e-4, n).astype(np.float32)
    dp, dg, dm, dv = _dev(p), _dev(g), _dev(m), _dev(v)
    acs.acs_mlp_adam(dp, dg, dm, dv, 3, 2e-3, 0.9, 0.999, 1e-8, torch.cuda.current_stream())
    # the oracle takes the hyper-parameters the kernel receives (FP32 values)
    f32 = lambda x: float(np.float32(x))
    P = {"x": p.astype(np.float64)}
    st = {"m_x": m.astype(np.float64), "v_x": v.astype(np.float64)}
    mlp.adam(P, {"x": g.astype(np.float64)}, st, 3, lr=f32(2e-3), b1=f32(0.9), b2=f32(0.999),
             eps=f32(1e-8))
    # FP32 rounding of each term of the moment updates (a few ulps of the terms)
    eps32 = 2.0 ** -23
    bm = 4 * eps32 * (0.9 * np.abs(m) + 0.1 * np.abs(g))
    bv = 4 * eps32 * (0.999 * v + 0.001 * g * g.astype(np.float64))
    assert np.all(np.abs(dm.cpu().numpy() - st["m_x"]) <= bm)
    assert np.all(np.abs(dv.cpu().numpy() - st["v_x"]) <= bv)
    assert np.allclose(dp.cpu().numpy(), P["x"], rtol=2.0 ** -22, atol=1e-8)


# ------------------------------------------------------------------ labels
def test_count_best_edges_against_oracle_tour(oracle_mod):
    xy = instances.clustered(400, seed=12)
    col = acs.Colony(xy, acs.params(m=16, cl=32, seed=2))
    count = torch.zeros(400 * 32, device="cuda")
    with pytest.raises(acs.AcsError):     # no best-so-far tour before an iteration
        acs.acs_prior_count_best_edges(col.ctx, 0, count, torch.cuda.current_stream())
    ref = oracle.Colony(xy, oracle.make_params(m=16, cl=32, seed=2))
    col.run(4)
    ref.run(4)
    for _ in range(2):
        acs.acs_prior_count_best_edges(col.ctx, 0, count, torch.cuda.current_stream())
    tour, _ = ref.best()
    edges = {frozenset((int(tour[i]), int(tour[(i + 1) % 400]))) for i in range(400)}
    want = np.zeros((400, 32), np.float32)
    for i in range(400):
        for k in range(32):
            want[i, k] = 2.0 if frozenset((i, int(ref.nn[i][k]))) in edges else 0.0
    assert np.array_equal(count.cpu().numpy().reshape(400, 32), want)
    col.close()


# ------------------------------------------------------------------ pruned tables + ACS
def _scores(n, seed):
    # quantised to 1/64 so that ties (-> lower rank) are common
    rng = np.random.default_rng(seed)
    return (np.floor(rng.uniform(1, 64, (n, 32))) / 64).astype(np.float32)


@pytest.mark.parametrize("memory", [0, 1])
def test_apply_prior_tables_and_run_bit_exact(oracle_mod, memory):
    n = 700
    xy = instances.clustered(n, seed=8)
    p = _scores(n, 1)
    col = acs.Colony(xy, acs.params(m=32, cl=32, memory=memory, spm_slots=8, seed=5))
    acs.acs_apply_prior(col.ctx, 0, _dev(p.reshape(-1)), 16, torch.cuda.current_stream())
    nn_g, w_g, tau0, _ = col.setup(0)
    assert nn_g.shape == (n, 16)
    plain = oracle.Colony(xy, oracle.make_params(m=32, cl=32, memory=memory, spm_slots=8, seed=5))
    onn, ow = mlp.select_prior(plain.nn, plain.w, p, 16)
    assert np.array_equal(nn_g, onn)
    assert np.array_equal(w_g.view(np.uint32), ow.view(np.uint32))
    ref = oracle.Colony(xy, oracle.make_params(m=32, cl=32, memory=memory, spm_slots=8, seed=5),
                        nn=onn, w=ow)
    assert tau0 == ref.tau0
    col.run(3)
    ref.run(3)
    _assert_same(col, ref, memory)
    col.close()


def test_apply_prior_on_one_instance_of_a_batch(oracle_mod):
    xy, off = instances.batch([150, 400, 260], ["uniform", "clustered", "uniform"], seed=4)
    p = _scores(400, 2)
    col = acs.Colony(xy, acs.params(m=24, cl=32, seed=9), offsets=off)
    acs.acs_apply_prior(col.ctx, 1, _dev(p.reshape(-1)), 12, torch.cuda.current_stream())
    col.run(3)
    for b in range(3):
        sub = xy[off[b]:off[b + 1]]
        prm = oracle.make_params(m=24, cl=32, seed=9)
        if b == 1:
            plain = oracle.Colony(sub, prm, instance=b)
            onn, ow = mlp.select_prior(plain.nn, plain.w, p, 12)
            ref = oracle.Colony(sub, prm, instance=b, nn=onn, w=ow)
        else:
            ref = oracle.Colony(sub, prm, instance=b)
        ref.run(3)
        _assert_same(col, ref, 0, b)
    col.close()


def test_set_candidates_runs_like_oracle_tables(oracle_mod):
    n = 250
    xy = instances.uniform(n, seed=30)
    plain = oracle.Colony(xy, oracle.make_params(m=16, cl=32, seed=3))
    rng = np.random.default_rng(5)
    nn = plain.nn[:, :24].copy()
    w = (plain.w[:, :24] * rng.uniform(0.5, 1.5, (n, 24))).astype(np.float32)
    col = acs.Colony(xy, acs.params(m=16, cl=32, seed=3))
    acs.acs_set_candidates(col.ctx, 0, nn, w)
    ref = oracle.Colony(xy, oracle.make_params(m=16, cl=32, seed=3), nn=nn, w=w)
    col.run(3)
    ref.run(3)
    _assert_same(col, ref, 0)
    # invalid tables are rejected and leave the context usable
    bad = nn.copy()
    bad[3, 2] = 3
    for t_nn, t_w in ((bad, w), (np.full_like(nn, n), w), (nn, -w)):
        with pytest.raises(acs.AcsError) as e:
            acs.acs_set_candidates(col.ctx, 0, t_nn, t_w)
        assert e.value.status == acs.ACS_EINVAL
    col.run(1)
    ref.run(1)
    _assert_same(col, ref, 0)
    col.close()


def test_apply_prior_rejects_bad_keep():
    xy = instances.uniform(60, seed=2)
    col = acs.Colony(xy, acs.params(m=4, cl=32, seed=1))
    p = _dev(np.full(60 * 32, 0.5, np.float32))
    for keep in (0, 33):
        with pytest.raises(acs.AcsError) as e:
            acs.acs_apply_prior(col.ctx, 0, p, keep, torch.cuda.current_stream())
        assert e.value.status == acs.ACS_EINVAL
    col.close()


# ------------------------------------------------------------------ training
def test_training_reduces_loss_and_ranks_tour_edges():
    prior = _prior()
    xy, off, _, _ = instances.mixed_batch(24, 100, 220, seed=5)
    label = prior.edge_labels(xy, off, runs=2, iters=30, m=16, seed=3, tune=False)
    col = acs.Colony(xy, acs.params(m=1, cl=32, memory=1, seed=1), offsets=off)
    feat = prior.batch_features(col)
    col.close()
    tr = prior.Trainer(prior.init_params(1), lr=3e-3)
    rng = np.random.default_rng(0)
    losses = [tr.epoch(feat, label, 512, rng) for _ in range(6)]
    assert losses[-1] < 0.8 * losses[0]
    p = prior.score(tr.params, feat).cpu().numpy()
    y = label.cpu().numpy()
    pos, neg = p[y > 0.5], p[y == 0]      # n >= 33: every row is a real candidate
    # area under the ROC curve of the scores for tour vs non-tour edges
    order = np.argsort(np.concatenate([pos, neg]), kind="stable")
    ranks = np.empty(len(order))
    ranks[order] = np.arange(1, len(order) + 1)
    auc = (ranks[:len(pos)].sum() - len(pos) * (len(pos) + 1) / 2) / (len(pos) * len(neg))
    assert auc > 0.85, auc


def test_trained_prior_gains_at_equal_gpu_time():
    # train on small generated instances, evaluate on held-out larger ones:
    # the prior-pruned colony gets the GPU time the plain colony used
    import time

    prior = _prior()
    xy, off, _, _ = instances.mixed_batch(120, 200, 600, seed=41)
    label = prior.edge_labels(xy, off, runs=2, iters=60, m=32, seed=41, tune=False)
    col = acs.Colony(xy, acs.params(m=1, cl=32, memory=1, seed=1), offsets=off)
    feat = prior.batch_features(col)
    col.close()
    tr = prior.Trainer(prior.init_params(41), lr=2e-3)
    rng = np.random.default_rng(1)
    for _ in range(4):
        tr.epoch(feat, label, 4096, rng)

    def run(xy, use_prior, budget=None, iters=None):
        c = acs.Colony(xy, acs.params(m=64, cl=32, seed=3))
        if use_prior:
            prior.apply(c, tr.params, keep=16)
        c.run(1)
        torch.cuda.synchronize()
        t0, done = time.perf_counter(), 0
        while (iters is not None and done < iters) or (budget is not None and
                                                       time.perf_counter() - t0 < budget):
            c.run(10)
            torch.cuda.synchronize()
            done += 10
        spent = time.perf_counter() - t0
        best = c.best(0)[1]
        c.close()
        return best, spent

    gaps = {"plain": [], "prior": []}
    for xy_e in (instances.clustered(1500, seed=77), instances.uniform(1500, seed=78)):
        Lp, spent = run(xy_e, False, iters=120)
        Lq, _ = run(xy_e, True, budget=spent)
        best = min(Lp, Lq)
        gaps["plain"].append((Lp - best) / best)
        gaps["prior"].append((Lq - best) / best)
    assert np.mean(gaps["prior"]) < np.mean(gaps["plain"]), gaps
