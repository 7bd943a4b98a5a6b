"""Full-shape runs of the batched and the large-scale workloads on the GPU.

Outputs the oracle can reproduce in seconds are compared bit for bit on
sampled instances; the rest is checked through properties that hold at any
size: every tour is a permutation, lengths equal the recomputed EUC_2D sums,
the best-so-far is the minimum seen, and tau0 <= tau <= 1/L_best.
"""
import numpy as np
import pytest

import oracle
from paper_1605_02669_gb300 import acs, instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _lengths(xy, tours):
    p = xy.astype(np.int64)
    a = p[tours]
    b = p[np.roll(tours, -1, axis=1)]
    d2 = ((a - b) ** 2).sum(-1)
    d = np.floor(np.sqrt(d2.astype(np.float64)) + 0.5).astype(np.int64)
    return d.sum(1)


def _check_properties(xy, tours, lens, best, best_len):
    n = xy.shape[0]
    assert (np.sort(tours, axis=1) == np.arange(n)).all()
    assert np.array_equal(_lengths(xy, tours), lens)
    assert best_len <= lens.min()
    assert np.array_equal(np.sort(best), np.arange(n))
    assert _lengths(xy, best[None, :])[0] == best_len


def _assert_same(gpu, ref, memory, b):
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


@pytest.mark.parametrize("memory", [0, 1])
def test_batched_256_instances(oracle_mod, memory):
    # 256 instances, n uniform in [100, 2500], even b uniform / odd b clustered,
    # m=64, 32-NN, one launch per iteration for the whole batch; on the SPM
    # with the records in global memory, the placement the autotuner picks
    # for this batch
    xy, off, sizes, kinds = instances.mixed_batch(256, 100, 2500, seed=3)
    p = acs.params(m=64, cl=32, q0=0.9, memory=memory, spm_slots=8, seed=7)
    gpu = acs.Colony(xy, p, offsets=off)
    if memory == 1:
        gpu.set_spm_resident(0)
    gpu.run(2)
    for b in range(256):
        t, L = gpu.tours(b)
        bt, bl = gpu.best(b)
        _check_properties(xy[off[b]:off[b + 1]], t, L, bt, bl)
    # bit-exact against the oracle on 32 instances: the smallest, the largest
    # and 30 spread over the size order (the oracle colonies run in threads)
    from concurrent.futures import ThreadPoolExecutor

    order = np.argsort(sizes)
    pick = sorted({int(order[i]) for i in np.linspace(0, 255, 32).round().astype(int)})

    def ref_of(b):
        r = oracle.Colony(xy[off[b]:off[b + 1]],
                          oracle.make_params(m=64, cl=32, q0=0.9, memory=memory, spm_slots=8, seed=7),
                          instance=b)
        r.run(2)
        return r

    with ThreadPoolExecutor(16) as ex:
        refs = list(ex.map(ref_of, pick))
    for b, ref in zip(pick, refs):
        _assert_same(gpu, ref, memory, b)


@pytest.mark.parametrize("memory", [0, 1])
def test_large_n10000_m256_one_iteration(oracle_mod, memory):
    xy = instances.uniform(10000, side=100000, seed=5)
    p = acs.params(m=256, cl=32, memory=memory, spm_slots=8, seed=3)
    gpu = acs.Colony(xy, p)
    ref = oracle.Colony(xy, oracle.make_params(m=256, cl=32, memory=memory, spm_slots=8, seed=3))
    gpu.run(1)
    ref.run(1)
    _assert_same(gpu, ref, memory, 0)


def test_large_n20000_batch_properties(oracle_mod):
    # two n=20000 instances on the matrix (1.6 GB each) and on the SPM
    xy0 = instances.uniform(20000, side=100000, seed=6)
    xy1 = instances.uniform(20000, side=100000, seed=7)
    xy = np.concatenate([xy0, xy1])
    off = np.array([0, 20000, 40000], np.int64)
    for memory in (0, 1):
        gpu = acs.Colony(xy, acs.params(m=256, cl=32, memory=memory, spm_slots=8, seed=4),
                         offsets=off)
        gpu.run(2)
        for b in range(2):
            t, L = gpu.tours(b)
            bt, bl = gpu.best(b)
            _check_properties(xy[off[b]:off[b + 1]], t, L, bt, bl)
        if memory == 0:
            tau = gpu.pheromone(0)
            _, bl = gpu.best(0)
            nn, w, tau0, _ = gpu.setup(0)
            np.fill_diagonal(tau, tau0)
            assert tau.min() >= tau0
            assert tau.max() <= np.float32(1.0 / bl) * (1 + 2.0 ** -22)
        gpu.close()


@pytest.mark.parametrize("memory", [0, 1])
def test_maximum_n_65536_properties(memory):
    # the largest instance the library accepts (n = 65536, coordinates up to
    # 2^20 - 1). The oracle's set-up alone takes most of an hour at this size,
    # so the checks are those that hold at any size, plus the candidate lists
    # of sampled nodes against a brute-force sort.
    n = 65536
    xy = instances.uniform(n, side=(1 << 20) - 1, seed=23)
    gpu = acs.Colony(xy, acs.params(m=8, cl=32, memory=memory, spm_slots=8, seed=2))
    gpu.run(2)
    t, L = gpu.tours(0)
    bt, bl = gpu.best(0)
    _check_properties(xy, t, L, bt, bl)
    nn, w, tau0, _ = gpu.setup(0)
    rng = np.random.default_rng(0)
    p = xy.astype(np.int64)
    for i in rng.choice(n, 24, replace=False):
        d = np.floor(np.sqrt(((p - p[i]) ** 2).sum(1).astype(np.float64)) + 0.5).astype(np.int64)
        d[i] = np.iinfo(np.int64).max
        order = np.lexsort((np.arange(n), d))[:32]
        assert np.array_equal(nn[i], order)
    if memory == 1:
        val, idx, tail = gpu.pheromone(0)
        live = idx >= 0
        assert val[live].min() >= tau0
        assert val[live].max() <= np.float32(1.0 / bl) * (1 + 2.0 ** -22)
    gpu.close()
