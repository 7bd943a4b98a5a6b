"""The relaxed construction (ACS-GPU-Alt, Sec. 3.1.2) on the GPU.

Its local updates race by design, so there is no bit-exact parity; the
checks are the properties that hold for any interleaving: every tour is a
permutation, lengths equal the recomputed EUC_2D sums, the best-so-far is the
minimum seen and only improves, tau0 <= tau <= 1/L_best on the matrix, the
counters add up, and with a single ant (no races) the colony equals the
synchronous one bit for bit.
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
    d = np.floor(np.sqrt(((a - b) ** 2).sum(-1).astype(np.float64)) + 0.5).astype(np.int64)
    return d.sum(1)


@pytest.mark.parametrize("n,m,kind", [(198, 32, "uniform"), (1002, 128, "clustered"),
                                      (33, 64, "uniform"), (5, 3, "uniform")])
def test_relaxed_tours_valid_and_pheromone_bounded(n, m, kind):
    xy = instances.uniform(n, seed=8) if kind == "uniform" else instances.clustered(n, seed=8)
    col = acs.Colony(xy, acs.params(m=m, cl=32, seed=3, relaxed=True))
    prev = None
    for it in range(4):
        col.run(1)
        t, L = col.tours(0)
        assert (np.sort(t, axis=1) == np.arange(n)).all()
        assert np.array_equal(_lengths(xy, t), L)
        bt, bl = col.best(0)
        assert np.array_equal(np.sort(bt), np.arange(n))
        assert _lengths(xy, bt[None, :])[0] == bl
        assert bl <= L.min()
        if prev is not None:
            assert bl <= prev
        prev = bl
    tau = col.pheromone(0)
    _, _, tau0, _ = col.setup(0)
    np.fill_diagonal(tau, tau0)
    assert tau.min() >= tau0
    assert tau.max() <= np.float32(1.0 / prev) * (1 + 2.0 ** -22)
    st = col.stats(0)
    assert st[1] == 4 * m * (n - 1)
    assert col.iteration == 4
    col.close()


def test_relaxed_single_ant_equals_synchronous(oracle_mod):
    # one ant has no races and its updates are seen at once by itself, as in
    # the synchronous step: the two constructions coincide
    xy = instances.clustered(300, seed=9)
    col = acs.Colony(xy, acs.params(m=1, cl=32, seed=5, relaxed=True))
    ref = oracle.Colony(xy, oracle.make_params(m=1, cl=32, seed=5))
    for _ in range(3):
        col.run(1)
        ref.run(1)
        tg, lg = col.tours(0)
        tr, lr = ref.tours()
        assert np.array_equal(tg, tr) and np.array_equal(lg, lr)
    assert np.array_equal(col.pheromone(0).view(np.uint32), ref.pheromone().view(np.uint32))
    col.close()


def test_relaxed_batch_and_launch_count():
    xy, off = instances.batch([120, 400, 260], ["uniform", "clustered", "uniform"], seed=2)
    col = acs.Colony(xy, acs.params(m=40, cl=32, seed=6, relaxed=True), offsets=off)
    assert col.autotune(1) == (32, 1)
    col.run(2)
    assert acs.acs_last_launch_count(col.ctx) == 4
    for b in range(3):
        sub = xy[off[b]:off[b + 1]]
        t, L = col.tours(b)
        assert (np.sort(t, axis=1) == np.arange(sub.shape[0])).all()
        assert np.array_equal(_lengths(sub, t), L)
    col.close()
