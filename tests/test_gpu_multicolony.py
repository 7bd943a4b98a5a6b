"""Multi-colony best-tour exchange on the GPU, against the oracle fed the same
offers: the colony state stays bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1605_02669_gb300 import acs, instances, multicolony

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _same(gpu, ref, b=0, memory=0):
    tg, lg = gpu.tours(b)
    tr, lr = ref.tours()
    assert np.array_equal(tg, tr) and np.array_equal(lg, lr)
    bg, blg = gpu.best(b)
    br, blr = ref.best()
    assert blg == blr and np.array_equal(bg, br)
    if memory == 0:
        assert np.array_equal(gpu.pheromone(b).view(np.uint32), ref.pheromone().view(np.uint32))


@pytest.mark.parametrize("memory", [0, 1])
def test_offer_best_then_run_matches_oracle(oracle_mod, memory):
    xy = instances.clustered(400, seed=21)
    kw = dict(m=32, cl=32, q0=0.9, memory=memory, spm_slots=8, seed=7)
    gpu = acs.Colony(xy, acs.params(**kw))
    ref = oracle.Colony(xy, oracle.make_params(**kw))
    gpu.run(2)
    ref.run(2)
    # a better tour from another (longer) colony with another seed
    other = oracle.Colony(xy, oracle.make_params(**dict(kw, seed=99)))
    other.run(12)
    tour, L = other.best()
    got = gpu.offer_best(tour)
    ref.offer_best(tour)
    assert got == L
    assert gpu.best(0)[1] == ref.best()[1] == min(L, ref.best()[1])
    gpu.run(2)
    ref.run(2)
    _same(gpu, ref, memory=memory)
    # a longer tour is refused; a non-permutation is an error
    before = gpu.best(0)[1]
    gpu.offer_best(np.arange(400, dtype=np.int32))
    assert gpu.best(0)[1] == before
    with pytest.raises(acs.AcsError):
        gpu.offer_best(np.zeros(400, np.int32))


def test_replica_exchange_matches_oracle(oracle_mod):
    base = instances.uniform(300, seed=22)
    xy = np.concatenate([base] * 3)
    off = np.array([0, 300, 600, 900], np.int64)
    kw = dict(m=24, cl=32, q0=0.9, seed=5)
    gpu = acs.Colony(xy, acs.params(**kw), offsets=off)
    refs = [oracle.Colony(base, oracle.make_params(**kw), instance=b) for b in range(3)]
    for _ in range(3):
        gpu.run(2)
        for r in refs:
            r.run(2)
        win, L = multicolony.exchange_replicas(gpu, [0, 1, 2])
        # the same exchange on the oracle side
        lens = [r.best()[1] for r in refs]
        rwin = min(range(3), key=lambda b: (lens[b], b))
        assert (win, L) == (rwin, lens[rwin])
        for b in range(3):
            if b != rwin:
                refs[b].offer_best(refs[rwin].best()[0])
        for b in range(3):
            assert gpu.best(b)[1] == L
    for b in range(3):
        _same(gpu, refs[b], b)
