"""The autotuning cache on the GPU: a miss tunes and stores, a hit applies the
stored shape, and the colony stays bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1605_02669_gb300 import acs, instances, tuning

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("memory", [0, 1])
def test_cached_shape_is_applied_and_results_unchanged(oracle_mod, tmp_path, memory):
    path = str(tmp_path / "tune.json")
    xy, off = instances.batch([300, 520], ["clustered", "uniform"], seed=5)
    p = acs.params(m=48, cl=32, memory=memory, spm_slots=8, seed=4)
    first = acs.Colony(xy, p, offsets=off)
    ent, hit = tuning.tune(first, path, trial_iters=1)
    assert not hit
    first.close()
    col = acs.Colony(xy, p, offsets=off)
    ent2, hit2 = tuning.tune(col, path)
    assert hit2 and ent2 == ent
    assert col.threads_per_ant == ent["threads_per_ant"]
    assert col.cluster_size == ent["cluster_size"]
    col.run(2)
    for b in range(2):
        ref = oracle.Colony(xy[off[b]:off[b + 1]],
                            oracle.make_params(m=48, cl=32, memory=memory, spm_slots=8, seed=4),
                            instance=b)
        ref.run(2)
        tg, lg = col.tours(b)
        tr, lr = ref.tours()
        assert np.array_equal(tg, tr) and np.array_equal(lg, lr)
    col.close()
