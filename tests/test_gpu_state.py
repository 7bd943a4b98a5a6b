"""Checkpoint / resume (acs_get_state, acs_set_state) and placement-independent
instance ids (acs_create_batch_ids), through the C ABI on the GPU.

The loop state of Alg. 1 is the pheromone memory, the best-so-far tour and
its length, and the iteration counter (the Philox counter word 0), so a run
split by a checkpoint must be bit-identical to the unsplit run; an instance's
random stream is keyed by its id, so running it alone or inside a batch must
give the same result.
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


def _same(a, b, memory, ia=0, ib=0):
    ta, la = a.tours(ia)
    tb, lb = b.tours(ib)
    assert np.array_equal(ta, tb) and np.array_equal(la, lb)
    assert a.best(ia)[1] == b.best(ib)[1]
    assert np.array_equal(a.best(ia)[0], b.best(ib)[0])
    if memory == 0:
        assert np.array_equal(a.pheromone(ia).view(np.uint32), b.pheromone(ib).view(np.uint32))
    else:
        for x, y in zip(a.pheromone(ia), b.pheromone(ib)):
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    assert a.stats(ia) == b.stats(ib)


@pytest.mark.parametrize("memory", [0, 1])
def test_split_run_equals_unsplit_run(oracle_mod, memory):
    xy = instances.clustered(500, seed=31)
    p = acs.params(m=48, cl=32, memory=memory, spm_slots=8, seed=9)
    whole = acs.Colony(xy, p)
    whole.run(20)
    first = acs.Colony(xy, p)
    first.run(7)
    buf = first.get_state()
    assert buf.nbytes == acs.acs_state_size(first.ctx, 0)
    first.close()
    second = acs.Colony(xy, p)
    second.set_state(buf)
    assert second.iteration == 7
    second.run(13)
    assert second.iteration == 20
    # tours of the last iteration, best tour, pheromone bytes, counters
    _same(whole, second, memory)
    ref = oracle.Colony(xy, oracle.make_params(m=48, cl=32, memory=memory, spm_slots=8, seed=9))
    ref.run(20)
    t, L = second.tours()
    assert np.array_equal(t, ref.tours()[0]) and np.array_equal(L, ref.tours()[1])
    assert second.stats() == ref.stats()


def test_state_restores_caller_candidate_rows(oracle_mod):
    # rows rewritten after set-up (as a learned prior does) belong to the state
    xy = instances.uniform(300, seed=32)
    p = acs.params(m=32, cl=32, seed=4)
    a = acs.Colony(xy, p)
    nn, w, _, _ = a.setup()
    keep = 12
    nn2 = np.ascontiguousarray(nn[:, ::-1][:, :keep])
    w2 = np.ascontiguousarray(w[:, ::-1][:, :keep] * np.float32(1.5))
    acs.acs_set_candidates(a.ctx, 0, nn2, w2)
    a.run(5)
    buf = a.get_state()
    b = acs.Colony(xy, p)
    b.set_state(buf)
    nb, wb, _, _ = b.setup()
    assert np.array_equal(nb, nn2) and np.array_equal(wb.view(np.uint32), w2.view(np.uint32))
    a.run(6)
    b.run(6)
    _same(a, b, 0)


def test_state_of_one_instance_of_a_batch(oracle_mod):
    xy, off, _, _ = instances.mixed_batch(3, 150, 400, seed=33)
    p = acs.params(m=24, cl=16, memory=1, spm_slots=4, seed=2)
    whole = acs.Colony(xy, p, offsets=off)
    whole.run(9)
    part = acs.Colony(xy, p, offsets=off)
    part.run(4)
    buf = part.get_state(2)
    fresh = acs.Colony(xy, p, offsets=off)
    fresh.run(4)          # instances 0 and 1 advance on their own
    fresh.set_state(buf, 2)
    fresh.run(5)
    for b in range(3):
        _same(whole, fresh, 1, b, b)


def test_bad_states_are_rejected_and_change_nothing(oracle_mod):
    xy = instances.uniform(200, seed=34)
    p = acs.params(m=16, cl=16, seed=3)
    a = acs.Colony(xy, p)
    a.run(3)
    good = a.get_state()
    b = acs.Colony(xy, p)
    b.run(2)
    before = b.get_state()

    def rejected(buf, target=b, inst=0):
        with pytest.raises(acs.AcsError) as e:
            target.set_state(buf, inst)
        assert e.value.status == acs.ACS_EINVAL

    rejected(good[:-1])                          # too short
    bad = good.copy()
    bad[0] ^= 1                                   # magic
    rejected(bad)
    hdr_best = 128 + 256 * 200                    # header, nn and w rows: best tour
    bad = good.copy()
    bad[hdr_best:hdr_best + 4] = bad[hdr_best + 4:hdr_best + 8]   # not a permutation
    rejected(bad)
    bad = good.copy()
    bad[128:132] = np.frombuffer(np.int32(200).tobytes(), np.uint8)   # node out of range
    rejected(bad)
    # another instance of the same size (other coordinates, other tau0)
    other = acs.Colony(instances.uniform(200, seed=35), p)
    rejected(good, other)
    # another size, another memory kind, other parameters
    rejected(good, acs.Colony(instances.uniform(201, seed=34), p))
    rejected(good, acs.Colony(xy, acs.params(m=16, cl=16, seed=3, memory=1)))
    rejected(good, acs.Colony(xy, acs.params(m=17, cl=16, seed=3)))
    rejected(good, acs.Colony(xy, acs.params(m=16, cl=16, seed=3, q0=0.8)))
    # the rejected calls left b as it was
    assert np.array_equal(b.get_state(), before)
    # a different seed is accepted (a fork of the run)
    c = acs.Colony(xy, acs.params(m=16, cl=16, seed=77))
    c.set_state(good)
    c.run(1)


def test_best_tour_available_after_restoring_a_state(oracle_mod):
    xy = instances.uniform(120, seed=36)
    p = acs.params(m=16, cl=16, seed=3)
    a = acs.Colony(xy, p)
    a.run(2)
    b = acs.Colony(xy, p)
    with pytest.raises(acs.AcsError):
        b.best()                                  # no iteration yet
    b.set_state(a.get_state())
    assert b.best()[1] == a.best()[1]


@pytest.mark.parametrize("memory", [0, 1])
def test_instance_alone_with_its_id_equals_inside_the_batch(oracle_mod, memory):
    # Philox counter word 3 is the instance id: a shard of a batch run with the
    # global ids reproduces the whole batch instance by instance
    xy, off, _, _ = instances.mixed_batch(5, 100, 500, seed=37)
    p = acs.params(m=32, cl=32, memory=memory, spm_slots=8, seed=6)
    whole = acs.Colony(xy, p, offsets=off)
    whole.run(4)
    shard_ids = [3, 1]
    sxy = np.concatenate([xy[off[b]:off[b + 1]] for b in shard_ids])
    soff = np.zeros(len(shard_ids) + 1, np.int64)
    soff[1:] = np.cumsum([off[b + 1] - off[b] for b in shard_ids])
    shard = acs.Colony(sxy, p, offsets=soff, instance_ids=shard_ids)
    shard.run(4)
    for k, b in enumerate(shard_ids):
        _same(whole, shard, memory, b, k)
    alone = acs.Colony(xy[off[4]:off[5]], p, instance_ids=[4])
    alone.run(4)
    _same(whole, alone, memory, 4, 0)
    ref = oracle.Colony(xy[off[4]:off[5]], oracle.make_params(m=32, cl=32, memory=memory,
                                                                spm_slots=8, seed=6), instance=4)
    ref.run(4)
    assert np.array_equal(alone.tours()[0], ref.tours()[0])
