"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer and index results (tours, lengths, SPM slots) and FP32 pheromone
bytes must be identical: the determinism contract fixes one correct result
per (instance, parameters, seed).
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


def _pair(xy, memory=0, **kw):
    p = acs.params(memory=memory, **kw)
    q = oracle.make_params(memory=memory, **kw)
    return acs.Colony(xy, p), oracle.Colony(xy, q)


def assert_same_state(gpu, ref, memory, b=0):
    tg, lg = gpu.tours(b)
    tr, lr = ref.tours()
    assert np.array_equal(tg, tr), "tours differ (first ant %d)" % int(
        np.where((tg != tr).any(1))[0][0])
    assert np.array_equal(lg, lr)
    bg, blg = gpu.best(b)
    br, blr = ref.best()
    assert blg == blr and np.array_equal(bg, br)
    if memory == 0:
        a = gpu.pheromone(b).view(np.uint32)
        r = ref.pheromone().view(np.uint32)
        assert np.array_equal(a, r), "pheromone differs at %d entries" % int((a != r).sum())
    else:
        gv, gi, gt = gpu.pheromone(b)
        rv, ri, rt = ref.pheromone()
        assert np.array_equal(gi, ri), "SPM slot indices differ"
        assert np.array_equal(gt, rt), "SPM tails differ"
        assert np.array_equal(gv.view(np.uint32), rv.view(np.uint32)), "SPM trails differ"
    sg = gpu.stats(b)
    sr = ref.stats()
    assert sg == sr, (sg, sr)


def test_setup_tables_match(oracle_mod):
    xy = instances.clustered(300, seed=4)
    gpu, ref = _pair(xy, m=8, cl=32)
    nn, w, tau0, lnn = gpu.setup()
    assert np.array_equal(nn, ref.nn)
    assert np.array_equal(w.view(np.uint32), ref.w.view(np.uint32))
    assert tau0 == ref.tau0 and lnn == ref.L_nn


@pytest.mark.parametrize("memory", [0, 1])
def test_config_n198_m32_every_iteration(oracle_mod, memory):
    # n=198 uniform in [0,10000]^2, m=32, 32-NN, beta=2, q0=0.9, rho=xi=0.1, seed 1
    xy = instances.uniform(198, side=10000, seed=1)
    gpu, ref = _pair(xy, memory=memory, m=32, cl=32, spm_slots=8, seed=1)
    for _ in range(8):
        gpu.run(1)
        ref.run(1)
        assert_same_state(gpu, ref, memory)


@pytest.mark.parametrize("memory", [0, 1])
def test_config_n198_m32_200_iterations(oracle_mod, memory):
    # the single-instance configuration over its full 200 iterations: the state
    # stays bit-identical through long stagnation (ties, repeated best tours)
    xy = instances.uniform(198, side=10000, seed=1)
    gpu, ref = _pair(xy, memory=memory, m=32, cl=32, spm_slots=8, seed=1)
    for _ in range(4):
        gpu.run(50)
        ref.run(50)
        assert_same_state(gpu, ref, memory)
    assert np.array_equal(np.asarray(gpu.stats(0)), np.asarray(ref.stats()))


EDGE_CASES = [
    dict(n=3, m=1, cl=32),
    dict(n=4, m=3, cl=32, q0=0.0),
    dict(n=5, m=7, cl=2, q0=1.0),
    dict(n=9, m=5, cl=8, beta=0),
    dict(n=31, m=33, cl=32, q0=0.5),
    dict(n=32, m=16, cl=5, beta=5),
    dict(n=33, m=40, cl=32, local_period=2),
    dict(n=65, m=64, cl=16, local_period=3, q0=0.3),
    dict(n=65, m=9, cl=1, q0=1.0, beta=0),
    dict(n=100, m=70, cl=10, q0=0.0),
    # small candidate lists: many full-scan fallbacks per step, queued by
    # several CTAs of a cluster at once
    dict(n=300, m=48, cl=4, q0=0.9),
    dict(n=300, m=48, cl=4, beta=0),
    dict(n=520, m=20, cl=2, q0=0.5),
]


@pytest.mark.parametrize("case", EDGE_CASES, ids=lambda c: "-".join("%s%s" % kv for kv in c.items()))
@pytest.mark.parametrize("memory,slots", [(0, 8), (1, 1), (1, 3), (1, 8)])
def test_edge_cases(oracle_mod, case, memory, slots):
    case = dict(case)
    n = case.pop("n")
    xy = instances.uniform(n, side=1000, seed=n)
    gpu, ref = _pair(xy, memory=memory, spm_slots=slots, seed=5, **case)
    for _ in range(4):
        gpu.run(1)
        ref.run(1)
        assert_same_state(gpu, ref, memory)


@pytest.mark.parametrize("tpa,m,n0,ndup", [(4, 16, 600, 120), (32, 4, 900, 200)])
@pytest.mark.parametrize("beta", [0, 2, 8])
def test_spm_extended_list_ties(oracle_mod, beta, tpa, m, n0, ndup):
    # The SPM settles empty candidate sets from a per-node list sorted by the
    # full scan's key when a scan would be long. 160 instances on one-CTA
    # clusters (more clusters than SMs, so small CTAs: m x lanes per ant = 64
    # or 128 threads, and a scan of n0 + ndup nodes would deal each warp more
    # than two items) select that path, with 4 and with 32 lanes per ant. Duplicated points (d = 0 weighs like d = 1), beta 0
    # (every heuristic equal: the lowest index wins) and beta 8 (products
    # underflow to denormals and to zero) make many equal keys; two candidates
    # make empty candidate sets frequent, so the list path and, once all 256
    # listed nodes are visited, the full scan both run.
    B = 160
    parts = []
    for b in range(B):
        base = instances.uniform(n0, side=700, seed=beta + 3, stream=b)
        parts.append(np.concatenate([base, base[:ndup]]))
    xy = np.concatenate(parts).astype(np.int32)
    off = np.arange(B + 1, dtype=np.int64) * (n0 + ndup)
    kw = dict(memory=1, m=m, cl=2, spm_slots=4, beta=beta, seed=9)
    gpu = acs.Colony(xy, acs.params(**kw), offsets=off)
    gpu.set_cluster_size(1)
    gpu.set_threads_per_ant(tpa)
    gpu.run(2)
    for b in (0, 1, 37, 80, 121, 159):
        ref = oracle.Colony(xy[off[b]:off[b + 1]], oracle.make_params(**kw), instance=b)
        ref.run(2)
        assert_same_state(gpu, ref, 1, b)


@pytest.mark.parametrize("memory", [0, 1])
def test_m128_n1002_clustered(oracle_mod, memory):
    xy = instances.clustered(1002, seed=2)
    gpu, ref = _pair(xy, memory=memory, m=128, cl=32, spm_slots=8, seed=1)
    for _ in range(2):
        gpu.run(1)
        ref.run(1)
    assert_same_state(gpu, ref, memory)


@pytest.mark.parametrize("memory", [0, 1])
def test_full_size_n2392_m128(oracle_mod, memory):
    # the bench workload's larger instance, one iteration, full state
    xy = instances.clustered(2392, seed=2)
    gpu, ref = _pair(xy, memory=memory, m=128, cl=32, spm_slots=8, seed=1)
    gpu.run(1)
    ref.run(1)
    assert_same_state(gpu, ref, memory)


def test_visited_in_global_memory_path(oracle_mod):
    # m=1024 ants on 1200 nodes: the visited bitmasks exceed shared memory
    xy = instances.uniform(1200, seed=9)
    gpu, ref = _pair(xy, m=1024, cl=32, q0=0.7, seed=3)
    gpu.run(1)
    ref.run(1)
    assert_same_state(gpu, ref, 0)


@pytest.mark.parametrize("memory", [0, 1])
def test_batch_matches_per_instance_oracle(oracle_mod, memory):
    sizes = [50, 301, 7, 128, 33, 260]
    kinds = ["uniform", "clustered"] * 3
    xy, off = instances.batch(sizes, kinds, seed=4)
    p = acs.params(m=24, cl=16, memory=memory, spm_slots=6, seed=11)
    gpu = acs.Colony(xy, p, offsets=off)
    refs = [oracle.Colony(xy[off[b]:off[b + 1]],
                          oracle.make_params(m=24, cl=16, memory=memory, spm_slots=6, seed=11),
                          instance=b) for b in range(len(sizes))]
    for _ in range(3):
        gpu.run(1)
        for r in refs:
            r.run(1)
        for b, r in enumerate(refs):
            assert_same_state(gpu, r, memory, b)


def test_contexts_of_different_sizes_interleaved(oracle_mod):
    # a large layout created first, a small one second, then both used in turn:
    # the second context must not break the first one's launches
    xa = instances.clustered(1002, seed=8)
    xb = instances.uniform(40, seed=8)
    ga, ra = _pair(xa, m=128, cl=32, seed=2)
    gb, rb = _pair(xb, m=4, cl=8, seed=2)
    for _ in range(2):
        gb.run(1)
        rb.run(1)
        ga.run(1)
        ra.run(1)
    assert_same_state(ga, ra, 0)
    assert_same_state(gb, rb, 0)


@pytest.mark.parametrize("tpa", [4, 8, 16, 32])
@pytest.mark.parametrize("memory", [0, 1])
def test_threads_per_ant_variants_are_identical(oracle_mod, tpa, memory):
    xy = instances.clustered(700, seed=12)
    gpu, ref = _pair(xy, memory=memory, m=96, cl=32, spm_slots=8, q0=0.8, seed=4)
    gpu.set_threads_per_ant(tpa)
    for _ in range(2):
        gpu.run(1)
        ref.run(1)
    assert_same_state(gpu, ref, memory)


@pytest.mark.parametrize("tpa", [4, 32])
@pytest.mark.parametrize("case", [dict(n=33, m=40, cl=32, local_period=2),
                                  dict(n=300, m=48, cl=4, beta=0),
                                  dict(n=65, m=9, cl=1, q0=1.0, beta=0)])
def test_edge_cases_other_widths(oracle_mod, tpa, case):
    case = dict(case)
    n = case.pop("n")
    xy = instances.uniform(n, side=1000, seed=n)
    for memory in (0, 1):
        gpu, ref = _pair(xy, memory=memory, spm_slots=3, seed=5, **case)
        gpu.set_threads_per_ant(tpa)
        for _ in range(3):
            gpu.run(1)
            ref.run(1)
        assert_same_state(gpu, ref, memory)


@pytest.mark.parametrize("csize", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("memory", [0, 1])
def test_cluster_sizes_are_identical(oracle_mod, csize, memory):
    # one instance shared by csize CTAs exchanging edges through DSMEM
    xy = instances.clustered(700, seed=14)
    gpu, ref = _pair(xy, memory=memory, m=96, cl=32, spm_slots=8, q0=0.8, seed=9)
    try:
        gpu.set_cluster_size(csize)
    except acs.AcsError as e:
        if csize == 16 and e.status == acs.ACS_EINVAL:
            pytest.skip("16-CTA clusters cannot be scheduled for this layout")
        raise
    assert gpu.cluster_size == csize
    for _ in range(2):
        gpu.run(1)
        ref.run(1)
    assert_same_state(gpu, ref, memory)


@pytest.mark.parametrize("csize,tpa", [(1, 8), (4, 16), (16, 32)])
def test_spm_records_in_global_memory(oracle_mod, csize, tpa):
    # records kept in global memory instead of the cluster's shared memory
    xy = instances.clustered(700, seed=16)
    gpu, ref = _pair(xy, memory=1, m=96, cl=32, spm_slots=8, q0=0.8, seed=11)
    gpu.set_spm_resident(0)
    gpu.set_cluster_size(csize)
    gpu.set_threads_per_ant(tpa)
    assert gpu.kernel_mode == 1
    for _ in range(2):
        gpu.run(1)
        ref.run(1)
    assert_same_state(gpu, ref, 1)
    gpu.set_spm_resident(1)
    assert gpu.kernel_mode == 2
    gpu.run(1)
    ref.run(1)
    assert_same_state(gpu, ref, 1)


@pytest.mark.parametrize("resident", [1, 0])
def test_spm_skip_default_variant(oracle_mod, resident):
    # the variant of the insert rule: absent edges keep tau0 without an insert
    xy = instances.clustered(600, seed=18)
    kw = dict(m=64, cl=32, q0=0.85, memory=1, spm_slots=4, seed=12)
    gpu = acs.Colony(xy, acs.params(spm_skip_default=True, **kw))
    gpu.set_spm_resident(resident)
    ref = oracle.Colony(xy, oracle.make_params(spm_skip_default=True, **kw))
    for _ in range(3):
        gpu.run(1)
        ref.run(1)
        assert_same_state(gpu, ref, 1)
    assert np.array_equal(np.asarray(gpu.stats(0)), np.asarray(ref.stats()))


@pytest.mark.parametrize("slots", [1, 2, 4, 8, 16, 32])
def test_spm_hit_ratio_sweep(oracle_mod, slots):
    # the hit ratio of the SPM counters, bit-exact with the oracle, in [0, 1]
    xy = instances.uniform(400, seed=19)
    kw = dict(m=32, cl=32, q0=0.9, memory=1, spm_slots=slots, seed=13)
    gpu = acs.Colony(xy, acs.params(**kw))
    ref = oracle.Colony(xy, oracle.make_params(**kw))
    gpu.run(3)
    ref.run(3)
    g = np.asarray(gpu.stats(0))
    assert np.array_equal(g, np.asarray(ref.stats()))
    hits, misses = int(g[2]), int(g[3])
    assert 0 <= hits / (hits + misses) <= 1


def test_uneven_ant_split_over_cluster(oracle_mod):
    # m not a multiple of the cluster size: the last CTA owns fewer ants
    xy = instances.uniform(260, seed=15)
    for memory in (0, 1):
        gpu, ref = _pair(xy, memory=memory, m=37, cl=16, spm_slots=4, q0=0.6, seed=10)
        gpu.set_cluster_size(8)
        gpu.set_threads_per_ant(16)
        for _ in range(3):
            gpu.run(1)
            ref.run(1)
        assert_same_state(gpu, ref, memory)


def test_autotune_keeps_state(oracle_mod):
    xy = instances.clustered(500, seed=13)
    gpu, ref = _pair(xy, m=64, cl=32, seed=6)
    gpu.run(1)
    ref.run(1)
    tpa, cs = gpu.autotune(2)
    assert tpa in (4, 8, 16, 32) and cs in (1, 2, 4, 8, 16) and gpu.iteration == 1
    assert gpu.threads_per_ant == tpa and gpu.cluster_size == cs
    gpu.run(2)
    ref.run(2)
    assert_same_state(gpu, ref, 0)


def test_autotune_on_fresh_batch_then_parity(oracle_mod):
    # the autotuner snapshots and restores the full state between trials; on
    # a fresh context the best tour is still uninitialised, so a restore that
    # raced with the next trial would feed garbage nodes to the kernel
    sizes = [120, 300, 77, 260]
    xy, off = instances.batch(sizes, ["uniform", "clustered"] * 2, seed=9)
    p = acs.params(m=32, cl=16, seed=12)
    gpu = acs.Colony(xy, p, offsets=off)
    tpa, cs = gpu.autotune(2)
    assert gpu.iteration == 0
    refs = [oracle.Colony(xy[off[b]:off[b + 1]], oracle.make_params(m=32, cl=16, seed=12),
                          instance=b) for b in range(len(sizes))]
    gpu.run(2)
    for b, r in enumerate(refs):
        r.run(2)
        assert_same_state(gpu, r, 0, b)


@pytest.mark.parametrize("memory", [0, 1])
def test_dynamic_instance_schedule_parity(oracle_mod, memory):
    # 400 instances on 1024-thread CTAs (32 lanes x 32 ants, one cluster of
    # one CTA per instance): at most one CTA per SM is resident, so the
    # clusters take instances from the counter after the first wave
    rng = np.random.default_rng(31)
    sizes = [int(x) for x in rng.integers(20, 90, 400)]
    xy, off = instances.batch(sizes, ["uniform", "clustered"] * 200, seed=17)
    kw = dict(m=32, cl=16, memory=memory, spm_slots=4, seed=5)
    gpu = acs.Colony(xy, acs.params(**kw), offsets=off)
    gpu.set_cluster_size(1)
    gpu.set_threads_per_ant(32)
    assert gpu.cluster_size == 1 and gpu.threads_per_ant == 32
    gpu.run(2)
    for b in range(len(sizes)):
        r = oracle.Colony(xy[off[b]:off[b + 1]], oracle.make_params(**kw), instance=b)
        r.run(2)
        assert_same_state(gpu, r, memory, b)


def test_group_autotune_keeps_state(oracle_mod):
    import torch

    sizes = [150, 320, 90, 260, 200, 120]
    xy, off = instances.batch(sizes, ["uniform", "clustered"] * 3, seed=23)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    cols, kws = [], []
    for memory, st in zip((0, 1), streams):
        kw = dict(m=32, cl=16, memory=memory, spm_slots=8, seed=3)
        c = acs.Colony(xy, acs.params(**kw), offsets=off)
        c.set_stream(st.cuda_stream)
        c.run(1)
        cols.append(c)
        kws.append(kw)
    acs.autotune_group(cols, trial_iters=1)
    for c in cols:
        assert c.iteration == 1
        c.run(2)
    torch.cuda.synchronize()
    for c, kw in zip(cols, kws):
        for b in range(len(sizes)):
            r = oracle.Colony(xy[off[b]:off[b + 1]], oracle.make_params(**kw), instance=b)
            r.run(3)
            assert_same_state(c, r, kw["memory"], b)


def test_repeatable_bits(oracle_mod):
    xy = instances.clustered(400, seed=6)
    runs = []
    for _ in range(3):
        g = acs.Colony(xy, acs.params(m=64, cl=32, seed=2))
        g.run(3)
        runs.append((g.tours()[0], g.pheromone().view(np.uint32)))
        g.close()
    for t, tau in runs[1:]:
        assert np.array_equal(t, runs[0][0]) and np.array_equal(tau, runs[0][1])
