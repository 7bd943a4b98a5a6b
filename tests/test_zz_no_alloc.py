"""acs_iterate_noalloc: the entry point for callers that cannot allocate device
memory (code running inside an arena or pool it does not own, or on a hot
path where cudaMalloc is not allowed). It must give the same iteration as the
allocating entry points, using only the buffers the caller passes plus the
library's fixed static scratch array.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1605_02669_gb300 import acs, instances


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    return acs.load()


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    # m*ceil(n/32) > 1046464 words does not fit the 4 MiB scratch: rejected on
    # the host before any device work
    p = acs.params(m=1024, cl=32)
    rc = acs.acs_iterate_noalloc(8, 40000, 8, 8, 32, 1e-6, 8, 8, 8, 8, 8, 0, p)
    assert rc == acs.ACS_EINVAL
    rc = acs.acs_iterate_noalloc(8, 100, 8, 8, 32, 1e-6, 8, 8, 8, 8, 8, 0,
                                 acs.params(memory=acs.ACS_MEM_SPM))
    assert rc == acs.ACS_EINVAL


def _device_setup(xy, p, dev):
    """The allocating path's context for xy, and device copies of its tables
    padded to 32 columns, as a caller of acs_iterate_noalloc would hold them."""
    import torch

    n, m = xy.shape[0], p.m
    ref = acs.Colony(xy, p)
    nn, w, tau0, _ = ref.setup()
    cl = nn.shape[1]
    nn32 = np.full((n, 32), -1, np.int32)
    nn32[:, :cl] = nn
    w32 = np.zeros((n, 32), np.float32)
    w32[:, :cl] = w
    bufs = dict(
        xy=torch.from_numpy(np.ascontiguousarray(xy)).to(dev),
        nn=torch.from_numpy(nn32).to(dev),
        w=torch.from_numpy(w32).to(dev),
        tau=torch.full((n, n), float(tau0), dtype=torch.float32, device=dev),
        tours=torch.zeros((m, n), dtype=torch.int32, device=dev),
        lens=torch.zeros(m, dtype=torch.int64, device=dev),
        best=torch.zeros(n, dtype=torch.int32, device=dev),
        best_len=torch.full((1,), np.iinfo(np.int64).max, dtype=torch.int64, device=dev),
    )
    return ref, cl, float(tau0), bufs


def _call(b, n, cl, tau0, it, p, stream):
    return acs.acs_iterate_noalloc(b["xy"].data_ptr(), n, b["nn"].data_ptr(), b["w"].data_ptr(),
                                   cl, tau0, b["tau"].data_ptr(), b["tours"].data_ptr(),
                                   b["lens"].data_ptr(), b["best"].data_ptr(),
                                   b["best_len"].data_ptr(), it, p, stream)


def _assert_equal_state(b, tours, lens, best, best_len, tau):
    # same tolerance as every other parity test here: bit-identical
    assert np.array_equal(b["tours"].cpu().numpy(), tours)
    assert np.array_equal(b["lens"].cpu().numpy(), lens)
    assert np.array_equal(b["best"].cpu().numpy(), best)
    assert int(b["best_len"].cpu()[0]) == best_len
    assert np.array_equal(b["tau"].cpu().numpy().view(np.uint32), tau.view(np.uint32))


@pytest.mark.gpu
@pytest.mark.parametrize("n,m", [(300, 48), (700, 128)])
def test_noalloc_matches_allocating_entry_point_and_oracle_two_calls(lib, oracle_mod, n, m):
    # m = 128 gives the no-allocation launch its full 1024-thread CTA
    import torch

    import oracle

    dev = torch.device("cuda:0")
    xy = instances.clustered(n, seed=21)
    p = acs.params(m=m, cl=32, q0=0.9, seed=5)
    ref, cl, tau0, bufs = _device_setup(xy, p, dev)
    orc = oracle.Colony(xy, oracle.make_params(m=m, cl=32, q0=0.9, seed=5))
    assert np.float32(tau0) == orc.tau0
    stream = torch.cuda.current_stream(dev).cuda_stream
    torch.cuda.synchronize()
    for it in range(2):
        rc = _call(bufs, n, cl, tau0, it, p, stream)
        assert rc == acs.ACS_OK, acs.strerror(rc)
        ref.run(1)
        orc.run(1)
        t, L = ref.tours()
        bt, bl = ref.best()
        _assert_equal_state(bufs, t, L, bt, bl, ref.pheromone())
        t, L = orc.tours()
        bt, bl = orc.best()
        _assert_equal_state(bufs, t, L, bt, bl, orc.pheromone())
    ref.close()


@pytest.mark.gpu
def test_noalloc_at_the_scratch_bound_matches_allocating_entry_point(lib):
    # m * ceil(n/32) = 1024 * 1021 = 1,045,504 visited words, just under the
    # 1,046,464 that the 4 MiB array holds; m = 1024 is also the largest m.
    # (The oracle needs minutes at this size; the allocating path is the
    # reference here.)
    import torch

    dev = torch.device("cuda:0")
    n, m = 32672, 1024
    assert m * ((n + 31) // 32) <= 1046464 < m * ((n + 32 + 31) // 32)
    xy = instances.uniform(n, side=100000, seed=22)
    p = acs.params(m=m, cl=32, q0=0.9, seed=6)
    ref, cl, tau0, bufs = _device_setup(xy, p, dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    torch.cuda.synchronize()
    rc = _call(bufs, n, cl, tau0, 0, p, stream)
    assert rc == acs.ACS_OK, acs.strerror(rc)
    ref.run(1)
    t, L = ref.tours()
    bt, bl = ref.best()
    _assert_equal_state(bufs, t, L, bt, bl, ref.pheromone())
    # one node more does not fit
    assert _call(bufs, n + 32, cl, tau0, 1, p, stream) == acs.ACS_EINVAL
    ref.close()
