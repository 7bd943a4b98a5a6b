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


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_two_calls(lib):
    import torch

    dev = torch.device("cuda:0")
    xy = instances.clustered(300, seed=21)
    n, m = xy.shape[0], 48
    p = acs.params(m=m, cl=32, q0=0.9, seed=5)
    ref = acs.Colony(xy, p)
    nn, w, tau0, _ = ref.setup()
    cl = nn.shape[1]
    nn32 = np.full((n, 32), -1, np.int32)
    nn32[:, :cl] = nn
    w32 = np.zeros((n, 32), np.float32)
    w32[:, :cl] = w

    d_xy = torch.from_numpy(np.ascontiguousarray(xy)).to(dev)
    d_nn = torch.from_numpy(nn32).to(dev)
    d_w = torch.from_numpy(w32).to(dev)
    d_tau = torch.full((n, n), float(tau0), dtype=torch.float32, device=dev)
    d_tours = torch.zeros((m, n), dtype=torch.int32, device=dev)
    d_lens = torch.zeros(m, dtype=torch.int64, device=dev)
    d_best = torch.zeros(n, dtype=torch.int32, device=dev)
    d_best_len = torch.full((1,), np.iinfo(np.int64).max, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    torch.cuda.synchronize()

    for it in range(2):
        rc = acs.acs_iterate_noalloc(d_xy.data_ptr(), n, d_nn.data_ptr(), d_w.data_ptr(), cl,
                                     float(tau0), d_tau.data_ptr(), d_tours.data_ptr(),
                                     d_lens.data_ptr(), d_best.data_ptr(),
                                     d_best_len.data_ptr(), it, p, stream)
        assert rc == acs.ACS_OK, acs.strerror(rc)
        ref.run(1)
        tours, lens = ref.tours()
        best, best_len = ref.best()
        # same tolerance as every other parity test here: bit-identical
        assert np.array_equal(d_tours.cpu().numpy(), tours)
        assert np.array_equal(d_lens.cpu().numpy(), lens)
        assert np.array_equal(d_best.cpu().numpy(), best)
        assert int(d_best_len.cpu()[0]) == best_len
        assert np.array_equal(d_tau.cpu().numpy().view(np.uint32),
                              ref.pheromone().view(np.uint32))
    ref.close()
