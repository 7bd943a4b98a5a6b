"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/*.h, and rejects bad arguments before
touching the device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_1605_02669_gb300 import acs, instances

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    return acs.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(acs_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"acs_create", "acs_create_batch", "acs_run_iterations", "acs_best_tour",
            "acs_destroy"} <= names
    for name in sorted(names):
        assert hasattr(lib, name), name


def test_strerror(lib):
    for s in range(6):
        assert acs.strerror(s)
    assert "invalid" in acs.strerror(acs.ACS_EINVAL)


def _create_status(coords, p, n=None):
    coords = np.ascontiguousarray(coords, np.int32)
    h = ctypes.c_void_p()
    n = coords.shape[0] if n is None else n
    return acs.load().acs_create(coords.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(p),
                                 ctypes.byref(h)), h


@pytest.mark.parametrize("kw", [dict(m=0), dict(m=1025), dict(cl=0), dict(cl=33),
                                dict(q0=-0.1), dict(q0=1.5), dict(rho=0.0), dict(rho=1.0),
                                dict(xi=0.0), dict(beta=-1), dict(beta=9),
                                dict(memory=3), dict(memory=1, spm_slots=0),
                                dict(memory=1, spm_slots=33), dict(local_period=0),
                                dict(memory=1, relaxed=True)])
def test_bad_params_rejected_on_host(lib, kw):
    xy = instances.uniform(20, seed=1)
    rc, h = _create_status(xy, acs.params(**kw))
    assert rc == acs.ACS_EINVAL and not h.value


def test_unknown_flags_rejected_on_host(lib):
    xy = instances.uniform(20, seed=1)
    p = acs.params()
    p.flags = 4
    rc, h = _create_status(xy, p)
    assert rc == acs.ACS_EINVAL and not h.value


def test_bad_coords_and_sizes_rejected_on_host(lib):
    xy = instances.uniform(20, seed=1)
    rc, _ = _create_status(xy, acs.params(), n=2)
    assert rc == acs.ACS_EINVAL
    bad = xy.copy()
    bad[3, 1] = 1 << 20
    assert _create_status(bad, acs.params())[0] == acs.ACS_EINVAL
    bad[3, 1] = -5
    assert _create_status(bad, acs.params())[0] == acs.ACS_EINVAL
    p = acs.params()
    assert lib.acs_create(None, 20, ctypes.byref(p), None) == acs.ACS_EINVAL
    off = np.array([0, 10, 12], np.int64)  # second instance has 2 nodes
    h = ctypes.c_void_p()
    xy = np.ascontiguousarray(xy)
    assert lib.acs_create_batch(xy.ctypes.data_as(ctypes.c_void_p),
                                off.ctypes.data_as(ctypes.c_void_p), 2, ctypes.byref(p),
                                ctypes.byref(h)) == acs.ACS_EINVAL
    # more instances than a grid dimension holds: rejected before any device work
    assert lib.acs_create_batch(xy.ctypes.data_as(ctypes.c_void_p),
                                off.ctypes.data_as(ctypes.c_void_p), 65536, ctypes.byref(p),
                                ctypes.byref(h)) == acs.ACS_EINVAL


def test_null_context_calls(lib):
    assert lib.acs_run_iterations(None, 1) == acs.ACS_EINVAL
    assert lib.acs_best_tour(None, 0, None, None) == acs.ACS_EINVAL
    assert lib.acs_iteration(None) == -1
    assert lib.acs_set_spm_resident(None, 1) == acs.ACS_EINVAL
    assert lib.acs_set_cluster_size(None, 2) == acs.ACS_EINVAL
    assert lib.acs_set_threads_per_ant(None, 8) == acs.ACS_EINVAL
    assert lib.acs_autotune(None, 1, None, None) == acs.ACS_EINVAL
    assert lib.acs_autotune_group(None, 2, 1) == acs.ACS_EINVAL
    nulls = (ctypes.c_void_p * 2)(None, None)
    assert lib.acs_autotune_group(nulls, 2, 1) == acs.ACS_EINVAL
    assert lib.acs_autotune_group(nulls, 0, 1) == acs.ACS_EINVAL
    lib.acs_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(acs, "_lib", None)
    monkeypatch.setattr(acs, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        acs.load()


def test_prior_calls_reject_bad_arguments_on_host(lib):
    E = acs.ACS_EINVAL
    vp = ctypes.c_void_p
    fake = vp(0x1000)   # never dereferenced: every call below fails its checks first
    assert lib.acs_prior_features(None, 0, fake, None) == E
    assert lib.acs_prior_features(fake, 0, None, None) == E
    assert lib.acs_prior_count_best_edges(None, 0, fake, None) == E
    assert lib.acs_apply_prior(None, 0, fake, 16, None) == E
    assert lib.acs_apply_prior(fake, 0, None, 16, None) == E
    assert lib.acs_set_candidates(None, 0, fake, fake, 16) == E
    assert lib.acs_mlp_forward(fake, fake, -1, fake, None) == E
    assert lib.acs_mlp_forward(None, fake, 5, fake, None) == E
    assert lib.acs_mlp_forward(None, None, 0, None, None) == acs.ACS_OK   # nothing to do
    assert lib.acs_mlp_forward(fake, vp(0x1008), 5, fake, None) == E   # feature rows not 16-byte aligned
    assert lib.acs_mlp_train_batch(fake, fake, fake, 0, 0, 1, 1, 0, fake, fake, None) == E
    assert lib.acs_mlp_train_batch(fake, fake, fake, 10, 0, 0, 1, 0, fake, fake, None) == E
    assert lib.acs_mlp_train_batch(fake, fake, fake, 10, 0, 4, 0, 0, fake, fake, None) == E
    assert lib.acs_mlp_train_batch(fake, fake, None, 10, 0, 4, 1, 0, fake, fake, None) == E
    assert lib.acs_mlp_train_batch(fake, vp(0x1008), fake, 10, 0, 4, 1, 0, fake, fake, None) == E
    assert lib.acs_mlp_adam(fake, fake, fake, fake, 0, 1e-3, 0.9, 0.999, 1e-8, None) == E
    assert lib.acs_mlp_adam(None, fake, fake, fake, 1, 1e-3, 0.9, 0.999, 1e-8, None) == E
    assert lib.acs_kernel_mode(None) == -1
