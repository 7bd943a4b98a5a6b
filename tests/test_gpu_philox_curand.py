"""The device Philox4x32-10 against cuRAND's device function of the same name
(a library routine, on counters and keys drawn at random): an independent
check of the stream that the kernels draw from."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_device_philox_equals_curand(tmp_path):
    from paper_1605_02669_gb300 import build

    so = str(tmp_path / "philox_pair.so")
    cmd = [build._nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
           "-Xcompiler", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "paper_1605_02669_gb300", "csrc"),
           os.path.join(HERE, "cuda", "philox_vs_curand.cu"), "-o", so]
    subprocess.check_call(cmd)
    lib = ctypes.CDLL(so)
    rng = np.random.default_rng(5)
    count = 20000
    ctr = rng.integers(0, 2 ** 32, (count, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (count, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = 0
    ctr[4:8] = 0xFFFFFFFF
    key[:2] = 0
    ours = np.zeros((count, 4), np.uint32)
    theirs = np.zeros((count, 4), np.uint32)
    vp = ctypes.c_void_p
    rc = lib.philox_pair(ctr.ctypes.data_as(vp), key.ctypes.data_as(vp), count,
                         ours.ctypes.data_as(vp), theirs.ctypes.data_as(vp))
    assert rc == 0
    assert np.array_equal(ours, theirs)
