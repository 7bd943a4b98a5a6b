"""ctypes loader for the plain C oracle in ``acs_oracle.c``.

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``. The
product package never imports this module.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "acs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_acs.so")
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

_lib = None


def build(force=False):
    """Compile the oracle with gcc (no FMA contraction, IEEE FP32)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "acs_oracle.h"))
    ):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int32),
        ("cl", ctypes.c_int32),
        ("beta", ctypes.c_int32),
        ("q0", ctypes.c_float),
        ("rho", ctypes.c_float),
        ("xi", ctypes.c_float),
        ("memory", ctypes.c_int32),
        ("spm_slots", ctypes.c_int32),
        ("local_period", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


FLAG_SPM_SKIP_DEFAULT = 2


def make_params(m=32, cl=32, beta=2, q0=0.9, rho=0.1, xi=0.1, memory=0,
                spm_slots=8, local_period=1, seed=1, spm_skip_default=False):
    return Params(m, cl, beta, q0, rho, xi, memory, spm_slots, local_period,
                  FLAG_SPM_SKIP_DEFAULT if spm_skip_default else 0, seed)


_P = np.ctypeslib.ndpointer
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_vp = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.acsref_philox4x32_10.argtypes = [_P(np.uint32), _P(np.uint32), _P(np.uint32)]
        L.acsref_dist.argtypes = [_P(np.int32), _i32, _i32]
        L.acsref_dist.restype = _i32
        L.acsref_heuristic.argtypes = [_i32, _i32]
        L.acsref_heuristic.restype = ctypes.c_float
        L.acsref_scan32.argtypes = [_P(np.float32), _P(np.float32)]
        L.acsref_pick.argtypes = [_P(np.float32), _P(np.int32), ctypes.c_float,
                                  ctypes.c_float, ctypes.c_float]
        L.acsref_pick.restype = _i32
        L.acsref_local_value.argtypes = [ctypes.c_float] * 3
        L.acsref_local_value.restype = ctypes.c_float
        L.acsref_global_value.argtypes = [ctypes.c_float] * 3
        L.acsref_global_value.restype = ctypes.c_float
        L.acsref_decay_table.argtypes = [ctypes.c_float, _i32, _P(np.float32)]
        L.acsref_knn.argtypes = [_P(np.int32), _i32, _i32, _P(np.int32)]
        L.acsref_knn.restype = ctypes.c_int
        L.acsref_nn_tour_length.argtypes = [_P(np.int32), _i32]
        L.acsref_nn_tour_length.restype = _i64
        L.acsref_spm_update.argtypes = [_P(np.int32), _P(np.float32), _P(np.int32), _i32,
                                        _i32, ctypes.c_float, _i32, ctypes.c_float,
                                        ctypes.c_float, _P(np.int64), _P(np.int64)]
        L.acsref_create.argtypes = [_P(np.int32), _i32, ctypes.POINTER(Params), _i32,
                                    ctypes.POINTER(_vp)]
        L.acsref_create.restype = ctypes.c_int
        L.acsref_create_tables.argtypes = [_P(np.int32), _i32, _P(np.int32), _P(np.float32),
                                           _i32, ctypes.POINTER(Params), _i32,
                                           ctypes.POINTER(_vp)]
        L.acsref_create_tables.restype = ctypes.c_int
        L.acsref_run.argtypes = [_vp, _i32]
        L.acsref_run.restype = ctypes.c_int
        L.acsref_local_step.argtypes = [_vp, _P(np.int32), _P(np.int32)]
        L.acsref_local_step.restype = ctypes.c_int
        L.acsref_get_tours.argtypes = [_vp, _P(np.int32), _P(np.int64)]
        L.acsref_best.argtypes = [_vp, _P(np.int32), ctypes.POINTER(_i64)]
        L.acsref_best.restype = ctypes.c_int
        L.acsref_offer_best.argtypes = [_vp, _P(np.int32)]
        L.acsref_offer_best.restype = ctypes.c_int
        L.acsref_get_pheromone.argtypes = [_vp, _P(np.float32), _vp, _vp]
        L.acsref_get_setup.argtypes = [_vp, _P(np.int32), _P(np.float32),
                                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_i64),
                                       ctypes.POINTER(_i32)]
        L.acsref_iteration.argtypes = [_vp]
        L.acsref_iteration.restype = _i64
        L.acsref_stats.argtypes = [_vp, _P(np.int64)]
        L.acsref_destroy.argtypes = [_vp]
        _lib = L
    return _lib


def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().acsref_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def dist(xy, i, j):
    return lib().acsref_dist(np.ascontiguousarray(xy, np.int32).reshape(-1), i, j)


def heuristic(d, beta):
    return np.float32(lib().acsref_heuristic(int(d), int(beta)))


def scan32(v):
    P = np.zeros(32, np.float32)
    lib().acsref_scan32(np.ascontiguousarray(v, np.float32), P)
    return P


def pick(v, unvisited, q, q0, r):
    return lib().acsref_pick(np.ascontiguousarray(v, np.float32),
                             np.ascontiguousarray(unvisited, np.int32), q, q0, r)


def local_value(tau, tau0, Pk):
    return np.float32(lib().acsref_local_value(tau, tau0, Pk))


def global_value(tau, delta, rho):
    return np.float32(lib().acsref_global_value(tau, delta, rho))


def decay_table(xi, kmax):
    P = np.zeros(kmax + 1, np.float32)
    lib().acsref_decay_table(xi, kmax, P)
    return P


def knn(xy, cl):
    xy = np.ascontiguousarray(xy, np.int32)
    n = xy.shape[0]
    nn = np.zeros((n, cl), np.int32)
    rc = lib().acsref_knn(xy.reshape(-1), n, cl, nn)
    assert rc == 0
    return nn


def nn_tour_length(xy):
    xy = np.ascontiguousarray(xy, np.int32)
    return int(lib().acsref_nn_tour_length(xy.reshape(-1), xy.shape[0]))


def spm_update(idx, val, tail, nb, tau0, mode, coef, target, hits, misses):
    """In-place Alg. 3 update of one record (numpy arrays; tail/hits/misses 1-elt)."""
    lib().acsref_spm_update(idx, val, tail, idx.shape[0], nb, tau0, mode, coef, target,
                            hits, misses)


class OracleError(RuntimeError):
    pass


class Colony:
    """One colony of the oracle: ``run()`` iterations, then read the state."""

    def __init__(self, xy, params, instance=0, nn=None, w=None):
        self.xy = np.ascontiguousarray(xy, np.int32)
        self.n = int(self.xy.shape[0])
        self.params = params
        self._h = _vp()
        L = lib()
        if nn is None:
            rc = L.acsref_create(self.xy.reshape(-1), self.n, ctypes.byref(params),
                                 instance, ctypes.byref(self._h))
        else:
            nn = np.ascontiguousarray(nn, np.int32)
            w = np.ascontiguousarray(w, np.float32)
            rc = L.acsref_create_tables(self.xy.reshape(-1), self.n, nn.reshape(-1),
                                        w.reshape(-1), nn.shape[1], ctypes.byref(params),
                                        instance, ctypes.byref(self._h))
        if rc != 0:
            raise OracleError("acsref_create failed with status %d" % rc)
        self.m = params.m
        cl = _i32()
        tau0 = ctypes.c_float()
        lnn = _i64()
        self.cl = min(params.cl, self.n - 1) if nn is None else int(nn.shape[1])
        nnb = np.zeros((self.n, self.cl), np.int32)
        wb = np.zeros((self.n, self.cl), np.float32)
        L.acsref_get_setup(self._h, nnb, wb, ctypes.byref(tau0), ctypes.byref(lnn),
                           ctypes.byref(cl))
        self.nn, self.w = nnb, wb
        self.tau0 = np.float32(tau0.value)
        self.L_nn = int(lnn.value)

    def run(self, iters):
        rc = lib().acsref_run(self._h, iters)
        if rc != 0:
            raise OracleError("acsref_run failed with status %d" % rc)

    def local_step(self, frm, to):
        """Apply the local updates of one synchronous step (ant a took frm[a] -> to[a])."""
        rc = lib().acsref_local_step(self._h, np.ascontiguousarray(frm, np.int32),
                                     np.ascontiguousarray(to, np.int32))
        if rc != 0:
            raise OracleError("bad step")

    @property
    def iteration(self):
        return int(lib().acsref_iteration(self._h))

    def tours(self):
        t = np.zeros((self.m, self.n), np.int32)
        L = np.zeros(self.m, np.int64)
        lib().acsref_get_tours(self._h, t, L)
        return t, L

    def offer_best(self, tour):
        rc = lib().acsref_offer_best(self._h, np.ascontiguousarray(tour, np.int32))
        if rc != 0:
            raise OracleError("not a tour of this instance")

    def best(self):
        t = np.zeros(self.n, np.int32)
        L = _i64()
        rc = lib().acsref_best(self._h, t, ctypes.byref(L))
        if rc != 0:
            raise OracleError("no best tour yet")
        return t, int(L.value)

    def pheromone(self):
        """Matrix: (n, n) float32. SPM: (val (n,s) float32, idx (n,s), tail (n,))."""
        if self.params.memory == 0:
            tau = np.zeros((self.n, self.n), np.float32)
            lib().acsref_get_pheromone(self._h, tau, None, None)
            return tau
        s = self.params.spm_slots
        val = np.zeros((self.n, s), np.float32)
        idx = np.zeros((self.n, s), np.int32)
        tail = np.zeros(self.n, np.int32)
        lib().acsref_get_pheromone(self._h, val, idx.ctypes.data, tail.ctypes.data)
        return val, idx, tail

    def stats(self):
        """(fallback steps, selection steps, SPM hits, SPM misses)."""
        out = np.zeros(4, np.int64)
        lib().acsref_stats(self._h, out)
        return tuple(int(x) for x in out)

    def close(self):
        if self._h:
            lib().acsref_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
