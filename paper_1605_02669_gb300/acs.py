"""Thin ctypes binding of libacs (include/acs.h): argument marshalling only.

Every step of the colony runs in the CUDA library; there is no CPU path. If
libacs.so is missing or cannot be loaded, importing the library raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libacs.so")

ACS_OK, ACS_EINVAL, ACS_ENOMEM, ACS_ECUDA, ACS_ETIMEOUT, ACS_ESTATE = range(6)
ACS_MEM_MATRIX, ACS_MEM_SPM = 0, 1


class AcsError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, strerror(status), status))


class acs_params(ctypes.Structure):
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


ACS_FLAG_RELAXED = 1
ACS_FLAG_SPM_SKIP_DEFAULT = 2


def params(m=32, cl=32, beta=2, q0=0.9, rho=0.1, xi=0.1, memory=ACS_MEM_MATRIX,
           spm_slots=8, local_period=1, seed=1, relaxed=False, spm_skip_default=False):
    flags = (ACS_FLAG_RELAXED if relaxed else 0) | \
            (ACS_FLAG_SPM_SKIP_DEFAULT if spm_skip_default else 0)
    return acs_params(m, cl, beta, q0, rho, xi, memory, spm_slots, local_period, flags, seed)


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


def load():
    """Load libacs.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libacs.so not built at %s; run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    L.acs_create.argtypes = [_vp, _i32, P(acs_params), P(_vp)]
    L.acs_create_batch.argtypes = [_vp, _vp, _i32, P(acs_params), P(_vp)]
    L.acs_create_batch_ids.argtypes = [_vp, _vp, _vp, _i32, P(acs_params), P(_vp)]
    L.acs_state_size.argtypes = [_vp, _i32, _vp]
    L.acs_get_state.argtypes = [_vp, _i32, _vp, _i64]
    L.acs_set_state.argtypes = [_vp, _i32, _vp, _i64]
    L.acs_set_stream.argtypes = [_vp, _vp]
    L.acs_run_iterations.argtypes = [_vp, _i32]
    L.acs_best_tour.argtypes = [_vp, _i32, _vp, _vp]
    L.acs_get_tours.argtypes = [_vp, _i32, _vp, _vp]
    L.acs_get_pheromone.argtypes = [_vp, _i32, _vp, _vp, _vp]
    L.acs_get_setup.argtypes = [_vp, _i32, _vp, _vp, _vp, _vp, _vp]
    L.acs_get_stats.argtypes = [_vp, _i32, _vp]
    L.acs_iteration.argtypes = [_vp]
    L.acs_iteration.restype = _i64
    L.acs_num_instances.argtypes = [_vp]
    L.acs_num_instances.restype = _i32
    L.acs_instance_size.argtypes = [_vp, _i32]
    L.acs_instance_size.restype = _i32
    L.acs_last_launch_count.argtypes = [_vp]
    L.acs_last_launch_count.restype = _i64
    L.acs_strerror.argtypes = [ctypes.c_int]
    L.acs_strerror.restype = ctypes.c_char_p
    L.acs_destroy.argtypes = [_vp]
    L.acs_destroy.restype = None
    L.acs_iterate_noalloc.argtypes = [_vp, _i32, _vp, _vp, _i32, ctypes.c_float, _vp, _vp,
                                      _vp, _vp, _vp, _i64, P(acs_params), _vp]
    L.acs_set_threads_per_ant.argtypes = [_vp, _i32]
    L.acs_threads_per_ant.argtypes = [_vp]
    L.acs_threads_per_ant.restype = _i32
    L.acs_autotune.argtypes = [_vp, _i32, _vp, _vp]
    L.acs_autotune_group.argtypes = [_vp, _i32, _i32]
    L.acs_set_cluster_size.argtypes = [_vp, _i32]
    L.acs_cluster_size.argtypes = [_vp]
    L.acs_cluster_size.restype = _i32
    L.acs_offer_best_tour.argtypes = [_vp, _i32, _vp, _vp]
    L.acs_offer_best_tour.restype = ctypes.c_int
    L.acs_set_spm_resident.argtypes = [_vp, _i32]
    L.acs_set_spm_resident.restype = ctypes.c_int
    L.acs_kernel_mode.argtypes = [_vp]
    L.acs_kernel_mode.restype = _i32
    L.acs_prior_features.argtypes = [_vp, _i32, _vp, _vp]
    L.acs_prior_count_best_edges.argtypes = [_vp, _i32, _vp, _vp]
    L.acs_mlp_forward.argtypes = [_vp, _vp, _i64, _vp, _vp]
    L.acs_mlp_train_batch.argtypes = [_vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _vp, _vp, _vp]
    _f = ctypes.c_float
    L.acs_mlp_adam.argtypes = [_vp, _vp, _vp, _vp, _i32, _f, _f, _f, _f, _vp]
    L.acs_apply_prior.argtypes = [_vp, _i32, _vp, _i32, _vp]
    L.acs_set_candidates.argtypes = [_vp, _i32, _vp, _vp, _i32]
    L.acs_mlp_sync.argtypes = [_vp]
    L.acs_mlp_test_wait_hook.argtypes = [_i64, _i32]
    for name in ["acs_prior_features", "acs_prior_count_best_edges", "acs_mlp_forward",
                 "acs_mlp_train_batch", "acs_mlp_adam", "acs_apply_prior", "acs_set_candidates",
                 "acs_mlp_sync", "acs_mlp_test_wait_hook"]:
        getattr(L, name).restype = ctypes.c_int
    for name in ["acs_create_batch_ids", "acs_state_size", "acs_get_state", "acs_set_state",
                 "acs_autotune_group"]:
        getattr(L, name).restype = ctypes.c_int
    for name in ["acs_set_threads_per_ant", "acs_autotune", "acs_set_cluster_size", "acs_iterate_noalloc", "acs_create", "acs_create_batch", "acs_set_stream", "acs_run_iterations",
                 "acs_best_tour", "acs_get_tours", "acs_get_pheromone", "acs_get_setup",
                 "acs_get_stats"]:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def strerror(status):
    try:
        return load().acs_strerror(status).decode()
    except ImportError:
        return "status %d" % status


def _check(rc, what):
    if rc != ACS_OK:
        raise AcsError(rc, what)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_vp)


# ---- the C ABI under the same names -------------------------------------------------

def acs_create(coords, p):
    coords = np.ascontiguousarray(coords, np.int32)
    h = _vp()
    _check(load().acs_create(_ptr(coords), coords.shape[0], ctypes.byref(p), ctypes.byref(h)),
           "acs_create")
    return h


def acs_create_batch(coords, offsets, p):
    coords = np.ascontiguousarray(coords, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    h = _vp()
    _check(load().acs_create_batch(_ptr(coords), _ptr(offsets), offsets.shape[0] - 1,
                                   ctypes.byref(p), ctypes.byref(h)), "acs_create_batch")
    return h


def acs_create_batch_ids(coords, offsets, instance_ids, p):
    coords = np.ascontiguousarray(coords, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = None if instance_ids is None else np.ascontiguousarray(instance_ids, np.int32)
    h = _vp()
    _check(load().acs_create_batch_ids(_ptr(coords), _ptr(offsets), _ptr(ids),
                                       offsets.shape[0] - 1, ctypes.byref(p), ctypes.byref(h)),
           "acs_create_batch_ids")
    return h


def acs_state_size(ctx, instance):
    b = np.zeros(1, np.int64)
    _check(load().acs_state_size(ctx, instance, _ptr(b)), "acs_state_size")
    return int(b[0])


def acs_get_state(ctx, instance):
    """The instance's loop state as an opaque byte image (numpy uint8)."""
    buf = np.zeros(acs_state_size(ctx, instance), np.uint8)
    _check(load().acs_get_state(ctx, instance, _ptr(buf), buf.nbytes), "acs_get_state")
    return buf


def acs_set_state(ctx, instance, buf):
    buf = np.ascontiguousarray(buf, np.uint8)
    _check(load().acs_set_state(ctx, instance, _ptr(buf), buf.nbytes), "acs_set_state")


def acs_set_stream(ctx, stream_handle):
    _check(load().acs_set_stream(ctx, _vp(stream_handle or 0)), "acs_set_stream")


def acs_run_iterations(ctx, iters):
    _check(load().acs_run_iterations(ctx, int(iters)), "acs_run_iterations")


def acs_best_tour(ctx, instance, n):
    t = np.zeros(n, np.int32)
    L = np.zeros(1, np.int64)
    _check(load().acs_best_tour(ctx, instance, _ptr(t), _ptr(L)), "acs_best_tour")
    return t, int(L[0])


def acs_offer_best_tour(ctx, instance, tour):
    tour = np.ascontiguousarray(tour, np.int32)
    L = np.zeros(1, np.int64)
    _check(load().acs_offer_best_tour(ctx, instance, _ptr(tour), _ptr(L)), "acs_offer_best_tour")
    return int(L[0])


def acs_get_tours(ctx, instance, m, n):
    t = np.zeros((m, n), np.int32)
    L = np.zeros(m, np.int64)
    _check(load().acs_get_tours(ctx, instance, _ptr(t), _ptr(L)), "acs_get_tours")
    return t, L


def acs_get_pheromone(ctx, instance, n, memory, s=0):
    if memory == ACS_MEM_MATRIX:
        tau = np.zeros((n, n), np.float32)
        _check(load().acs_get_pheromone(ctx, instance, _ptr(tau), None, None), "acs_get_pheromone")
        return tau
    val = np.zeros((n, s), np.float32)
    idx = np.zeros((n, s), np.int32)
    tail = np.zeros(n, np.int32)
    _check(load().acs_get_pheromone(ctx, instance, _ptr(val), _ptr(idx), _ptr(tail)),
           "acs_get_pheromone")
    return val, idx, tail


def acs_get_setup(ctx, instance, n, cl_max):
    cl = np.zeros(1, np.int32)
    tau0 = np.zeros(1, np.float32)
    lnn = np.zeros(1, np.int64)
    _check(load().acs_get_setup(ctx, instance, None, None, _ptr(tau0), _ptr(lnn), _ptr(cl)),
           "acs_get_setup")
    c = int(cl[0])
    nn = np.zeros((n, c), np.int32)
    w = np.zeros((n, c), np.float32)
    _check(load().acs_get_setup(ctx, instance, _ptr(nn), _ptr(w), None, None, None),
           "acs_get_setup")
    return nn, w, np.float32(tau0[0]), int(lnn[0])


def acs_get_stats(ctx, instance):
    out = np.zeros(4, np.int64)
    _check(load().acs_get_stats(ctx, instance, _ptr(out)), "acs_get_stats")
    return tuple(int(x) for x in out)


def acs_iteration(ctx):
    return int(load().acs_iteration(ctx))


def acs_num_instances(ctx):
    return int(load().acs_num_instances(ctx))


def acs_instance_size(ctx, instance):
    return int(load().acs_instance_size(ctx, instance))


def acs_last_launch_count(ctx):
    return int(load().acs_last_launch_count(ctx))


def acs_set_threads_per_ant(ctx, tpa):
    _check(load().acs_set_threads_per_ant(ctx, int(tpa)), "acs_set_threads_per_ant")


def acs_threads_per_ant(ctx):
    return int(load().acs_threads_per_ant(ctx))


def acs_set_cluster_size(ctx, csize):
    _check(load().acs_set_cluster_size(ctx, int(csize)), "acs_set_cluster_size")


def acs_cluster_size(ctx):
    return int(load().acs_cluster_size(ctx))


def acs_set_spm_resident(ctx, resident):
    _check(load().acs_set_spm_resident(ctx, int(resident)), "acs_set_spm_resident")


def acs_kernel_mode(ctx):
    return int(load().acs_kernel_mode(ctx))


def acs_autotune(ctx, trial_iters):
    tpa = np.zeros(1, np.int32)
    cs = np.zeros(1, np.int32)
    _check(load().acs_autotune(ctx, int(trial_iters), _ptr(tpa), _ptr(cs)), "acs_autotune")
    return int(tpa[0]), int(cs[0])


def acs_autotune_group(ctxs, trial_iters):
    arr = (_vp * len(ctxs))(*ctxs)
    _check(load().acs_autotune_group(arr, len(ctxs), int(trial_iters)), "acs_autotune_group")


def autotune_group(colonies, trial_iters=2):
    """Tune the launch shapes of colonies that run concurrently on their own
    streams (acs_autotune_group)."""
    acs_autotune_group([c.ctx for c in colonies], trial_iters)


def acs_iterate_noalloc(dev_coords, n, dev_nn32, dev_w32, cl, tau0, dev_tau, dev_tours,
                        dev_lens, dev_best, dev_best_len, iteration, p, stream=0):
    """One iteration on caller-owned device buffers (addresses as ints); no allocation."""
    return int(load().acs_iterate_noalloc(_vp(dev_coords), int(n), _vp(dev_nn32), _vp(dev_w32),
                                          int(cl), float(tau0), _vp(dev_tau), _vp(dev_tours),
                                          _vp(dev_lens), _vp(dev_best), _vp(dev_best_len),
                                          int(iteration), ctypes.byref(p), _vp(stream or 0)))


# ---- learned prior (include/acs_prior.h); device buffers are torch tensors or raw
# device addresses, streams torch streams, raw handles or None (legacy default)

ACS_MLP_FEATURES, ACS_MLP_HIDDEN, ACS_MLP_PARAMS = 8, 64, 4801


def _dev(t):
    if t is None:
        return None
    return _vp(t if isinstance(t, int) else t.data_ptr())


def _strm(s):
    if s is None:
        return None
    return _vp(s if isinstance(s, int) else s.cuda_stream)


def acs_prior_features(ctx, instance, dev_feat, stream=None):
    _check(load().acs_prior_features(ctx, instance, _dev(dev_feat), _strm(stream)),
           "acs_prior_features")


def acs_prior_count_best_edges(ctx, instance, dev_count, stream=None):
    _check(load().acs_prior_count_best_edges(ctx, instance, _dev(dev_count), _strm(stream)),
           "acs_prior_count_best_edges")


def acs_mlp_forward(dev_params, dev_feat, rows, dev_p, stream=None):
    _check(load().acs_mlp_forward(_dev(dev_params), _dev(dev_feat), rows, _dev(dev_p),
                                  _strm(stream)), "acs_mlp_forward")


def acs_mlp_train_batch(dev_params, dev_feat, dev_label, total, first, batch, perm_a, perm_c,
                        dev_grad, dev_loss, stream=None):
    _check(load().acs_mlp_train_batch(_dev(dev_params), _dev(dev_feat), _dev(dev_label), total,
                                      first, batch, perm_a, perm_c, _dev(dev_grad),
                                      _dev(dev_loss), _strm(stream)), "acs_mlp_train_batch")


def acs_mlp_adam(dev_params, dev_grad, dev_m, dev_v, step, lr=1e-3, beta1=0.9, beta2=0.999,
                 eps=1e-8, stream=None):
    _check(load().acs_mlp_adam(_dev(dev_params), _dev(dev_grad), _dev(dev_m), _dev(dev_v), step,
                               lr, beta1, beta2, eps, _strm(stream)), "acs_mlp_adam")


def acs_mlp_sync(stream=None):
    _check(load().acs_mlp_sync(_strm(stream)), "acs_mlp_sync")


def acs_apply_prior(ctx, instance, dev_p, keep, stream=None):
    _check(load().acs_apply_prior(ctx, instance, _dev(dev_p), keep, _strm(stream)),
           "acs_apply_prior")


def acs_set_candidates(ctx, instance, nn, w):
    nn = np.ascontiguousarray(nn, np.int32)
    w = np.ascontiguousarray(w, np.float32)
    assert nn.shape == w.shape and nn.ndim == 2
    _check(load().acs_set_candidates(ctx, instance, _ptr(nn), _ptr(w), nn.shape[1]),
           "acs_set_candidates")


def acs_destroy(ctx):
    if ctx:
        load().acs_destroy(ctx)


# ---- convenience wrapper ---------------------------------------------------------

class Colony:
    """One context (one instance, or a batch) with numpy in/out."""

    def __init__(self, coords, p, offsets=None, instance_ids=None):
        self.p = p
        coords = np.ascontiguousarray(coords, np.int32)
        if offsets is None and instance_ids is None:
            self.ctx = acs_create(coords, p)
            self.sizes = [coords.shape[0]]
        else:
            if offsets is None:
                offsets = np.array([0, coords.shape[0]], np.int64)
            self.ctx = acs_create_batch_ids(coords, offsets, instance_ids, p)
            off = np.asarray(offsets, np.int64)
            self.sizes = [int(x) for x in np.diff(off)]

    def run(self, iters):
        acs_run_iterations(self.ctx, iters)

    def set_threads_per_ant(self, tpa):
        acs_set_threads_per_ant(self.ctx, tpa)

    def set_cluster_size(self, csize):
        acs_set_cluster_size(self.ctx, csize)

    @property
    def cluster_size(self):
        return acs_cluster_size(self.ctx)

    def set_spm_resident(self, resident):
        acs_set_spm_resident(self.ctx, resident)

    @property
    def kernel_mode(self):
        return acs_kernel_mode(self.ctx)

    @property
    def threads_per_ant(self):
        return acs_threads_per_ant(self.ctx)

    def autotune(self, trial_iters=2):
        return acs_autotune(self.ctx, trial_iters)

    def set_stream(self, handle):
        acs_set_stream(self.ctx, handle)

    @property
    def iteration(self):
        return acs_iteration(self.ctx)

    def offer_best(self, tour, b=0):
        return acs_offer_best_tour(self.ctx, b, tour)

    def best(self, b=0):
        return acs_best_tour(self.ctx, b, self.sizes[b])

    def tours(self, b=0):
        return acs_get_tours(self.ctx, b, self.p.m, self.sizes[b])

    def pheromone(self, b=0):
        return acs_get_pheromone(self.ctx, b, self.sizes[b], self.p.memory, self.p.spm_slots)

    def setup(self, b=0):
        return acs_get_setup(self.ctx, b, self.sizes[b], 32)

    def stats(self, b=0):
        return acs_get_stats(self.ctx, b)

    def get_state(self, b=0):
        return acs_get_state(self.ctx, b)

    def set_state(self, buf, b=0):
        acs_set_state(self.ctx, b, buf)

    def close(self):
        if self.ctx:
            acs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
