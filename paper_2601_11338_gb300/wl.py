"""Thin ctypes binding of libwl.so (include/wl.h), same names as the C ABI.

Argument marshalling only: every computation runs in the CUDA library. Array
arguments may be numpy arrays (host) or torch tensors (host or CUDA); they
are passed as raw pointers. The library must be built (see `build.py`); if
it is missing or fails to load, every call raises - there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

WL_OK = 0
WL_ERR_INVALID_ARG = -1
WL_ERR_NOT_SYMMETRIC = -2
WL_ERR_SELF_LOOP = -3
WL_ERR_UNSORTED = -4
WL_ERR_ALPHA_RANGE = -5
WL_ERR_NOT_SPD = -6
WL_ERR_NONFINITE = -7
WL_ERR_NO_CONVERGENCE = -8
WL_ERR_TIMEOUT = -9
WL_ERR_OOM = -10
WL_ERR_CUDA = -11
WL_ERR_UNSUPPORTED = -12

WL_ALLWALK, WL_NBT, WL_BTDW = 0, 1, 2
WL_F_RESOLVENT, WL_F_EXP, WL_F_IDENTITY = 0, 1, 2
WL_FP64, WL_REFINED, WL_SKETCH = 0, 1, 2


class wl_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p)]


class wl_params(ctypes.Structure):
    _fields_ = [("f", ctypes.c_int), ("alpha", ctypes.c_double), ("alpha_rel", ctypes.c_double),
                ("beta", ctypes.c_double), ("mu", ctypes.c_double), ("prec", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("outer_tol", ctypes.c_double), ("stream", ctypes.c_void_p), ("reorder", ctypes.c_int),
                ("reorth", ctypes.c_int), ("shift", ctypes.c_double), ("gram", ctypes.c_int)]


class wl_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("refinements", ctypes.c_int), ("rel_res", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("nnz_rhs_iters", ctypes.c_double), ("bytes_alg", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("mu", ctypes.c_double),
                ("rho", ctypes.c_double), ("lambda_max", ctypes.c_double), ("launches", ctypes.c_int),
                ("k_cg_launches", ctypes.c_int), ("k_cg_iters", ctypes.c_int), ("k_cg_ms", ctypes.c_double),
                ("k_cg_bytes", ctypes.c_double), ("k_res_launches", ctypes.c_int), ("k_res_ms", ctypes.c_double),
                ("k_lan_launches", ctypes.c_int), ("k_lan_ms", ctypes.c_double), ("reorth_blocks", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class WLError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status}) {last_error()}")


_lib = None
LIB_PATH = _build.LIB


def lib():
    """Load libwl.so (building it first if its sources are newer)."""
    global _lib
    if _lib is None:
        if _build.needs_build():
            _build.build()
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.wl_build.argtypes = [ctypes.POINTER(wl_csr), c_int, ctypes.POINTER(wl_params),
                               ctypes.POINTER(vp), ctypes.POINTER(wl_stats)]
        L.wl_set_params.argtypes = [vp, ctypes.POINTER(wl_params)]
        L.wl_degrees.argtypes = [vp, vp, ctypes.POINTER(wl_stats)]
        L.wl_apply.argtypes = [vp, vp, i64, c_int, vp, i64, ctypes.POINTER(wl_stats)]
        L.wl_expmv.argtypes = [vp, vp, i64, c_int, vp, c_int, vp, i64, ctypes.POINTER(wl_stats)]
        L.wl_trace.argtypes = [vp, c_int, ctypes.c_uint64, vp, vp, vp, ctypes.POINTER(wl_stats)]
        L.wl_markov.argtypes = [vp, vp, i64, c_int, vp, c_int, vp, i64, ctypes.POINTER(wl_stats)]
        L.wl_return_prob.argtypes = [vp, c_int, ctypes.c_uint64, vp, c_int, vp, vp, ctypes.POINTER(wl_stats)]
        L.wl_set_warm_start.argtypes = [vp, vp]
        L.wl_get_info.argtypes = [vp, ctypes.POINTER(wl_stats)]
        L.wl_destroy.argtypes = [vp]
        L.wl_destroy.restype = None
        L.wl_status_string.argtypes = [c_int]
        L.wl_status_string.restype = ctypes.c_char_p
        L.wl_last_error.restype = ctypes.c_char_p
        L.wl_degrees_noalloc.argtypes = [ctypes.POINTER(wl_csr), c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, c_int, vp, vp, ctypes.POINTER(wl_stats)]
        L.wl_degrees_noalloc.restype = c_int
        L.wl_rcm_order.argtypes = [vp, vp, i64, vp]
        L.wl_rcm_order.restype = c_int
        L.wl_selftest_bounded_wait.argtypes = [c_int, vp]
        L.wl_selftest_bounded_wait.restype = c_int
        L.wl_batch_build.argtypes = [vp, c_int, vp, c_int, ctypes.POINTER(wl_params), ctypes.POINTER(vp),
                                     ctypes.POINTER(wl_stats)]
        L.wl_batch_build.restype = c_int
        L.wl_batch_run.argtypes = [vp, vp, c_int, vp, vp, c_int, ctypes.POINTER(wl_stats)]
        L.wl_batch_run.restype = c_int
        dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(c_int)
        L.wl_batch_info.argtypes = [vp, c_int, c_int, dp, dp, dp, ip, ip, ip]
        L.wl_batch_info.restype = c_int
        L.wl_batch_tile_rows.argtypes = [vp, c_int]
        L.wl_batch_tile_rows.restype = c_int
        L.wl_mlp_save.argtypes = [ctypes.c_char_p, vp]
        L.wl_mlp_save.restype = c_int
        L.wl_mlp_load.argtypes = [ctypes.c_char_p, vp]
        L.wl_mlp_load.restype = c_int
        L.wl_mlp_param_count.restype = c_int
        L.wl_mlp_param_count.argtypes = []
        L.wl_mlp_features.argtypes = [vp, vp, vp, ctypes.POINTER(wl_stats)]
        L.wl_mlp_train.argtypes = [vp, vp, vp, i64, c_int, i64, ctypes.c_float, c_int,
                                   ctypes.POINTER(ctypes.c_double), vp]
        L.wl_mlp_loss_grad.argtypes = [vp, vp, vp, i64, ctypes.POINTER(ctypes.c_double), vp, vp]
        L.wl_mlp_predict.argtypes = [vp, vp, i64, vp, vp, vp]
        L.wl_mlp_targets.argtypes = [vp, vp, i64, vp, vp]
        L.wl_mlp_warm_start.argtypes = [vp, vp, ctypes.POINTER(wl_stats)]
        for name in ("wl_mlp_features", "wl_mlp_train", "wl_mlp_loss_grad", "wl_mlp_predict", "wl_mlp_targets",
                     "wl_mlp_warm_start"):
            getattr(L, name).restype = c_int
        L.wl_sketch_gram.argtypes = [vp, vp, i64, c_int, c_int, c_int, vp, vp]
        L.wl_sketch_gram.restype = c_int
        L.wl_pool_release.argtypes = []
        L.wl_pool_release.restype = None
        L.wl_pool_cached_bytes.argtypes = []
        L.wl_pool_cached_bytes.restype = ctypes.c_size_t
        L.wl_batch_destroy.argtypes = [vp]
        L.wl_batch_destroy.restype = None
        for name in ("wl_build", "wl_set_params", "wl_degrees", "wl_apply", "wl_expmv", "wl_trace",
                     "wl_markov", "wl_return_prob", "wl_set_warm_start", "wl_get_info"):
            getattr(L, name).restype = c_int
        _lib = L
    return _lib


def status_string(s):
    return lib().wl_status_string(int(s)).decode()


def last_error():
    return lib().wl_last_error().decode()


def _ptr(a):
    """Raw address of a numpy array or torch tensor (no copy)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def make_params(f=WL_F_RESOLVENT, alpha=0.0, alpha_rel=0.0, beta=0.0, mu=0.0, prec=WL_FP64, tol=0.0,
                max_iter=0, max_outer=0, outer_tol=0.0, stream=None, reorder=1, reorth=0, shift=0.0, gram=0):
    return wl_params(f, alpha, alpha_rel, beta, mu, prec, tol, max_iter, max_outer, outer_tol, stream, reorder,
                     reorth, shift, gram)


class Handle:
    """Owns a wl_handle*; keeps references to nothing else (the library copies the graph)."""

    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "ptr", None):
            lib().wl_destroy(self.ptr)
            self.ptr = None


def _check(rc, where, allow=()):
    if rc != WL_OK and rc not in allow:
        raise WLError(rc, where)
    return rc


def wl_build(row_ptr, col_idx, n, nnz, variant, params, stats=None):
    A = wl_csr(n, nnz, _ptr(row_ptr), _ptr(col_idx))
    h = ctypes.c_void_p()
    st = stats if stats is not None else wl_stats()
    _check(lib().wl_build(ctypes.byref(A), variant, ctypes.byref(params), ctypes.byref(h), ctypes.byref(st)),
           "wl_build")
    return Handle(h)


def wl_set_params(h, params):
    _check(lib().wl_set_params(h.ptr, ctypes.byref(params)), "wl_set_params")


def wl_degrees(h, Df, stats=None, allow=()):
    st = stats if stats is not None else wl_stats()
    return _check(lib().wl_degrees(h.ptr, _ptr(Df), ctypes.byref(st)), "wl_degrees", allow)


def wl_apply(h, V, ldv, k, W, ldw, stats=None, allow=()):
    st = stats if stats is not None else wl_stats()
    return _check(lib().wl_apply(h.ptr, _ptr(V), ldv, k, _ptr(W), ldw, ctypes.byref(st)), "wl_apply", allow)


def wl_expmv(h, U0, ldu, k, taus, U, ldo, stats=None, allow=()):
    st = stats if stats is not None else wl_stats()
    taus = np.ascontiguousarray(taus, dtype=np.float64)
    return _check(lib().wl_expmv(h.ptr, _ptr(U0), ldu, k, taus.ctypes.data, len(taus), _ptr(U), ldo,
                                 ctypes.byref(st)), "wl_expmv", allow)


def wl_markov(h, P0, ldp, k, steps, out, ldo, stats=None, allow=()):
    st = stats if stats is not None else wl_stats()
    steps = np.ascontiguousarray(steps, dtype=np.int32)
    return _check(lib().wl_markov(h.ptr, _ptr(P0), ldp, k, steps.ctypes.data, len(steps), _ptr(out), ldo,
                                  ctypes.byref(st)), "wl_markov", allow)


def wl_return_prob(h, M, seed, ts, stats=None, allow=()):
    """Average return probability estimates (p(t), error estimate) for each t."""
    st = stats if stats is not None else wl_stats()
    ts = np.ascontiguousarray(ts, dtype=np.float64)
    p = np.zeros(len(ts))
    e = np.zeros(len(ts))
    _check(lib().wl_return_prob(h.ptr, M, seed, ts.ctypes.data, len(ts), p.ctypes.data, e.ctypes.data,
                                ctypes.byref(st)), "wl_return_prob", allow)
    return p, e


def wl_trace(h, M, seed, omega_out=None, stats=None):
    st = stats if stats is not None else wl_stats()
    est = ctypes.c_double()
    err = ctypes.c_double()
    _check(lib().wl_trace(h.ptr, M, seed, ctypes.byref(est), ctypes.byref(err), _ptr(omega_out),
                          ctypes.byref(st)), "wl_trace")
    return est.value, err.value


def wl_degrees_noalloc(row_ptr, col_idx, n, nnz, variant, mu, alpha, Df, tol=0.0, max_iter=0, stream=None,
                       stats=None, allow=()):
    """Walk degrees without any GPU allocation by the library (device CSR and
    output; at most 262144 nodes). See include/wl.h."""
    A = wl_csr(n, nnz, _ptr(row_ptr), _ptr(col_idx))
    st = stats if stats is not None else wl_stats()
    return _check(lib().wl_degrees_noalloc(ctypes.byref(A), variant, mu, alpha, tol, max_iter, _ptr(Df), stream,
                                           ctypes.byref(st)), "wl_degrees_noalloc", allow)


def wl_rcm_order(row_ptr, col_idx, n):
    """Reverse Cuthill-McKee order perm[new] = old of a host CSR (int32 arrays).
    See include/wl.h."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    perm = np.empty(max(int(n), 0), dtype=np.int32)
    _check(lib().wl_rcm_order(_ptr(rp), _ptr(ci) if ci.size else None, int(n), _ptr(perm)), "wl_rcm_order")
    return perm


def wl_selftest_bounded_wait(missing, stream=None):
    """Status of one CTA in the bounded grid barrier expecting 1 + missing CTAs:
    WL_OK when missing = 0, WL_ERR_TIMEOUT after the wait limit otherwise
    (the kernel returns; the context stays usable). See include/wl.h."""
    return lib().wl_selftest_bounded_wait(int(missing), stream)


def wl_set_warm_start(h, x0):
    _check(lib().wl_set_warm_start(h.ptr, _ptr(x0)), "wl_set_warm_start")


def wl_get_info(h):
    st = wl_stats()
    _check(lib().wl_get_info(h.ptr, ctypes.byref(st)), "wl_get_info")
    return st


class BatchHandle:
    """Owns a wl_batch*."""

    def __init__(self, ptr, ngraph, nmu):
        self.ptr = ptr
        self.ngraph = ngraph
        self.nmu = nmu

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "ptr", None):
            lib().wl_batch_destroy(self.ptr)
            self.ptr = None


def wl_batch_build(graphs, mus, params, stats=None):
    """graphs: list of (row_ptr, col_idx, n, nnz) with host or device arrays."""
    arr = (wl_csr * len(graphs))(*[wl_csr(n, nnz, _ptr(rp), _ptr(ci)) for rp, ci, n, nnz in graphs])
    m = np.ascontiguousarray(np.asarray(mus, dtype=np.float64))
    h = ctypes.c_void_p()
    st = stats if stats is not None else wl_stats()
    _check(lib().wl_batch_build(ctypes.cast(arr, ctypes.c_void_p), len(graphs), m.ctypes.data, len(m),
                                ctypes.byref(params), ctypes.byref(h), ctypes.byref(st)), "wl_batch_build")
    return BatchHandle(h, len(graphs), len(m))


def wl_batch_run(b, V, k, Df, W, stepped=0, stats=None, allow=()):
    st = stats if stats is not None else wl_stats()
    return _check(lib().wl_batch_run(b.ptr, _ptr(V), k, _ptr(Df), _ptr(W), int(stepped), ctypes.byref(st)),
                  "wl_batch_run", allow)


def wl_batch_info(b, graph, mu_index):
    a, r, lm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    i1, i2, stt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().wl_batch_info(b.ptr, graph, mu_index, ctypes.byref(a), ctypes.byref(r), ctypes.byref(lm),
                               ctypes.byref(i1), ctypes.byref(i2), ctypes.byref(stt)), "wl_batch_info")
    return {"alpha": a.value, "rho": r.value, "lambda_max": lm.value, "iters_df": i1.value, "iters_v": i2.value,
            "status": stt.value}


def wl_batch_tile_rows(b, k):
    return lib().wl_batch_tile_rows(b.ptr, k)


# ------------------------------------------------------------ learned warm start
def wl_mlp_param_count():
    return lib().wl_mlp_param_count()


def wl_mlp_features(h, feats=None, xan=None, stats=None):
    st = stats if stats is not None else wl_stats()
    _check(lib().wl_mlp_features(h.ptr, _ptr(feats), _ptr(xan), ctypes.byref(st)), "wl_mlp_features")


def wl_mlp_train(params, feats, target, rows, steps, batch=0, lr=1e-3, standardize=1, stream=None):
    loss = ctypes.c_double()
    _check(lib().wl_mlp_train(_ptr(params), _ptr(feats), _ptr(target), rows, steps, batch, lr, standardize,
                              ctypes.byref(loss), stream), "wl_mlp_train")
    return loss.value


def wl_mlp_loss_grad(params, feats, target, rows, grad, stream=None):
    loss = ctypes.c_double()
    _check(lib().wl_mlp_loss_grad(_ptr(params), _ptr(feats), _ptr(target), rows, ctypes.byref(loss), _ptr(grad),
                                  stream), "wl_mlp_loss_grad")
    return loss.value


def wl_mlp_predict(params, feats, rows, xan, out, stream=None):
    _check(lib().wl_mlp_predict(_ptr(params), _ptr(feats), rows, _ptr(xan), _ptr(out), stream), "wl_mlp_predict")


def wl_mlp_targets(Df, xan, rows, target, stream=None):
    _check(lib().wl_mlp_targets(_ptr(Df), _ptr(xan), rows, _ptr(target), stream), "wl_mlp_targets")


def wl_mlp_warm_start(h, params, stats=None):
    st = stats if stats is not None else wl_stats()
    _check(lib().wl_mlp_warm_start(h.ptr, _ptr(params), ctypes.byref(st)), "wl_mlp_warm_start")
    return st


def wl_sketch_gram(omega, Y, n, M, ldy, tensor_cores, out, stream=None):
    """[Omega Y]^T Y (128 x 64 FP64) from device arrays; see include/wl.h."""
    return _check(lib().wl_sketch_gram(_ptr(omega), _ptr(Y), n, M, ldy, int(tensor_cores), _ptr(out), stream),
                  "wl_sketch_gram")


def wl_pool_release():
    lib().wl_pool_release()


def wl_pool_cached_bytes():
    return int(lib().wl_pool_cached_bytes())



def wl_mlp_save(path, params):
    """Write the network's parameter vector (host float32 array) to a checkpoint file."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    return _check(lib().wl_mlp_save(os.fsencode(path), p.ctypes.data), "wl_mlp_save")


def wl_mlp_load(path, allow=()):
    """Parameter vector (float32) read from a checkpoint file. A rejected file
    raises WLError, or returns None when its status is in `allow`."""
    p = np.empty(wl_mlp_param_count(), dtype=np.float32)
    rc = _check(lib().wl_mlp_load(os.fsencode(path), p.ctypes.data), "wl_mlp_load", allow)
    return p if rc == WL_OK else None
