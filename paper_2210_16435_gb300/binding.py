"""ctypes binding of libsfairsc.so: the C entry points under the same names.

This module only marshals arguments (pointers, sizes, enums); every step of
the computation runs inside the CUDA library.  Importing it does not load the
library; the first call does, and raises if the library is missing — there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

from . import buildlib as _build

SFAIRSC_F64, SFAIRSC_F32, SFAIRSC_BF16 = 0, 1, 2
SFAIRSC_PREC_FP64, SFAIRSC_PREC_MIXED = 0, 1
STATUS = {
    0: "OK", -1: "INVALID_ARG", -2: "BAD_CSR", -3: "ISOLATED_VERTEX", -4: "EMPTY_GROUP", -5: "K_TOO_LARGE",
    -6: "NONFINITE", -7: "NOT_CONVERGED", -8: "SHIFT", -9: "CUDA", -10: "OOM", -11: "DEVICE_TIMEOUT",
    -12: "UNSUPPORTED", -13: "BREAKDOWN",
}


class Opts(ctypes.Structure):
    _fields_ = [
        ("sigma", ctypes.c_double), ("tol", ctypes.c_double), ("max_restarts", ctypes.c_int32),
        ("basis", ctypes.c_int32), ("prec", ctypes.c_int32), ("block", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("kmeans_seed", ctypes.c_uint64), ("kmeans_n_init", ctypes.c_int32),
        ("kmeans_max_iter", ctypes.c_int32), ("validate", ctypes.c_int32), ("profile", ctypes.c_int32),
        ("wait_limit_us", ctypes.c_int32), ("fault_inject", ctypes.c_int32), ("spmv_window", ctypes.c_int32),
        ("orth_mode", ctypes.c_int32), ("restart_mode", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("restarts", ctypes.c_int32), ("matvecs", ctypes.c_int32),
        ("kmeans_iters", ctypes.c_int32), ("sigma", ctypes.c_double), ("max_resid", ctypes.c_double),
        ("fairness_err", ctypes.c_double), ("dorth_err", ctypes.c_double), ("kmeans_inertia", ctypes.c_double),
        ("ms_setup", ctypes.c_float), ("ms_solve", ctypes.c_float), ("ms_kmeans", ctypes.c_float),
        ("ms_total", ctypes.c_float), ("ms_operator", ctypes.c_float), ("ms_orth", ctypes.c_float),
        ("n_operator", ctypes.c_int32), ("n_orth", ctypes.c_int32), ("n_launches", ctypes.c_int32),
        ("orth_cols", ctypes.c_int32), ("basis", ctypes.c_int32), ("block", ctypes.c_int32),
        ("orth_sweeps", ctypes.c_int32), ("ms_restart", ctypes.c_float), ("ms_host_eig", ctypes.c_float),
        ("ms_final", ctypes.c_float), ("host_eig_fallbacks", ctypes.c_int32), ("spmv_segments", ctypes.c_int32),
        ("spmv_windowed", ctypes.c_int32), ("spmv_in_window", ctypes.c_float), ("restarts_tc", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 3),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class BatchGraph(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
        ("values", ctypes.c_void_p), ("group_labels", ctypes.c_void_p), ("h", ctypes.c_int32), ("k", ctypes.c_int32),
        ("eigenvalues", ctypes.c_void_p), ("H", ctypes.c_void_p),
    ]


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("converged", ctypes.c_int32), ("breakdowns", ctypes.c_int32),
        ("grid", ctypes.c_int32), ("restarts", ctypes.c_int64), ("matvecs", ctypes.c_int64),
        ("max_resid", ctypes.c_double), ("split", ctypes.c_double), ("ms_solve", ctypes.c_float),
        ("ms_autotune", ctypes.c_float), ("ctas_per_sm", ctypes.c_int32), ("max_team", ctypes.c_int32),
        ("autotuned", ctypes.c_int32), ("cuda_graph", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
        ("teams", ctypes.c_int32 * 5), ("reserved", ctypes.c_int32 * 6),
    ]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("reserved", "teams")}
        d["teams"] = list(self.teams)
        return d


class SFairSCError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({status}) {detail}".rstrip())


_lib = None


def library_path() -> str:
    return _build.library_path()


def load(path: str | None = None):
    """Load libsfairsc.so once.  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError(f"libsfairsc.so not built at {p}; run paper_2210_16435_gb300.buildlib.build() "
                           "(the CUDA library is required: there is no CPU fallback)")
    lib = ctypes.CDLL(p)
    vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    lib.sfairsc_strerror.restype = ctypes.c_char_p
    lib.sfairsc_strerror.argtypes = [ctypes.c_int]
    lib.sfairsc_last_error.restype = ctypes.c_char_p
    lib.sfairsc_last_error.argtypes = []
    lib.sfairsc_opts_default.argtypes = [ctypes.POINTER(Opts)]
    lib.sfairsc_create.argtypes = [ctypes.POINTER(vp), i64, i64, vp, vp, vp, i32, vp, i32, i32, i32,
                                   ctypes.POINTER(Opts), vp]
    lib.sfairsc_create_dense.argtypes = [ctypes.POINTER(vp), i64, i64, vp, vp, vp, i32, vp, i32, i32, i32,
                                         ctypes.POINTER(Opts), vp]
    lib.sfairsc_destroy.argtypes = [vp]
    lib.sfairsc_get_sigma.argtypes = [vp, ctypes.POINTER(dbl)]
    lib.sfairsc_apply_operator.argtypes = [vp, vp, vp, i32]
    lib.sfairsc_solve.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Info)]
    lib.sfairsc_kmeans.argtypes = [i64, i32, vp, i32, u64, i32, i32, vp, vp, vp, vp, vp]
    lib.sfairsc_backward.argtypes = [vp, vp, vp, dbl, vp]
    lib.sfairsc_backward_vectors.argtypes = [vp, vp, vp, vp, dbl, vp, i32, dbl, ctypes.POINTER(i32),
                                             ctypes.POINTER(dbl)]
    lib.sfairsc_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(BatchGraph), ctypes.POINTER(Opts),
                                         vp]
    lib.sfairsc_batch_autotune.argtypes = [vp]
    lib.sfairsc_batch_schedule.argtypes = [vp, i32, i32, dbl]
    lib.sfairsc_batch_solve.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(BatchInfo)]
    lib.sfairsc_batch_destroy.argtypes = [vp]
    lib.sfairsc_batch_stats.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(dbl)]
    lib.sfairsc_solve_batched.argtypes = [i32, ctypes.POINTER(BatchGraph), ctypes.POINTER(Opts),
                                          ctypes.POINTER(i32), ctypes.POINTER(BatchInfo), vp]
    for f in ("sfairsc_opts_default", "sfairsc_create", "sfairsc_create_dense", "sfairsc_destroy", "sfairsc_get_sigma",
              "sfairsc_apply_operator", "sfairsc_solve", "sfairsc_kmeans", "sfairsc_backward", "sfairsc_backward_vectors",
              "sfairsc_batch_create", "sfairsc_batch_autotune", "sfairsc_batch_schedule", "sfairsc_batch_solve", "sfairsc_batch_destroy", "sfairsc_batch_stats",
              "sfairsc_solve_batched"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int, where: str, ok=(0,)):
    if rc not in ok:
        raise SFairSCError(rc, where, load().sfairsc_last_error().decode())
    return rc


def sfairsc_strerror(status: int) -> str:
    return load().sfairsc_strerror(status).decode()


def sfairsc_opts_default() -> Opts:
    o = Opts()
    _check(load().sfairsc_opts_default(ctypes.byref(o)), "sfairsc_opts_default")
    return o


def sfairsc_create(n, nnz, row_ptr, col_idx, values, value_dtype, group_labels, h, k, normalized=1, opts=None,
                   stream=None) -> int:
    """Returns the context handle (int).  Pointer arguments are integer addresses."""
    ctx = ctypes.c_void_p()
    rc = load().sfairsc_create(ctypes.byref(ctx), int(n), int(nnz), row_ptr, col_idx, values, int(value_dtype),
                               group_labels, int(h), int(k), int(normalized),
                               ctypes.byref(opts) if opts is not None else None, stream)
    _check(rc, "sfairsc_create")
    return ctx.value


def sfairsc_create_dense(n, nnz, row_ptr, col_idx, values, value_dtype, F, p, k, normalized=1, opts=None,
                         stream=None) -> int:
    """Context with a dense constraint matrix F (n x p row-major FP64 address) in place of labels."""
    ctx = ctypes.c_void_p()
    rc = load().sfairsc_create_dense(ctypes.byref(ctx), int(n), int(nnz), row_ptr, col_idx, values, int(value_dtype),
                                     F, int(p), int(k), int(normalized),
                                     ctypes.byref(opts) if opts is not None else None, stream)
    _check(rc, "sfairsc_create_dense")
    return ctx.value


def sfairsc_destroy(ctx) -> None:
    _check(load().sfairsc_destroy(ctx), "sfairsc_destroy")


def sfairsc_get_sigma(ctx) -> float:
    s = ctypes.c_double()
    _check(load().sfairsc_get_sigma(ctx, ctypes.byref(s)), "sfairsc_get_sigma")
    return s.value


def sfairsc_apply_operator(ctx, w, out, nvec: int) -> None:
    _check(load().sfairsc_apply_operator(ctx, w, out, int(nvec)), "sfairsc_apply_operator")


def sfairsc_solve(ctx, eigenvalues, H, labels, allow=(0,)) -> tuple[int, Info]:
    info = Info()
    rc = load().sfairsc_solve(ctx, eigenvalues, H, labels, ctypes.byref(info))
    _check(rc, "sfairsc_solve", ok=allow)
    return rc, info


def sfairsc_kmeans(n, d, X, kc, seed, n_init, max_iter, labels, centroids=None, stream=None):
    inertia = ctypes.c_double()
    iters = ctypes.c_int32()
    rc = load().sfairsc_kmeans(int(n), int(d), X, int(kc), int(seed), int(n_init), int(max_iter), labels, centroids,
                               ctypes.byref(inertia), ctypes.byref(iters), stream)
    _check(rc, "sfairsc_kmeans")
    return inertia.value, iters.value


def sfairsc_backward_vectors(ctx, grad_H, grad_lambda, grad_values, bandwidth=0.0, want_bandwidth=False, max_iter=0,
                             rtol=0.0):
    """Returns (d loss / d bandwidth or None, CG iterations, largest final relative residual)."""
    gs = ctypes.c_double()
    it = ctypes.c_int32()
    rr = ctypes.c_double()
    rc = load().sfairsc_backward_vectors(ctx, grad_H, grad_lambda, grad_values, float(bandwidth),
                                         ctypes.byref(gs) if want_bandwidth else None, int(max_iter), float(rtol),
                                         ctypes.byref(it), ctypes.byref(rr))
    _check(rc, "sfairsc_backward_vectors")
    return (gs.value if want_bandwidth else None), it.value, rr.value


def sfairsc_backward(ctx, grad_lambda, grad_values, bandwidth=0.0, want_bandwidth=False):
    gs = ctypes.c_double()
    rc = load().sfairsc_backward(ctx, grad_lambda, grad_values, float(bandwidth),
                                 ctypes.byref(gs) if want_bandwidth else None)
    _check(rc, "sfairsc_backward")
    return gs.value if want_bandwidth else None


def _graph_array(graphs):
    arr = (BatchGraph * len(graphs))()
    for i, g in enumerate(graphs):
        arr[i] = g
    return arr


def sfairsc_batch_create(graphs, opts=None, stream=None) -> int:
    """graphs: sequence of BatchGraph (device pointers as integers).  Returns the batch handle."""
    b = ctypes.c_void_p()
    arr = _graph_array(graphs)
    rc = load().sfairsc_batch_create(ctypes.byref(b), len(graphs), arr,
                                     ctypes.byref(opts) if opts is not None else None, stream)
    _check(rc, "sfairsc_batch_create")
    return b.value


def sfairsc_batch_autotune(batch) -> None:
    _check(load().sfairsc_batch_autotune(batch), "sfairsc_batch_autotune")


def sfairsc_batch_schedule(batch, ctas_per_sm: int, max_team: int, split: float) -> None:
    _check(load().sfairsc_batch_schedule(batch, int(ctas_per_sm), int(max_team), float(split)),
           "sfairsc_batch_schedule")


def sfairsc_batch_solve(batch, count: int, allow=(0,)):
    """Returns (rc, per-graph status list, BatchInfo)."""
    st = (ctypes.c_int32 * count)()
    info = BatchInfo()
    rc = load().sfairsc_batch_solve(batch, st, ctypes.byref(info))
    _check(rc, "sfairsc_batch_solve", ok=allow)
    return rc, list(st), info


def sfairsc_batch_stats(batch, count: int):
    """Per-graph (restarts, matvecs, residual / sigma) lists of the last solve."""
    r = (ctypes.c_int32 * count)()
    m = (ctypes.c_int32 * count)()
    d = (ctypes.c_double * count)()
    _check(load().sfairsc_batch_stats(batch, r, m, d), "sfairsc_batch_stats")
    return list(r), list(m), list(d)


def sfairsc_batch_destroy(batch) -> None:
    _check(load().sfairsc_batch_destroy(batch), "sfairsc_batch_destroy")


def sfairsc_solve_batched(graphs, opts=None, stream=None, allow=(0,)):
    st = (ctypes.c_int32 * len(graphs))()
    info = BatchInfo()
    arr = _graph_array(graphs)
    rc = load().sfairsc_solve_batched(len(graphs), arr, ctypes.byref(opts) if opts is not None else None, st,
                                      ctypes.byref(info), stream)
    _check(rc, "sfairsc_solve_batched", ok=allow)
    return rc, list(st), info


def make_opts(prec="mixed", block=1, tol=1e-6, basis=0, max_restarts=200, sigma=None, seed=1, kmeans_seed=0,
              kmeans_n_init=1, kmeans_max_iter=100, validate=1, profile=0, wait_limit_us=0, fault_inject=0,
              spmv_window=0, orth_mode=0, restart_mode=0) -> Opts:
    o = sfairsc_opts_default()
    o.prec = SFAIRSC_PREC_FP64 if prec == "fp64" else SFAIRSC_PREC_MIXED
    o.block = int(block)
    o.tol = float(tol)
    o.basis = int(basis)
    o.max_restarts = int(max_restarts)
    o.sigma = math.nan if sigma is None else float(sigma)
    o.seed = int(seed)
    o.kmeans_seed = int(kmeans_seed)
    o.kmeans_n_init = int(kmeans_n_init)
    o.kmeans_max_iter = int(kmeans_max_iter)
    o.validate = int(validate)
    o.profile = int(profile)
    o.wait_limit_us = int(wait_limit_us)
    o.fault_inject = int(fault_inject)
    o.spmv_window = int(spmv_window)
    o.orth_mode = int(orth_mode)
    o.restart_mode = int(restart_mode)
    return o
