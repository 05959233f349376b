"""Python binding of libgblu (the C ABI declared in include/gblu.h).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  Device arrays are torch tensors (float64, contiguous, on the
handle's device); the stream defaults to torch's current stream.  There is
no CPU fallback: if the library cannot be loaded or the device cannot be
used, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK = 0
REPIVOTED = 1
ERR_INVALID_INPUT = -1
ERR_SINGULAR = -2
ERR_NOT_ANALYZED = -3
ERR_NOMEM = -4
ERR_DEVICE_TIMEOUT = -5
ERR_CUDA = -6
ERR_NOT_FACTORIZED = -7
ERR_INTERNAL = -8
ERR_BUSY = -9
ERR_NONFINITE = -10

SCHED = {"auto": 0, "level": 1, "syncfree": 2}

_lock = threading.Lock()
_lib = None

EXPORTED = [
    "gblu_default_opts", "gblu_last_error", "gblu_create", "gblu_destroy", "gblu_analyze",
    "gblu_factorize", "gblu_refactorize", "gblu_solve", "gblu_residual", "gblu_get_stats",
    "gblu_export_factors", "gblu_order_mindeg", "gblu_column_etree", "gblu_restart_set",
    "gblu_levels", "gblu_step_host", "gblu_solve_factors_noalloc", "gblu_refactorize_batch",
    "gblu_solve_batch", "gblu_refactorize_f32", "gblu_solve_refined", "gblu_refactorize_forced",
    "gblu_refactorize_multi", "gblu_solve_multi", "gblu_step", "gblu_get_opts", "gblu_set_opts",
    "gblu_autotune", "gblu_static_pivot", "gblu_permute_rows", "gblu_gather_scale", "gblu_order_nd",
    "gblu_symmetric_fill", "gblu_order_cnd", "gblu_symmetric_cost", "gblu_order_cmd", "gblu_order_auto",
    "gblu_order_amf", "gblu_last_status", "gblu_solve_partition",
    "gblu_server_last_error", "gblu_server_create", "gblu_server_add_pattern", "gblu_server_pattern_info",
    "gblu_server_submit", "gblu_server_wait", "gblu_server_get_stats", "gblu_server_destroy",
    "gblu_fp64_fma_rate", "gblu_step_batch", "gblu_symmetric_structure", "gblu_predicted_structure",
]

NOALLOC_MAX_N = 524288


class GbluError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gblu error {code}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("pivot_tol", ctypes.c_double), ("sched_mode", ctypes.c_int),
                ("solve_mode", ctypes.c_int), ("alpha", ctypes.c_double),
                ("spin_limit", ctypes.c_longlong), ("solve_dense_frac", ctypes.c_double),
                ("solve_dense_min", ctypes.c_longlong), ("solve_slices", ctypes.c_int),
                ("solve_dense_density", ctypes.c_double), ("dense_min_rows", ctypes.c_int),
                ("warp_column_max", ctypes.c_int), ("speculate_first", ctypes.c_int),
                ("batch_group", ctypes.c_int), ("solve_ctas_per_sm", ctypes.c_int), ("max_sms", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz_a", ctypes.c_int64), ("nnz_l", ctypes.c_int64),
                ("nnz_u", ctypes.c_int64), ("flops", ctypes.c_double),
                ("n_levels", ctypes.c_int32), ("div_level", ctypes.c_int32),
                ("n_solve_levels_l", ctypes.c_int32), ("n_solve_levels_u", ctypes.c_int32),
                ("solve_p0_l", ctypes.c_int32), ("solve_p0_u", ctypes.c_int32),
                ("solve_slices_l", ctypes.c_int32), ("solve_slices_u", ctypes.c_int32),
                ("etree_height", ctypes.c_int32), ("n_refactor", ctypes.c_int64),
                ("n_repivot", ctypes.c_int64), ("n_restart_cols", ctypes.c_int64),
                ("last_first_bad", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("dense_rows", ctypes.c_int32),
                ("tail_kernel_ms", ctypes.c_double), ("tail_repack_ms", ctypes.c_double),
                ("tail_schedule_ms", ctypes.c_double), ("tail_upload_ms", ctypes.c_double),
                ("tail_passes", ctypes.c_int32), ("first_mode", ctypes.c_int32),
                ("first_symbolic_ms", ctypes.c_double), ("wide_cols", ctypes.c_int64),
                ("repredictions", ctypes.c_int32)]


class RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("repivoted", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("pattern", ctypes.c_int32), ("berr", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("refine_iters", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("reserved_bytes", ctypes.c_int64),
                ("n_patterns", ctypes.c_int32), ("max_batch_seen", ctypes.c_int32),
                ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("repivots", ctypes.c_int64)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgblu.so (building it with nvcc first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise OSError(f"libgblu not built: {path}")
            path = _build.build()
        lib = ctypes.CDLL(path)
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.gblu_default_opts.argtypes = [ctypes.POINTER(Opts)]
        lib.gblu_default_opts.restype = None
        lib.gblu_last_error.argtypes = []
        lib.gblu_last_error.restype = ctypes.c_char_p
        lib.gblu_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(Opts)]
        lib.gblu_destroy.argtypes = [P]
        lib.gblu_destroy.restype = None
        lib.gblu_analyze.argtypes = [P, I32, P, P, P]
        lib.gblu_factorize.argtypes = [P, P, P]
        lib.gblu_refactorize.argtypes = [P, P, P, ctypes.POINTER(I32)]
        lib.gblu_refactorize_forced.argtypes = [P, P, P, I32, ctypes.POINTER(I32)]
        lib.gblu_refactorize_multi.argtypes = [I32, P, P, P, P]
        lib.gblu_step.argtypes = [P, P, P, P, P, ctypes.POINTER(I32)]
        lib.gblu_get_opts.argtypes = [P, ctypes.POINTER(Opts)]
        lib.gblu_static_pivot.argtypes = [I32, P, P, P, P, P, P]
        lib.gblu_permute_rows.argtypes = [I32, P, P, P, P, P]
        lib.gblu_gather_scale.argtypes = [I64, P, P, P, P, P]
        lib.gblu_set_opts.argtypes = [P, ctypes.POINTER(Opts), P]
        lib.gblu_autotune.argtypes = [P, P, P, P, I32, P, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
        lib.gblu_solve_multi.argtypes = [I32, P, P, P, P]
        lib.gblu_solve.argtypes = [P, P, P, P]
        lib.gblu_residual.argtypes = [P, P, P, P, P, P]
        lib.gblu_step_host.argtypes = [P, P, P, P, P, ctypes.POINTER(I32)]
        lib.gblu_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
        lib.gblu_export_factors.argtypes = [P] * 9
        lib.gblu_order_mindeg.argtypes = [I32, P, P, P]
        lib.gblu_order_nd.argtypes = [I32, P, P, P]
        lib.gblu_order_nd.restype = ctypes.c_int
        lib.gblu_symmetric_fill.argtypes = [I32, P, P, P]
        lib.gblu_symmetric_fill.restype = I64
        lib.gblu_symmetric_structure.argtypes = [I32, P, P, P, P, P, P]
        lib.gblu_symmetric_structure.restype = I64
        lib.gblu_predicted_structure.argtypes = [I32, P, P, P, P, P, P, P]
        lib.gblu_predicted_structure.restype = I64
        lib.gblu_order_cnd.argtypes = [I32, P, P, P]
        lib.gblu_order_cnd.restype = ctypes.c_int
        lib.gblu_symmetric_cost.argtypes = [I32, P, P, P, P, P]
        lib.gblu_symmetric_cost.restype = ctypes.c_int
        lib.gblu_solve_partition.argtypes = [I32, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_longlong,
                                             ctypes.c_int, ctypes.c_int, P, P]
        lib.gblu_solve_partition.restype = I32
        lib.gblu_last_status.argtypes = [P, P]
        lib.gblu_last_status.restype = ctypes.c_int
        lib.gblu_order_amf.argtypes = [I32, P, P, P]
        lib.gblu_order_amf.restype = ctypes.c_int
        lib.gblu_order_cmd.argtypes = [I32, P, P, P, P]
        lib.gblu_order_cmd.restype = ctypes.c_int
        lib.gblu_order_auto.argtypes = [I32, P, P, P, P]
        lib.gblu_order_auto.restype = ctypes.c_int
        lib.gblu_column_etree.argtypes = [I32, P, P, P, P]
        lib.gblu_restart_set.argtypes = [I32, P, P, P]
        lib.gblu_restart_set.restype = I64
        lib.gblu_solve_factors_noalloc.argtypes = [I32] + [P] * 12 + [ctypes.c_longlong, P]
        lib.gblu_solve_factors_noalloc.restype = ctypes.c_int
        lib.gblu_step_batch.argtypes = [P, I32, P, I64, P, I64, P, I64, P, I64, P, ctypes.POINTER(I32), P]
        lib.gblu_step_batch.restype = ctypes.c_int
        lib.gblu_fp64_fma_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        lib.gblu_fp64_fma_rate.restype = ctypes.c_int
        lib.gblu_levels.argtypes = [I32, P, P, P]
        lib.gblu_levels.restype = I32
        lib.gblu_refactorize_batch.argtypes = [P, I32, P, I64, P, I64, P, ctypes.POINTER(I32), P]
        lib.gblu_solve_batch.argtypes = [P, I32, P, I64, P, I64, P, I64, P]
        lib.gblu_refactorize_f32.argtypes = [P, P, P, ctypes.POINTER(I32)]
        lib.gblu_solve_refined.argtypes = [P, P, P, P, ctypes.c_double, I32, P, ctypes.POINTER(I32),
                                           ctypes.POINTER(ctypes.c_double)]
        lib.gblu_server_last_error.argtypes = []
        lib.gblu_server_last_error.restype = ctypes.c_char_p
        lib.gblu_server_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, I64, I32, ctypes.POINTER(Opts)]
        lib.gblu_server_add_pattern.argtypes = [P, I32, P, P, P, P, ctypes.POINTER(I32), ctypes.POINTER(I32)]
        lib.gblu_server_pattern_info.argtypes = [P, I32, ctypes.POINTER(I32), ctypes.POINTER(I64),
                                                 ctypes.POINTER(I64)]
        lib.gblu_server_submit.argtypes = [P, I32, P, P, P, I32, ctypes.POINTER(I64)]
        lib.gblu_server_wait.argtypes = [P, I64, ctypes.c_double, ctypes.POINTER(RequestResult)]
        lib.gblu_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
        lib.gblu_server_destroy.argtypes = [P]
        lib.gblu_server_destroy.restype = None
        for f in ("gblu_server_create", "gblu_server_add_pattern", "gblu_server_pattern_info",
                  "gblu_server_submit", "gblu_server_wait", "gblu_server_get_stats"):
            getattr(lib, f).restype = ctypes.c_int
        for f in ("gblu_create", "gblu_analyze", "gblu_factorize", "gblu_refactorize", "gblu_step_host",
                  "gblu_solve", "gblu_residual", "gblu_get_stats", "gblu_export_factors",
                  "gblu_order_mindeg", "gblu_column_etree", "gblu_refactorize_batch", "gblu_solve_batch",
                  "gblu_refactorize_f32", "gblu_solve_refined", "gblu_refactorize_forced",
                  "gblu_refactorize_multi", "gblu_solve_multi", "gblu_step", "gblu_get_opts",
                  "gblu_set_opts", "gblu_autotune", "gblu_static_pivot", "gblu_permute_rows",
                  "gblu_gather_scale"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(code):
    if code < 0:
        raise GbluError(code, load().gblu_last_error().decode())
    return code


def _dev_ptr(t, device, n=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("expected a CUDA float64 torch tensor")
    if t.device.index != device:
        raise ValueError(f"tensor on cuda:{t.device.index}, handle on cuda:{device}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Solver:
    """One handle: analyze a pattern once, then factorize / refactorize / solve."""

    def __init__(self, device=0, pivot_tol=1e-3, sched_mode="auto", solve_mode="auto",
                 alpha=2.0, spin_limit=1 << 24, solve_dense_frac=None, solve_dense_min=None,
                 solve_slices=None, solve_dense_density=None, dense_min_rows=None, warp_column_max=None,
                 speculate_first=None):
        lib = load()
        o = Opts()
        lib.gblu_default_opts(ctypes.byref(o))
        o.pivot_tol = pivot_tol
        o.sched_mode = SCHED[sched_mode]
        o.solve_mode = SCHED[solve_mode]
        o.alpha = alpha
        o.spin_limit = spin_limit
        if solve_dense_frac is not None:
            o.solve_dense_frac = solve_dense_frac
        if solve_dense_min is not None:
            o.solve_dense_min = solve_dense_min
        if solve_slices is not None:
            o.solve_slices = solve_slices
        if solve_dense_density is not None:
            o.solve_dense_density = solve_dense_density
        if dense_min_rows is not None:
            o.dense_min_rows = dense_min_rows
        if warp_column_max is not None:
            o.warp_column_max = warp_column_max
        if speculate_first is not None:
            o.speculate_first = int(speculate_first)
        h = ctypes.c_void_p()
        _check(lib.gblu_create(ctypes.byref(h), int(device), ctypes.byref(o)))
        self._h = h
        self.device = int(device)
        self.n = None
        self.nnz = None

    def close(self):
        if getattr(self, "_h", None):
            load().gblu_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def analyze(self, n, Ap, Ai, Q=None):
        Ap, Ai = _i32(Ap), _i32(Ai)
        q = None if Q is None else _i32(Q)
        _check(load().gblu_analyze(self._h, int(n), _np_ptr(Ap), _np_ptr(Ai),
                                   None if q is None else _np_ptr(q)))
        self.n, self.nnz = int(n), int(Ap[-1])

    def factorize(self, Ax, stream=None):
        return _check(load().gblu_factorize(self._h, _dev_ptr(Ax, self.device, self.nnz),
                                            _stream(stream)))

    def refactorize(self, Ax, stream=None):
        rep = ctypes.c_int32(0)
        rc = _check(load().gblu_refactorize(self._h, _dev_ptr(Ax, self.device, self.nnz),
                                            _stream(stream), ctypes.byref(rep)))
        return rc, bool(rep.value)

    def opts(self):
        o = Opts()
        _check(load().gblu_get_opts(self._h, ctypes.byref(o)))
        return {f: getattr(o, f) for f, _ in Opts._fields_}

    def set_opts(self, stream=None, **kw):
        """Change options; the schedule is rebuilt for the current factors."""
        o = Opts()
        _check(load().gblu_get_opts(self._h, ctypes.byref(o)))
        for k, v in kw.items():
            if k in ("sched_mode", "solve_mode") and isinstance(v, str):
                v = SCHED[v]
            setattr(o, k, v)
        _check(load().gblu_set_opts(self._h, ctypes.byref(o), _stream(stream)))

    def autotune(self, Ax, b, x=None, reps=3, stream=None):
        """Measure schedule options on this matrix and keep the fastest;
        returns (chosen options, refactor ms, solve ms)."""
        import torch
        if x is None:
            x = torch.empty_like(b)
        o = Opts()
        tr, ts = ctypes.c_double(0), ctypes.c_double(0)
        _check(load().gblu_autotune(self._h, _dev_ptr(Ax, self.device, self.nnz), _dev_ptr(b, self.device, self.n),
                                    _dev_ptr(x, self.device, self.n), int(reps), _stream(stream), ctypes.byref(o),
                                    ctypes.byref(tr), ctypes.byref(ts)))
        return {f: getattr(o, f) for f, _ in Opts._fields_}, tr.value, ts.value

    def step(self, Ax, b, x=None, stream=None):
        """Checked re-factorization and solve replayed from a CUDA graph
        (gblu_step); returns (x, repivoted)."""
        import torch
        if x is None:
            x = torch.empty_like(b)
        rep = ctypes.c_int32(0)
        _check(load().gblu_step(self._h, _dev_ptr(Ax, self.device, self.nnz), _dev_ptr(b, self.device, self.n),
                                _dev_ptr(x, self.device, self.n), _stream(stream), ctypes.byref(rep)))
        return x, bool(rep.value)

    def refactorize_forced(self, Ax, force_col, stream=None):
        """refactorize with the check of step force_col failing (re-pivoting protocol)."""
        rep = ctypes.c_int32(0)
        rc = _check(load().gblu_refactorize_forced(self._h, _dev_ptr(Ax, self.device, self.nnz),
                                                   _stream(stream), int(force_col), ctypes.byref(rep)))
        return rc, bool(rep.value)

    def solve(self, b, x=None, stream=None):
        import torch
        if x is None:
            x = torch.empty_like(b)
        _check(load().gblu_solve(self._h, _dev_ptr(b, self.device, self.n),
                                 _dev_ptr(x, self.device, self.n), _stream(stream)))
        return x

    def refactorize_batch(self, Ax, LUx=None, stream=None):
        """Checked re-factorization of a batch of value sets on this structure.

        Ax: CUDA float64 tensor [nsets, nnz(A)].  Returns (LUx, failed): LUx
        [nsets, nnz(L+U)] holds each set's factor values (pass it to
        solve_batch), failed is a numpy int32 [nsets] (1: a pivot failed the
        check; that set needs a handle of its own)."""
        import torch
        if Ax.dim() != 2 or Ax.shape[1] != self.nnz:
            raise ValueError("Ax must be [nsets, nnz(A)]")
        _dev_ptr(Ax, self.device)
        nsets = Ax.shape[0]
        st = self.stats()
        nlu = st["nnz_l"] + st["nnz_u"]
        if LUx is None:
            LUx = torch.empty((nsets, nlu), dtype=torch.float64, device=Ax.device)
        if LUx.dim() != 2 or LUx.shape[0] != nsets or LUx.shape[1] != nlu:
            raise ValueError("LUx must be [nsets, nnz(L+U)]")
        _dev_ptr(LUx, self.device)
        failed = np.zeros(nsets, np.int32)
        nf = ctypes.c_int32(0)
        _check(load().gblu_refactorize_batch(self._h, nsets, ctypes.c_void_p(Ax.data_ptr()), self.nnz,
                                             ctypes.c_void_p(LUx.data_ptr()), nlu, _np_ptr(failed),
                                             ctypes.byref(nf), _stream(stream)))
        return LUx, failed

    def solve_batch(self, LUx, b, x=None, stream=None):
        """Solve every set of a batch: LUx [nsets, nnz(L+U)], b [nsets, n]."""
        import torch
        if x is None:
            x = torch.empty_like(b)
        for t in (LUx, b, x):
            _dev_ptr(t, self.device)
        if b.dim() != 2 or b.shape[1] != self.n or b.shape != x.shape or LUx.shape[0] != b.shape[0]:
            raise ValueError("b and x must be [nsets, n] and match LUx")
        _check(load().gblu_solve_batch(self._h, b.shape[0], ctypes.c_void_p(LUx.data_ptr()), LUx.shape[1],
                                       ctypes.c_void_p(b.data_ptr()), self.n, ctypes.c_void_p(x.data_ptr()),
                                       self.n, _stream(stream)))
        return x

    def step_batch(self, Ax, LUx, b, x, stream=None):
        """refactorize_batch + solve_batch replayed from a CUDA graph
        (gblu_step_batch); Ax [nsets, nnz(A)], LUx [nsets, nnz(L+U)], b and x
        [nsets, n].  Returns failed (numpy int32 [nsets])."""
        nsets = Ax.shape[0]
        for t in (Ax, LUx, b, x):
            _dev_ptr(t, self.device)
        if (Ax.dim() != 2 or Ax.shape[1] != self.nnz or LUx.dim() != 2 or LUx.shape[0] != nsets
                or b.shape != x.shape or b.dim() != 2 or b.shape[0] != nsets or b.shape[1] != self.n):
            raise ValueError("Ax [nsets, nnz(A)], LUx [nsets, nnz(L+U)], b and x [nsets, n]")
        failed = np.zeros(nsets, np.int32)
        nf = ctypes.c_int32(0)
        _check(load().gblu_step_batch(self._h, nsets, ctypes.c_void_p(Ax.data_ptr()), self.nnz,
                                      ctypes.c_void_p(LUx.data_ptr()), LUx.shape[1],
                                      ctypes.c_void_p(b.data_ptr()), self.n, ctypes.c_void_p(x.data_ptr()),
                                      self.n, _np_ptr(failed), ctypes.byref(nf), _stream(stream)))
        return failed

    def refactorize_f32(self, Ax, stream=None):
        """Single-precision checked re-factorization; returns True if a pivot failed."""
        failed = ctypes.c_int32(0)
        _check(load().gblu_refactorize_f32(self._h, _dev_ptr(Ax, self.device, self.nnz), _stream(stream),
                                           ctypes.byref(failed)))
        return bool(failed.value)

    def solve_refined(self, Ax, b, x=None, tol=1e-12, max_iter=10, stream=None):
        """Iterative refinement on the single-precision factors (double fallback).

        Returns (x, iters, berr); iters == -1 means the double fallback ran."""
        import torch
        if x is None:
            x = torch.empty_like(b)
        it = ctypes.c_int32(0)
        be = ctypes.c_double(0.0)
        _check(load().gblu_solve_refined(self._h, _dev_ptr(Ax, self.device, self.nnz),
                                         _dev_ptr(b, self.device, self.n), _dev_ptr(x, self.device, self.n),
                                         float(tol), int(max_iter), _stream(stream), ctypes.byref(it),
                                         ctypes.byref(be)))
        return x, it.value, be.value

    def step_host(self, Ax, b, x, stream=None):
        """Refactorize + solve from host numpy float64 arrays (x is written)."""
        for a, m in ((Ax, self.nnz), (b, self.n), (x, self.n)):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                    and a.size == m):
                raise ValueError("expected contiguous float64 numpy arrays of the right size")
        rep = ctypes.c_int32(0)
        rc = _check(load().gblu_step_host(self._h, _np_ptr(Ax), _np_ptr(b), _np_ptr(x),
                                          _stream(stream), ctypes.byref(rep)))
        return rc, bool(rep.value)

    def residual(self, Ax, b, x, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(4, dtype=torch.float64, device=b.device)
        _check(load().gblu_residual(self._h, _dev_ptr(Ax, self.device, self.nnz),
                                    _dev_ptr(b, self.device, self.n),
                                    _dev_ptr(x, self.device, self.n),
                                    _dev_ptr(out, self.device, 4), _stream(stream)))
        return out

    def last_status(self, stream=None) -> int:
        """gblu_last_status: the code of the handle's last device work (OK,
        REPIVOTED or a negative device error), returned, not raised."""
        return int(load().gblu_last_status(self._h, _stream(stream)))

    def stats(self) -> dict:
        s = Stats()
        _check(load().gblu_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def export_factors(self) -> dict:
        st = self.stats()
        n, nl, nu = st["n"], st["nnz_l"], st["nnz_u"]
        out = dict(Lp=np.empty(n + 1, np.int64), Li=np.empty(max(nl, 1), np.int32),
                   Lx=np.empty(max(nl, 1), np.float64), Up=np.empty(n + 1, np.int64),
                   Ui=np.empty(max(nu, 1), np.int32), Ux=np.empty(max(nu, 1), np.float64),
                   piv=np.empty(n, np.int32), q=np.empty(n, np.int32))
        _check(load().gblu_export_factors(self._h, *[_np_ptr(out[k]) for k in
                                                     ("Lp", "Li", "Lx", "Up", "Ui", "Ux", "piv", "q")]))
        for k, m in (("Li", nl), ("Lx", nl), ("Ui", nu), ("Ux", nu)):
            out[k] = out[k][:m]
        return out


def fp64_fma_rate(device=0) -> float:
    """gblu_fp64_fma_rate: the device's measured FP64 multiply-add rate, TFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(load().gblu_fp64_fma_rate(int(device), ctypes.byref(v)))
    return float(v.value)


def solve_factors_noalloc(n, Lrp, Lcol, Lval, Urp, Ucol, Uval, Udiag, piv, q, b, x,
                          status=None, stream=None, spin_limit=0):
    """Allocation-free solve from caller-held row-wise factors (all CUDA tensors:
    Lrp/Urp int64, Lcol/Ucol/piv/q int32, values float64); spin_limit <= 0:
    the library's default wait limit."""
    import torch
    ptrs = []
    for t, dt in ((Lrp, torch.int64), (Lcol, torch.int32), (Lval, torch.float64),
                  (Urp, torch.int64), (Ucol, torch.int32), (Uval, torch.float64),
                  (Udiag, torch.float64), (piv, torch.int32), (q, torch.int32),
                  (b, torch.float64), (x, torch.float64)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError(f"expected a contiguous CUDA {dt} tensor")
        ptrs.append(ctypes.c_void_p(t.data_ptr()))
    st = None if status is None else ctypes.c_void_p(status.data_ptr())
    return _check(load().gblu_solve_factors_noalloc(int(n), *ptrs, st, int(spin_limit), _stream(stream)))


# ---------------------------------------------------------------- host-only helpers
def order_mindeg(n, Ap, Ai):
    Ap, Ai = _i32(Ap), _i32(Ai)
    perm = np.empty(n, np.int32)
    _check(load().gblu_order_mindeg(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(perm)))
    return perm


def order_nd(n, Ap, Ai):
    """Nested dissection order without coordinates (gblu_order_nd, host)."""
    Ap, Ai = _i32(Ap), _i32(Ai)
    perm = np.empty(n, np.int32)
    _check(load().gblu_order_nd(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(perm)))
    return perm


def order_cnd(n, Ap, Ai):
    """Incomplete nested dissection + constrained minimum degree (gblu_order_cnd, host)."""
    Ap, Ai = _i32(Ap), _i32(Ai)
    perm = np.empty(n, np.int32)
    _check(load().gblu_order_cnd(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(perm)))
    return perm


def solve_partition(count_from, rowlen, density=0.0, frac=0.7, min_entries=300000, slices=8, max_piece=4096):
    """Section V-A's split of one triangle (gblu_solve_partition, host): (P0, cut rows)."""
    count_from = np.ascontiguousarray(count_from, dtype=np.int64)
    rowlen = np.ascontiguousarray(rowlen, dtype=np.int64)
    n = len(rowlen)
    cut = np.empty(n + 1, np.int32)
    ncut = ctypes.c_int32()
    p0 = load().gblu_solve_partition(int(n), _np_ptr(count_from), _np_ptr(rowlen), float(density), float(frac),
                                     int(min_entries), int(slices), int(max_piece), _np_ptr(cut),
                                     ctypes.byref(ncut))
    _check(min(p0, 0))
    return int(p0), cut[:ncut.value].copy()


def order_amf(n, Ap, Ai):
    """Approximate minimum deficiency order (gblu_order_amf, host)."""
    Ap, Ai = _i32(Ap), _i32(Ai)
    perm = np.empty(n, np.int32)
    _check(load().gblu_order_amf(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(perm)))
    return perm


def order_cmd(n, Ap, Ai, group):
    """Constrained minimum degree: groups eliminated in increasing order (gblu_order_cmd, host)."""
    Ap, Ai, group = _i32(Ap), _i32(Ai), _i32(group)
    perm = np.empty(n, np.int32)
    _check(load().gblu_order_cmd(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(group), _np_ptr(perm)))
    return perm


ORDER_METHODS = {0: "mindeg", 1: "nd", 2: "cnd", 3: "amf"}


def order_auto(n, Ap, Ai):
    """The candidate order of fewest flops (gblu_order_auto, host): (perm, method name)."""
    Ap, Ai = _i32(Ap), _i32(Ai)
    perm = np.empty(n, np.int32)
    m = ctypes.c_int32()
    _check(load().gblu_order_auto(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(perm), ctypes.byref(m)))
    return perm, ORDER_METHODS[m.value]


def symmetric_cost(n, Ap, Ai, Q):
    """(fill, flops) of an order when every diagonal pivot is kept (gblu_symmetric_cost, host)."""
    Ap, Ai, Q = _i32(Ap), _i32(Ai), _i32(Q)
    fill = ctypes.c_int64()
    flops = ctypes.c_double()
    _check(load().gblu_symmetric_cost(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(Q), ctypes.byref(fill),
                                      ctypes.byref(flops)))
    return int(fill.value), float(flops.value)


def symmetric_fill(n, Ap, Ai, Q):
    """Strict lower Cholesky entries of (A + A^T)(Q,Q) (gblu_symmetric_fill, host)."""
    Ap, Ai, Q = _i32(Ap), _i32(Ai), _i32(Q)
    v = load().gblu_symmetric_fill(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(Q))
    if v < 0:
        raise GbluError(int(v), "invalid pattern or order")
    return int(v)


def symmetric_structure(n, Ap, Ai, Q):
    """The structure gblu_factorize predicts for its first factorization
    (gblu_symmetric_structure, host): (LUp, LUi, nU) in step numbering."""
    Ap, Ai, Q = _i32(Ap), _i32(Ai), _i32(Q)
    lib = load()
    nnz = lib.gblu_symmetric_structure(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(Q), None, None, None)
    if nnz < 0:
        raise GbluError(int(nnz), "invalid pattern or order")
    LUp = np.empty(n + 1, np.int64)
    LUi = np.empty(max(nnz, 1), np.int32)
    nU = np.empty(n, np.int32)
    lib.gblu_symmetric_structure(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(Q), _np_ptr(LUp), _np_ptr(LUi),
                                 _np_ptr(nU))
    return LUp, LUi[:nnz], nU


def predicted_structure(n, Ap, Ai, Q, piv=None):
    """The structure predicted for the steps taking the original rows piv
    (gblu_predicted_structure, host; piv None = Q): (LUp, LUi, nU)."""
    Ap, Ai, Q = _i32(Ap), _i32(Ai), _i32(Q)
    pv = None if piv is None else _i32(piv)
    pp = None if pv is None else _np_ptr(pv)
    lib = load()
    nnz = lib.gblu_predicted_structure(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(Q), pp, None, None, None)
    if nnz < 0:
        raise GbluError(int(nnz), "invalid pattern, order or rows")
    LUp = np.empty(n + 1, np.int64)
    LUi = np.empty(max(nnz, 1), np.int32)
    nU = np.empty(n, np.int32)
    lib.gblu_predicted_structure(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(Q), pp, _np_ptr(LUp), _np_ptr(LUi),
                                 _np_ptr(nU))
    return LUp, LUi[:nnz], nU


def column_etree(n, Ap, Ai, Q=None):
    Ap, Ai = _i32(Ap), _i32(Ai)
    q = None if Q is None else _i32(Q)
    parent = np.empty(n, np.int32)
    _check(load().gblu_column_etree(int(n), _np_ptr(Ap), _np_ptr(Ai),
                                    None if q is None else _np_ptr(q), _np_ptr(parent)))
    return parent


def restart_set(parent, finished):
    parent = _i32(parent)
    fin = np.ascontiguousarray(finished, dtype=np.uint8)
    out = np.empty(len(parent), np.uint8)
    cnt = load().gblu_restart_set(len(parent), _np_ptr(parent), _np_ptr(fin), _np_ptr(out))
    _check(int(cnt) if cnt < 0 else 0)
    return out.astype(bool)


def levels(n, Up, Ui):
    Up = np.ascontiguousarray(Up, dtype=np.int64)
    Ui = _i32(Ui)
    lv = np.empty(n, np.int32)
    nl = load().gblu_levels(int(n), _np_ptr(Up), _np_ptr(Ui), _np_ptr(lv))
    _check(int(nl) if nl < 0 else 0)
    return lv, int(nl)



def refactorize_multi(solvers, Ax_list, stream=None):
    """One launch re-factorizing several handles of different patterns, each
    with its own values (gblu_refactorize_multi).  Returns the per-handle
    repivoted flags."""
    nh = len(solvers)
    if nh != len(Ax_list) or nh == 0:
        raise ValueError("one value array per solver")
    dev = solvers[0].device
    hs = (ctypes.c_void_p * nh)(*[s._h for s in solvers])
    ax = (ctypes.c_void_p * nh)(*[_dev_ptr(a, dev, s.nnz) for s, a in zip(solvers, Ax_list)])
    rep = (ctypes.c_int32 * nh)()
    _check(load().gblu_refactorize_multi(nh, hs, ax, _stream(stream), rep))
    return [bool(v) for v in rep]


def solve_multi(solvers, b_list, x_list=None, stream=None):
    """gblu_solve for every handle; returns the solutions."""
    import torch
    nh = len(solvers)
    if x_list is None:
        x_list = [torch.empty_like(b) for b in b_list]
    dev = solvers[0].device
    hs = (ctypes.c_void_p * nh)(*[s._h for s in solvers])
    bp = (ctypes.c_void_p * nh)(*[_dev_ptr(b, dev, s.n) for s, b in zip(solvers, b_list)])
    xp = (ctypes.c_void_p * nh)(*[_dev_ptr(x, dev, s.n) for s, x in zip(solvers, x_list)])
    _check(load().gblu_solve_multi(nh, hs, bp, xp, _stream(stream)))
    return x_list


def static_pivot(n, Ap, Ai, Ax):
    """Maximum-product static pivoting with scaling (gblu_static_pivot, host):
    returns (match, row_scale, col_scale)."""
    Ap, Ai = _i32(Ap), _i32(Ai)
    Ax = np.ascontiguousarray(Ax, dtype=np.float64)
    match = np.empty(n, np.int32)
    dr = np.empty(n, np.float64)
    dc = np.empty(n, np.float64)
    _check(load().gblu_static_pivot(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(Ax), _np_ptr(match), _np_ptr(dr),
                                    _np_ptr(dc)))
    return match, dr, dc


def permute_rows(n, Ap, Ai, match):
    """Pattern of P A (gblu_permute_rows): (Ai_out, src)."""
    Ap, Ai, match = _i32(Ap), _i32(Ai), _i32(match)
    Ai2 = np.empty_like(Ai)
    src = np.empty_like(Ai)
    _check(load().gblu_permute_rows(int(n), _np_ptr(Ap), _np_ptr(Ai), _np_ptr(match), _np_ptr(Ai2), _np_ptr(src)))
    return Ai2, src


def gather_scale(inp, out, src=None, scale=None, stream=None):
    """out[k] = inp[src[k]] * scale[k] on the device (gblu_gather_scale)."""
    dev = out.device.index
    m = out.numel()
    sp = None if src is None else ctypes.c_void_p(src.data_ptr())
    cp = None if scale is None else _dev_ptr(scale, dev, m)
    _check(load().gblu_gather_scale(int(m), sp, cp, _dev_ptr(inp, dev), _dev_ptr(out, dev, m), _stream(stream)))
    return out


class StaticScaling:
    """A pattern with static pivoting and scaling: analyze the returned
    pattern (Ap, Ai_scaled), then per value set map values and right-hand
    side to the scaled system on the device and map its solution back."""

    def __init__(self, n, Ap, Ai, Ax, device=0):
        import torch
        self.n = int(n)
        self.match, self.dr, self.dc = static_pivot(n, Ap, Ai, Ax)
        self.Ai_scaled, src = permute_rows(n, Ap, Ai, self.match)
        Ap, Ai = _i32(Ap), _i32(Ai)
        col = np.repeat(np.arange(n, dtype=np.int64), np.diff(Ap))
        scale = self.dr[Ai[src]] * self.dc[col]
        d = f"cuda:{device}"
        self._src = torch.from_numpy(src.astype(np.int32)).to(d)
        self._scale = torch.from_numpy(scale).to(d)
        self._bsrc = torch.from_numpy(self.match.astype(np.int32)).to(d)
        self._bscale = torch.from_numpy(self.dr[self.match]).to(d)
        self._dc = torch.from_numpy(self.dc).to(d)

    def values(self, Ax, out=None, stream=None):
        import torch
        out = torch.empty_like(Ax) if out is None else out
        return gather_scale(Ax, out, self._src, self._scale, stream)

    def rhs(self, b, out=None, stream=None):
        import torch
        out = torch.empty_like(b) if out is None else out
        return gather_scale(b, out, self._bsrc, self._bscale, stream)

    def solution(self, y, out=None, stream=None):
        import torch
        out = torch.empty_like(y) if out is None else out
        return gather_scale(y, out, None, self._dc, stream)

def _check_server(code):
    if code < 0:
        raise GbluError(code, load().gblu_server_last_error().decode())
    return code


class Server:
    """Solve server on one device (gblu_server_*): patterns stay resident,
    concurrent requests of one pattern are batched, patterns overlap.

    Requests take host numpy arrays; the server keeps references to them
    until the request is waited for."""

    def __init__(self, device=0, hbm_budget=16 << 30, max_batch=64, pivot_tol=1e-3):
        lib = load()
        o = Opts()
        lib.gblu_default_opts(ctypes.byref(o))
        o.pivot_tol = pivot_tol
        s = ctypes.c_void_p()
        _check_server(lib.gblu_server_create(ctypes.byref(s), int(device), int(hbm_budget), int(max_batch),
                                             ctypes.byref(o)))
        self._s = s
        self.device = int(device)
        self._pat = {}      # pattern id -> (n, nnz)
        self._live = {}     # request id -> (Ax, b, x) kept alive

    def add_pattern(self, n, Ap, Ai, Q, Ax0):
        """Register a pattern with its first values; returns (pattern id, slots)."""
        Ap, Ai = _i32(Ap), _i32(Ai)
        q = None if Q is None else _i32(Q)
        Ax0 = np.ascontiguousarray(Ax0, dtype=np.float64)
        pid, slots = ctypes.c_int32(0), ctypes.c_int32(0)
        _check_server(load().gblu_server_add_pattern(self._s, int(n), _np_ptr(Ap), _np_ptr(Ai),
                                                     None if q is None else _np_ptr(q), _np_ptr(Ax0),
                                                     ctypes.byref(pid), ctypes.byref(slots)))
        self._pat[pid.value] = (int(n), int(Ap[-1]))
        return pid.value, slots.value

    def pattern_info(self, pattern):
        slots, fp, nlu = ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _check_server(load().gblu_server_pattern_info(self._s, int(pattern), ctypes.byref(slots),
                                                      ctypes.byref(fp), ctypes.byref(nlu)))
        return {"slots": slots.value, "footprint_bytes": fp.value, "nnz_lu": nlu.value}

    def submit(self, pattern, Ax, b, x=None, mixed=False):
        """Queue a request; returns its id.  x (host float64[n]) receives the
        solution.  mixed=True: single-precision factors with refinement."""
        n, nnz = self._pat[pattern]
        Ax = np.ascontiguousarray(Ax, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        if Ax.size != nnz or b.size != n:
            raise ValueError(f"expected {nnz} values and {n} right-hand-side entries")
        if x is None:
            x = np.empty(n, np.float64)
        if x.dtype != np.float64 or not x.flags.c_contiguous or x.size != n:
            raise ValueError("x must be a contiguous float64 array of n entries")
        rid = ctypes.c_int64(0)
        _check_server(load().gblu_server_submit(self._s, int(pattern), _np_ptr(Ax), _np_ptr(b), _np_ptr(x),
                                                1 if mixed else 0, ctypes.byref(rid)))
        self._live[rid.value] = (Ax, b, x)
        return rid.value

    def wait(self, request, timeout=60.0):
        """Wait for a request; returns (x, result dict).  Raises GbluError
        (code ERR_BUSY) if it has not finished within the timeout."""
        r = RequestResult()
        _check_server(load().gblu_server_wait(self._s, int(request), float(timeout), ctypes.byref(r)))
        _, _, x = self._live.pop(request)
        return x, {f: getattr(r, f) for f, _ in RequestResult._fields_}

    def stats(self):
        st = ServerStats()
        _check_server(load().gblu_server_get_stats(self._s, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_s", None):
            load().gblu_server_destroy(self._s)
            self._s = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
