"""ctypes front end of the C oracle (``gp_oracle.c``) -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product path never does.

Functions (all arrays numpy, CSC int32 / float64):

* ``factorize(n, Ap, Ai, Ax, Q, eps, prefer)`` -- Gilbert-Peierls
  left-looking LU with threshold partial pivoting and a preferred pivot row
  per step (CKTSO Section II-A, Algorithm 1, transposed to CSC).
* ``refactorize(prev, Ap, Ai, Ax, eps)`` -- the same with the previous pivot
  sequence preferred (the result that re-factorization with pivot check and
  restart, Section IV, must produce).
* ``solve(lu, b)`` -- forward and back substitution (Algorithm 2).
* ``residual(n, Ap, Ai, Ax, x, b)`` -- ||b-Ax||_inf / (||A||_inf ||x||_inf);
  ``residual_parts`` gives the ratio and its three norms.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_INPUT = -1
ERR_SINGULAR = -2


def build(force=False) -> str:
    """Compile the oracle with gcc (no FMA contraction, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path):
    """Load a build of ``gp_oracle.c`` from ``path`` (used by the tests that
    plant mistakes in a copy of the source to show that the pins catch them)."""
    return _configure(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(lib):
    P = ctypes.c_void_p
    lib.orc_factorize.restype = P
    lib.orc_factorize.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_double, P]
    for f in ("orc_status", "orc_bad_step", "orc_rejected"):
        getattr(lib, f).restype = ctypes.c_int
        getattr(lib, f).argtypes = [P]
    for f in ("orc_nnz_l", "orc_nnz_u"):
        getattr(lib, f).restype = ctypes.c_longlong
        getattr(lib, f).argtypes = [P]
    lib.orc_export.restype = ctypes.c_int
    lib.orc_export.argtypes = [P] * 8
    lib.orc_solve.restype = ctypes.c_int
    lib.orc_solve.argtypes = [P, P, P]
    lib.orc_residual.restype = ctypes.c_int
    lib.orc_residual.argtypes = [ctypes.c_int, P, P, P, P, P, P]
    lib.orc_free.restype = None
    lib.orc_free.argtypes = [P]
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclasses.dataclass
class OracleLU:
    n: int
    status: int
    bad_step: int
    n_rejected: int
    Q: np.ndarray
    piv: np.ndarray | None = None
    Lp: np.ndarray | None = None
    Li: np.ndarray | None = None
    Lx: np.ndarray | None = None
    Up: np.ndarray | None = None
    Ui: np.ndarray | None = None
    Ux: np.ndarray | None = None
    eps: float = 1e-3
    inputs: tuple | None = None   # (Ap, Ai, Ax) it was computed from
    _h: object = None
    _lib: object = None

    def __del__(self):
        if self._h is not None and self._lib is not None:
            self._lib.orc_free(self._h)
            self._h = None

    @property
    def nnz_l(self):
        return int(self.Lp[-1])

    @property
    def nnz_u(self):
        return int(self.Up[-1])

    def dense_factors(self):
        """(P, L, U) as dense arrays with P @ A[:, Q] == L @ U (small n only)."""
        n = self.n
        L = np.eye(n)
        U = np.zeros((n, n))
        for k in range(n):
            L[self.Li[self.Lp[k]:self.Lp[k + 1]], k] = self.Lx[self.Lp[k]:self.Lp[k + 1]]
            U[self.Ui[self.Up[k]:self.Up[k + 1]], k] = self.Ux[self.Up[k]:self.Up[k + 1]]
        P = np.zeros((n, n))
        P[np.arange(n), self.piv] = 1.0
        return P, L, U


def factorize(n, Ap, Ai, Ax, Q, eps=1e-3, prefer=None, lib=None) -> OracleLU:
    lib = lib or _load()
    Ap = np.ascontiguousarray(Ap, dtype=np.int32)
    Ai = np.ascontiguousarray(Ai, dtype=np.int32)
    Ax = np.ascontiguousarray(Ax, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.int32)
    pref = None if prefer is None else np.ascontiguousarray(prefer, dtype=np.int32)
    h = lib.orc_factorize(int(n), _ptr(Ap), _ptr(Ai), _ptr(Ax), _ptr(Q), float(eps),
                          None if pref is None else _ptr(pref))
    if not h:
        raise MemoryError("oracle factorization ran out of memory")
    lu = OracleLU(n=int(n), status=lib.orc_status(h), bad_step=lib.orc_bad_step(h),
                  n_rejected=lib.orc_rejected(h), Q=Q.copy(), eps=eps, inputs=(Ap, Ai, Ax),
                  _h=h, _lib=lib)
    if lu.status == OK:
        nl, nu = lib.orc_nnz_l(h), lib.orc_nnz_u(h)
        lu.Lp = np.empty(n + 1, np.int32)
        lu.Up = np.empty(n + 1, np.int32)
        lu.Li = np.empty(max(nl, 1), np.int32)
        lu.Lx = np.empty(max(nl, 1), np.float64)
        lu.Ui = np.empty(max(nu, 1), np.int32)
        lu.Ux = np.empty(max(nu, 1), np.float64)
        lu.piv = np.empty(n, np.int32)
        rc = lib.orc_export(h, _ptr(lu.Lp), _ptr(lu.Li), _ptr(lu.Lx), _ptr(lu.Up),
                            _ptr(lu.Ui), _ptr(lu.Ux), _ptr(lu.piv))
        assert rc == OK
        lu.Li, lu.Lx = lu.Li[:nl], lu.Lx[:nl]
        lu.Ui, lu.Ux = lu.Ui[:nu], lu.Ux[:nu]
    return lu


def refactorize(prev: OracleLU, Ap, Ai, Ax, eps=None) -> OracleLU:
    """Factorization of new values preferring ``prev``'s pivot sequence."""
    return factorize(prev.n, Ap, Ai, Ax, prev.Q, prev.eps if eps is None else eps,
                     prefer=prev.piv, lib=prev._lib)


def solve(lu: OracleLU, b) -> np.ndarray:
    lib = lu._lib
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(lu.n, np.float64)
    rc = lib.orc_solve(lu._h, _ptr(b), _ptr(x))
    if rc != OK:
        raise RuntimeError(f"oracle solve failed: {rc}")
    return x


def residual(n, Ap, Ai, Ax, x, b, lib=None) -> float:
    """||b - A x||_inf / (||A||_inf ||x||_inf)."""
    return float(residual_parts(n, Ap, Ai, Ax, x, b, lib)[0])


def residual_parts(n, Ap, Ai, Ax, x, b, lib=None) -> np.ndarray:
    """[ratio, ||b - A x||_inf, ||A||_inf, ||x||_inf] (ratio = ||r|| when
    ||A|| or ||x|| is 0; every norm is NaN if an entry it takes is NaN)."""
    lib = lib or _load()
    out = np.zeros(4)
    Ap = np.ascontiguousarray(Ap, dtype=np.int32)
    Ai = np.ascontiguousarray(Ai, dtype=np.int32)
    Ax = np.ascontiguousarray(Ax, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    rc = lib.orc_residual(int(n), _ptr(Ap), _ptr(Ai), _ptr(Ax), _ptr(x), _ptr(b), _ptr(out))
    if rc != OK:
        raise RuntimeError(f"oracle residual failed: {rc}")
    return out
