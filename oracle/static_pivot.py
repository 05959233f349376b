"""Static pivoting and scaling -- test infrastructure only (the product path
never imports this module).

The optional pre-processing of CKTSO Section III-A: a row permutation that
maximizes the product of the diagonal magnitudes, and row/column scalings
that make those entries 1 in magnitude and every entry at most 1.

* ``max_product_matching(n, Ap, Ai, Ax)`` -- the definition written out: a
  minimum-cost assignment of rows to columns with cost
  log(max_i |a_ij|) - log|a_ij| on the nonzero entries, solved by scipy's
  ``linear_sum_assignment`` on the dense cost matrix (a library primitive;
  small n only).  Returns (match, objective) with match[j] = row of column j
  and objective = sum_j log|a_{match[j], j}|, the unique optimum value (the
  permutation itself need not be unique).
* ``brute_force_matching`` -- every permutation, for n <= 7.
* ``check_scaling`` -- the properties the scalings must have.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.optimize import linear_sum_assignment


def _dense(n, Ap, Ai, Ax):
    A = np.zeros((n, n))
    for j in range(n):
        for e in range(Ap[j], Ap[j + 1]):
            A[Ai[e], j] = Ax[e]
    return A


def max_product_matching(n, Ap, Ai, Ax):
    A = np.abs(_dense(n, Ap, Ai, Ax))
    if np.any(A.max(axis=0) == 0.0):
        return None, None
    with np.errstate(divide="ignore"):
        logs = np.where(A > 0, np.log(np.where(A > 0, A, 1.0)), -np.inf)
    big = 1e300
    cost = np.where(np.isfinite(logs), logs.max(axis=0)[None, :] - logs, big)
    rows, cols = linear_sum_assignment(cost)
    if np.any(cost[rows, cols] >= big):
        return None, None   # structurally singular on the nonzero entries
    match = np.empty(n, np.int64)
    match[cols] = rows
    return match, float(logs[match, np.arange(n)].sum())


def brute_force_matching(n, Ap, Ai, Ax):
    A = np.abs(_dense(n, Ap, Ai, Ax))
    best, arg = -np.inf, None
    for p in itertools.permutations(range(n)):
        d = A[list(p), range(n)]
        if np.all(d > 0):
            v = float(np.log(d).sum())
            if v > best:
                best, arg = v, np.array(p)
    return arg, (best if arg is not None else None)


def check_scaling(n, Ap, Ai, Ax, match, dr, dc, tol=1e-12):
    """|dr_i a_ij dc_j| <= 1 everywhere and == 1 on the matching."""
    A = _dense(n, Ap, Ai, Ax)
    S = np.abs(dr[:, None] * A * dc[None, :])
    ok_bound = bool(np.all(S <= 1.0 + tol))
    ok_diag = bool(np.allclose(S[match, np.arange(n)], 1.0, rtol=0, atol=tol))
    return ok_bound, ok_diag
