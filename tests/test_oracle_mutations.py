"""The oracle pins are strong enough to catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (on the CPU,
in a temporary directory), builds it, and requires that at least one pin
(golden examples, brute-force dense elimination, LAPACK at eps = 1, solve
against numpy, exact residuals of integer systems) rejects the planted build.
"""
import os
import subprocess

import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2411_14082_gb300 import inputs
from tests.golden_io import dense_lu, load
from tests.test_oracle import dense_of, dense_threshold_lu

SRC = os.path.join(os.path.dirname(O.__file__), "gp_oracle.c")

MUTATIONS = {
    "update_sign": ("x[L.i[e]] -= L.x[e] * xj;", "x[L.i[e]] += L.x[e] * xj;"),
    "dropped_eps": ("fabs(x[pref]) >= eps * m", "fabs(x[pref]) >= m"),
    "no_normalize": ("vec_push(&L, r, x[r] / d)", "vec_push(&L, r, x[r])"),
    "wrong_topo_order": ("for (int t = ntopo - 1; t >= 0; t--) {\n            int r = topo[t];\n            int j = pinv[r];\n            if (j < 0) continue;",
                         "for (int t = 0; t < ntopo; t++) {\n            int r = topo[t];\n            int j = pinv[r];\n            if (j < 0) continue;"),
    "tie_break": ("qinv[r] < qinv[best]", "qinv[r] > qinv[best]"),
    "l_row_numbering": ("lu->Li[e] = pinv[L.i[e]];", "lu->Li[e] = L.i[e];"),
    "solve_no_divide": ("double zk = y[k] / lu->Ux[dpos];", "double zk = y[k];"),
    "solve_no_perm_b": ("y[k] = b[lu->piv[k]];", "y[k] = b[k];"),
    "keep_zero_pivot": ("pref_cand && x[pref] != 0.0 && fabs", "pref_cand && fabs"),
    "residual_sign": ("r[Ai[p]] -= Ax[p] * x[c];", "r[Ai[p]] += Ax[p] * x[c];"),
    "residual_row_sum_no_abs": ("rs[Ai[p]] += fabs(Ax[p]);", "rs[Ai[p]] += Ax[p];"),
    "residual_col_sum": ("rs[Ai[p]] += fabs(Ax[p]);", "rs[c] += fabs(Ax[p]);"),
    "residual_nan_skipped": ("if (isnan(m) || isnan(v)) return NAN;", ""),
}


def _pins_pass(lib):
    """Run a compact version of every pin; False as soon as one fails."""
    # golden examples
    for name in ("mna_vsource_3x3.txt", "refactor_fail_col2_4x4.txt",
                 "restart_recompute_3x3.txt"):
        g = load(name)
        n = g["n"]
        if "Ax0" in g:
            lu0 = O.factorize(n, g["Ap"], g["Ai"], g["Ax0"], g["Q"], g["eps"], lib=lib)
            lu = O.refactorize(lu0, g["Ap"], g["Ai"], g["Ax"])
        else:
            lu = O.factorize(n, g["Ap"], g["Ai"], g["Ax"], g["Q"], g["eps"], g["prefer"], lib=lib)
        if lu.status != O.OK or not np.array_equal(lu.piv, g["piv"]):
            return False
        _, L, U = lu.dense_factors()
        Lg, Ug = dense_lu(g)
        if not (np.allclose(L, Lg, rtol=1e-14, atol=1e-15) and np.allclose(U, Ug, rtol=1e-14, atol=1e-15)):
            return False
        if "x" in g and not np.allclose(O.solve(lu, g["b"]), g["x"], rtol=1e-14):
            return False
    # LAPACK at eps = 1
    rng = np.random.default_rng(1)
    for n in (5, 12):
        A = rng.normal(size=(n, n))
        _, Ap, Ai, Ax = inputs.dense_to_csc(A, np.ones((n, n), dtype=bool))
        lu = O.factorize(n, Ap, Ai, Ax, np.arange(n), eps=1.0, lib=lib)
        P, Ls, Us = scipy.linalg.lu(A)
        if lu.status != O.OK or not np.array_equal(lu.piv, np.argmax(P, axis=0)):
            return False
        _, L, U = lu.dense_factors()
        if not (np.allclose(L, Ls, atol=1e-10) and np.allclose(U, Us, atol=1e-10)):
            return False
        b = rng.uniform(-1, 1, n)
        if not np.allclose(O.solve(lu, b), np.linalg.solve(A, b), rtol=1e-8, atol=1e-10):
            return False
    # residual: exact on small integer systems, NaN propagates
    from fractions import Fraction
    for trial in range(40):
        n = int(rng.integers(1, 9))
        _, Ap, Ai, Ax = inputs.random_sparse(n, 0.5, rng, zero_diag_frac=0.3, dominance=0.5)
        Ax = rng.integers(-9, 10, len(Ax)).astype(np.float64)
        x = rng.integers(-9, 10, n).astype(np.float64)
        b = rng.integers(-9, 10, n).astype(np.float64)
        r = [Fraction(int(v)) for v in b]
        rs = [Fraction(0)] * n
        for c in range(n):
            for p in range(Ap[c], Ap[c + 1]):
                r[Ai[p]] -= int(Ax[p]) * int(x[c])
                rs[Ai[p]] += abs(int(Ax[p]))
        out = O.residual_parts(n, Ap, Ai, Ax, x, b, lib=lib)
        if (out[1], out[2], out[3]) != (float(max(abs(v) for v in r)), float(max(rs)),
                                        float(np.abs(x).max())):
            return False
    xn = np.array([1.0, np.nan, 2.0])
    if not np.isnan(O.residual_parts(3, np.arange(4), np.arange(3), np.ones(3), xn, np.ones(3), lib=lib)[0]):
        return False
    # brute force on tiny matrices, real and small-integer values (ties)
    for trial in range(300):
        n = int(rng.integers(1, 8))
        _, Ap, Ai, Ax = inputs.random_sparse(n, rng.uniform(0.2, 0.8), rng, zero_diag_frac=0.3)
        if trial % 2:
            Ax = rng.choice([-2.0, -1.0, 1.0, 2.0], size=len(Ax))
        Q = rng.permutation(n).astype(np.int32)
        A, S = dense_of(n, Ap, Ai, Ax)
        ref = dense_threshold_lu(A, S, Q, 0.1, None)
        lu = O.factorize(n, Ap, Ai, Ax, Q, 0.1, lib=lib)
        if ref is None:
            if lu.status != O.ERR_SINGULAR:
                return False
            continue
        if lu.status != O.OK or not np.array_equal(lu.piv, ref[0]):
            return False
        _, L, U = lu.dense_factors()
        if not (np.allclose(L, ref[1], rtol=1e-9, atol=1e-12) and np.allclose(U, ref[2], rtol=1e-9, atol=1e-12)):
            return False
    return True


def test_unmodified_oracle_passes_compact_pins():
    assert _pins_pass(O._load())


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "gp_oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(mutated), "-lm"])
    assert not _pins_pass(O.load_library(str(so)))
