"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

* hand-worked examples (tests/golden/, each with its derivation);
* LAPACK getrf (scipy) at eps = 1: classic partial pivoting is the special
  case eps = 1 of the threshold rule of Section II-A, Algorithm 1;
* brute force on tiny matrices: a dense right-looking elimination with a
  boolean structure matrix (a different algorithm from the left-looking
  sparse one) must give the same pivots and factors;
* invariants: P A Q = L U within a backward-error bound, the threshold rule
  checked on the factors, uniqueness of L U for a fixed permutation,
  the residual of the solve (Algorithm 2), singular inputs.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2411_14082_gb300 import inputs
from tests.golden_io import dense_lu, load

U_ROUND = 2.0 ** -53


def dense_of(n, Ap, Ai, Ax):
    A = np.zeros((n, n))
    S = np.zeros((n, n), dtype=bool)
    for c in range(n):
        A[Ai[Ap[c]:Ap[c + 1]], c] = Ax[Ap[c]:Ap[c + 1]]
        S[Ai[Ap[c]:Ap[c + 1]], c] = True
    return A, S


# ---------------------------------------------------------------- golden
@pytest.mark.parametrize("name", ["mna_vsource_3x3.txt", "refactor_fail_col2_4x4.txt",
                                  "restart_recompute_3x3.txt", "repredict_cascade_3x3.txt"])
def test_golden_examples(name):
    g = load(name)
    n = g["n"]
    if "Ax0" in g:
        # the first factorization of the unperturbed values keeps every
        # preferred (diagonal) row, which is the pivot sequence preferred next
        lu0 = O.factorize(n, g["Ap"], g["Ai"], g["Ax0"], g["Q"], g["eps"])
        assert lu0.status == O.OK
        np.testing.assert_array_equal(lu0.piv, g["prefer"])
        assert lu0.n_rejected == 0
        lu = O.refactorize(lu0, g["Ap"], g["Ai"], g["Ax"])
    else:
        lu = O.factorize(n, g["Ap"], g["Ai"], g["Ax"], g["Q"], g["eps"], g["prefer"])
    assert lu.status == O.OK
    np.testing.assert_array_equal(lu.piv, g["piv"])
    assert lu.n_rejected == g["rejected"]
    _, L, U = lu.dense_factors()
    Lg, Ug = dense_lu(g)
    np.testing.assert_allclose(L, Lg, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(U, Ug, rtol=1e-15, atol=1e-15)
    if "x" in g:
        x = O.solve(lu, g["b"])
        np.testing.assert_allclose(x, g["x"], rtol=1e-15)


# ---------------------------------------------------------------- LAPACK
@pytest.mark.parametrize("n", [1, 2, 5, 12, 40])
@pytest.mark.parametrize("seed", range(5))
def test_eps1_dense_matches_lapack(n, seed):
    """eps = 1 on a dense matrix is LAPACK partial pivoting (getrf)."""
    rng = np.random.default_rng(1000 * n + seed)
    A = rng.normal(size=(n, n))
    _, Ap, Ai, Ax = inputs.dense_to_csc(A, np.ones((n, n), dtype=bool))
    lu = O.factorize(n, Ap, Ai, Ax, np.arange(n), eps=1.0)
    assert lu.status == O.OK
    P, Ls, Us = scipy.linalg.lu(A)          # A = P Ls Us
    piv_lapack = np.argmax(P, axis=0)       # row of A at step k
    np.testing.assert_array_equal(lu.piv, piv_lapack)
    _, L, U = lu.dense_factors()
    np.testing.assert_allclose(L, Ls, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(U, Us, rtol=1e-10, atol=1e-12 * np.abs(Us).max())


# ---------------------------------------------------------------- brute force
def dense_threshold_lu(A, S, Q, eps, prefer):
    """Right-looking dense elimination with the same pivot rule.

    Rows keep their original numbers; S tracks which entries are
    structurally nonzero (fill: S[r, c] |= S[r, k] & S[p, c]).
    Returns (piv, L, U) in step numbering, or None if singular.
    """
    n = len(Q)
    M = A[:, Q].astype(float).copy()
    T = S[:, Q].copy()
    qinv = np.empty(n, int)
    qinv[Q] = np.arange(n)
    pivotal = np.zeros(n, bool)
    step_of = np.full(n, -1)
    L = np.eye(n)
    U = np.zeros((n, n))
    piv = []
    for k in range(n):
        cand = [r for r in range(n) if not pivotal[r] and T[r, k]]
        pref = Q[k] if prefer is None else prefer[k]
        others = [abs(M[r, k]) for r in cand if r != pref]
        m = max(others) if others else 0.0
        if pref in cand and M[pref, k] != 0 and abs(M[pref, k]) >= eps * m:
            p = pref
        else:
            nz = [r for r in cand if abs(M[r, k]) > 0]
            if not nz:
                return None
            best = max(abs(M[r, k]) for r in nz)
            p = min((r for r in nz if abs(M[r, k]) == best), key=lambda r: qinv[r])
        piv.append(p)
        pivotal[p] = True
        step_of[p] = k
        for r in cand:
            if r == p:
                continue
            l = M[r, k] / M[p, k]
            M[r, k + 1:] -= l * M[p, k + 1:]
            T[r, k + 1:] |= T[p, k + 1:]
            M[r, k] = l
        for c in range(k, n):
            if T[p, c]:
                U[k, c] = M[p, c]
    for k in range(n):
        for r in range(n):
            if step_of[r] > k and T[r, k]:
                L[step_of[r], k] = M[r, k]
    return np.array(piv), L, U


@pytest.mark.parametrize("eps", [1e-3, 0.1, 1.0])
def test_tiny_random_vs_dense_right_looking(eps):
    rng = np.random.default_rng(7)
    checked = 0
    for trial in range(700):
        n = int(rng.integers(1, 9))
        density = rng.uniform(0.15, 0.8)
        _, Ap, Ai, Ax = inputs.random_sparse(n, density, rng, zero_diag_frac=0.3)
        Q = rng.permutation(n).astype(np.int32)
        A, S = dense_of(n, Ap, Ai, Ax)
        ref = dense_threshold_lu(A, S, Q, eps, None)
        lu = O.factorize(n, Ap, Ai, Ax, Q, eps)
        if ref is None:
            assert lu.status == O.ERR_SINGULAR
            continue
        assert lu.status == O.OK
        piv, Lr, Ur = ref
        np.testing.assert_array_equal(lu.piv, piv)
        _, L, U = lu.dense_factors()
        scale = max(1.0, np.abs(Ur).max())
        np.testing.assert_allclose(L, Lr, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(Lr).max()))
        np.testing.assert_allclose(U, Ur, rtol=1e-9, atol=1e-12 * scale)
        checked += 1
    assert checked > 300


def test_tiny_structure_matches_dense_fill():
    """Stored pattern = structural fill of the brute-force elimination."""
    rng = np.random.default_rng(11)
    for trial in range(300):
        n = int(rng.integers(2, 9))
        _, Ap, Ai, Ax = inputs.random_sparse(n, rng.uniform(0.2, 0.6), rng,
                                             zero_diag_frac=0.2, dominance=3.0)
        Q = np.arange(n, dtype=np.int32)
        lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
        if lu.status != O.OK:
            continue
        A, S = dense_of(n, Ap, Ai, Ax)
        # structural elimination with the oracle's pivot sequence
        T = S[lu.piv][:, Q].copy()
        for k in range(n):
            for r in range(k + 1, n):
                if T[r, k]:
                    T[r, k + 1:] |= T[k, k + 1:]
        for k in range(n):
            lrows = set(lu.Li[lu.Lp[k]:lu.Lp[k + 1]].tolist())
            urows = set(lu.Ui[lu.Up[k]:lu.Up[k + 1]].tolist())
            assert lrows == {r for r in range(k + 1, n) if T[r, k]}
            assert urows == {r for r in range(0, k + 1) if T[r, k]} | {k}


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("eps", [1e-3, 0.5])
def test_reconstruction_and_threshold_rule(eps):
    rng = np.random.default_rng(3)
    for trial in range(10000):
        n = int(rng.integers(1, 9))
        _, Ap, Ai, Ax = inputs.random_sparse(n, rng.uniform(0.2, 0.9), rng, zero_diag_frac=0.25)
        Q = rng.permutation(n).astype(np.int32)
        prefer = rng.permutation(n).astype(np.int32) if trial % 2 else None
        lu = O.factorize(n, Ap, Ai, Ax, Q, eps, prefer)
        if lu.status != O.OK:
            continue
        A, _ = dense_of(n, Ap, Ai, Ax)
        P, L, U = lu.dense_factors()
        err = np.abs(P @ A[:, Q] - L @ U).max()
        growth = max(1.0, np.abs(L).max() * np.abs(U).max() / max(np.abs(A).max(), 1e-300))
        assert err <= 10 * n * U_ROUND * np.abs(A).max() * growth
        # threshold rule on the factors: kept preferred rows keep |L| <= 1/eps,
        # argmax pivots keep |L| <= 1, and a rejected preferred candidate was
        # really below eps times the largest other candidate
        for k in range(n):
            pref = Q[k] if prefer is None else prefer[k]
            col = np.abs(lu.Lx[lu.Lp[k]:lu.Lp[k + 1]])
            if lu.piv[k] == pref:
                assert np.all(col <= 1.0 / eps * (1 + 1e-15))
            else:
                assert np.all(col <= 1.0)
                rows = lu.piv[lu.Li[lu.Lp[k]:lu.Lp[k + 1]]]
                if pref in rows:
                    lp = col[list(rows).index(pref)]
                    others = [c for r, c in zip(rows, col) if r != pref] + [1.0]
                    assert lp < eps * max(others) or lp == 0


def test_uniqueness_for_fixed_permutation():
    """With P and Q fixed, Doolittle elimination without pivoting of P A Q
    gives the same L and U (LU of a fixed permutation is unique)."""
    rng = np.random.default_rng(5)
    for trial in range(100):
        n = int(rng.integers(2, 10))
        _, Ap, Ai, Ax = inputs.random_sparse(n, 0.5, rng, zero_diag_frac=0.3)
        Q = rng.permutation(n).astype(np.int32)
        lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
        if lu.status != O.OK:
            continue
        A, _ = dense_of(n, Ap, Ai, Ax)
        B = A[lu.piv][:, Q]
        Ld, Ud = np.eye(n), np.zeros((n, n))
        for i in range(n):               # Doolittle, row by row
            for j in range(i, n):
                Ud[i, j] = B[i, j] - Ld[i, :i] @ Ud[:i, j]
            for j in range(i + 1, n):
                Ld[j, i] = (B[j, i] - Ld[j, :i] @ Ud[:i, i]) / Ud[i, i]
        _, L, U = lu.dense_factors()
        np.testing.assert_allclose(L, Ld, rtol=1e-9, atol=1e-10 * max(1, np.abs(Ld).max()))
        np.testing.assert_allclose(U, Ud, rtol=1e-9, atol=1e-10 * max(1, np.abs(Ud).max()))


def test_singular_and_bad_input():
    # zero column
    n, Ap, Ai, Ax = inputs.dense_to_csc(np.array([[1.0, 0.0], [2.0, 0.0]]),
                                        np.array([[True, False], [True, True]]))
    lu = O.factorize(n, Ap, Ai, Ax, np.arange(n), 1e-3)
    assert lu.status == O.ERR_SINGULAR and lu.bad_step == 1
    # structurally singular: two columns with the same single row
    n, Ap, Ai, Ax = inputs.dense_to_csc(np.array([[1.0, 1.0], [0.0, 0.0]]),
                                        np.array([[True, True], [False, False]]))
    lu = O.factorize(n, Ap, Ai, Ax, np.arange(n), 1e-3)
    assert lu.status == O.ERR_SINGULAR
    # Q not a permutation
    lu = O.factorize(n, Ap, Ai, Ax, np.array([0, 0]), 1e-3)
    assert lu.status == O.ERR_INPUT


def test_solve_matches_dense_solve():
    rng = np.random.default_rng(9)
    for trial in range(50):
        n = int(rng.integers(1, 30))
        _, Ap, Ai, Ax = inputs.random_sparse(n, 0.3, rng, zero_diag_frac=0.2, dominance=0.5)
        A, _ = dense_of(n, Ap, Ai, Ax)
        if np.linalg.cond(A) > 1e8:
            continue
        lu = O.factorize(n, Ap, Ai, Ax, rng.permutation(n), 1e-3)
        assert lu.status == O.OK
        b = rng.uniform(-1, 1, n)
        np.testing.assert_allclose(O.solve(lu, b), np.linalg.solve(A, b), rtol=1e-8, atol=1e-10)


# ---------------------------------------------------------------- MNA workload
def test_small_mna_workload_residual_and_refactor_sequence():
    """n = 2,020 MNA grid: first factorization, then 10 perturbed
    re-factorizations preferring the previous pivots; every solve meets the
    relative residual bound 1e-12."""
    ckt = inputs.workload_small()
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    rng = np.random.default_rng(inputs.BASE_SEED)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    assert lu.status == O.OK and lu.n_rejected > 0   # zero diagonals force pivoting
    b = inputs.rhs(n, rng)
    assert O.residual(n, Ap, Ai, Ax, O.solve(lu, b), b) <= 1e-12
    for it in range(10):
        ckt = inputs.perturb_elements(ckt, rng)
        Ax = ckt.values()
        lu2 = O.refactorize(lu, Ap, Ai, Ax)
        assert lu2.status == O.OK
        b = inputs.rhs(n, rng)
        assert O.residual(n, Ap, Ai, Ax, O.solve(lu2, b), b) <= 1e-12
        lu = lu2


def test_solution_matches_superlu_within_the_conditioning_bound():
    """The oracle's solution of the C1 grid and of a small RC mesh against
    SuperLU's (scipy.sparse.linalg.splu: its own ordering and pivoting, so
    only x is compared).  Two solutions with residuals r1, r2 differ by at
    most ||A^-1||_inf (||r1||_inf + ||r2||_inf); the bound uses a dense
    inverse of A, and each computed residual is widened by the rounding of
    its own evaluation (row length times unit roundoff times |A||x|)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    for ckt in (inputs.workload_small(), inputs.rc_mesh3d(12, 12, 4, seed=5, n_fet=30)):
        n, Ap, Ai, Ax = ckt.csc()
        A = sp.csc_matrix((Ax, Ai, Ap), shape=(n, n))
        lu = O.factorize(n, Ap, Ai, Ax, inputs.grid_nd_order(ckt), 1e-3)
        assert lu.status == O.OK
        b = inputs.rhs(n, np.random.default_rng(2))
        x_o = O.solve(lu, b)
        x_s = spla.splu(A).solve(b)
        absA = abs(A)
        row_len = np.diff(A.tocsr().indptr).max() + 1
        r_o = np.abs(b - A @ x_o).max() + row_len * U_ROUND * (absA @ np.abs(x_o) + np.abs(b)).max()
        r_s = np.abs(b - A @ x_s).max() + row_len * U_ROUND * (absA @ np.abs(x_s) + np.abs(b)).max()
        inv_norm = np.abs(np.linalg.inv(A.toarray())).sum(axis=1).max()
        assert np.abs(x_o - x_s).max() <= inv_norm * (r_o + r_s) * (1 + 1e-6)
        assert O.residual(n, Ap, Ai, Ax, x_o, b) <= 1e-12


# ---------------------------------------------------------------- residual
def test_residual_parts_exact_on_small_integer_systems():
    """||b - A x||_inf, ||A||_inf (largest row sum of |A|) and ||x||_inf of
    small integer systems, computed exactly with rationals: every partial
    sum is an integer below 2^53, so the oracle's float64 values must be
    exact, and the ratio must be their correctly rounded quotient."""
    from fractions import Fraction
    rng = np.random.default_rng(11)
    for trial in range(200):
        n = int(rng.integers(1, 12))
        _, Ap, Ai, Ax = inputs.random_sparse(n, 0.4, rng, zero_diag_frac=0.3, dominance=0.5)
        Ax = rng.integers(-50, 51, len(Ax)).astype(np.float64)
        x = rng.integers(-30, 31, n).astype(np.float64)
        b = rng.integers(-99, 100, n).astype(np.float64)
        r = [Fraction(int(v)) for v in b]
        rs = [Fraction(0)] * n
        for c in range(n):
            for p in range(Ap[c], Ap[c + 1]):
                r[Ai[p]] -= Fraction(int(Ax[p])) * int(x[c])
                rs[Ai[p]] += abs(Fraction(int(Ax[p])))
        rn = max(abs(v) for v in r)
        an = max(rs)
        xn = max(abs(int(v)) for v in x)
        out = O.residual_parts(n, Ap, Ai, Ax, x, b)
        assert out[1] == float(rn) and out[2] == float(an) and out[3] == float(xn)
        want = float(rn / (an * xn)) if an > 0 and xn > 0 else float(rn)
        assert out[0] == want


def test_residual_special_cases():
    """x = 0 gives ratio ||b||; A = 0 gives ratio ||b - 0||; the identity
    with x = b gives 0; a NaN anywhere in x or A makes the ratio NaN (the
    maximum of a set that holds a NaN is NaN), so it fails every bound."""
    n = 5
    Ap = np.arange(n + 1, dtype=np.int32)
    Ai = np.arange(n, dtype=np.int32)
    I = np.ones(n)
    b = np.array([1.0, -3.0, 2.0, 0.5, -0.25])
    out = O.residual_parts(n, Ap, Ai, I, np.zeros(n), b)
    assert out[0] == 3.0 and out[1] == 3.0 and out[2] == 1.0 and out[3] == 0.0
    out = O.residual_parts(n, Ap, Ai, np.zeros(n), b, b)
    assert out[0] == 3.0 and out[2] == 0.0
    assert O.residual_parts(n, Ap, Ai, I, b, b)[0] == 0.0
    for pos in range(n):
        x = b.copy()
        x[pos] = np.nan
        out = O.residual_parts(n, Ap, Ai, I, x, b)
        assert np.isnan(out[0]) and np.isnan(out[1]) and np.isnan(out[3])
        A = I.copy()
        A[pos] = np.nan
        out = O.residual_parts(n, Ap, Ai, A, b, b)
        assert np.isnan(out[0]) and np.isnan(out[2])
