"""CPU checks of the library's host-side logic and of its C ABI.

No device work: the library is loaded (libcudart is linked but no GPU is
needed for these calls), every symbol declared in include/gblu.h must be
exported, and the host-only helpers (column elimination tree, restart set,
levels, minimum-degree order) are checked against brute force.
"""
import os
import re

import numpy as np
import pytest

from paper_2411_14082_gb300 import gblu, inputs
from tests.golden_io import load as load_golden

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "gblu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gblu_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = gblu.load()
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/gblu.h but not exported"
    assert set(names) == set(gblu.EXPORTED)


def dense_pattern(n, Ap, Ai):
    S = np.zeros((n, n), dtype=bool)
    for c in range(n):
        S[Ai[Ap[c]:Ap[c + 1]], c] = True
    return S


def brute_etree_of(M):
    """Elimination tree of a symmetric boolean pattern M by symbolic Cholesky:
    parent(j) = first row below the diagonal of column j of the factor."""
    n = len(M)
    L = np.tril(M | M.T).copy()
    np.fill_diagonal(L, True)
    for k in range(n):   # fill rule: L(a, b) |= L(a, k) & L(b, k) for k < b < a
        rows = np.nonzero(L[k + 1:, k])[0] + k + 1
        for a in rows:
            for b in rows:
                if a > b:
                    L[a, b] = True
    parent = np.full(n, -1)
    for j in range(n):
        below = np.nonzero(L[j + 1:, j])[0]
        if len(below):
            parent[j] = below[0] + j + 1
    return parent


@pytest.mark.parametrize("seed", range(40))
def test_column_etree_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 14))
    _, Ap, Ai, _ = inputs.random_sparse(n, rng.uniform(0.1, 0.5), rng, zero_diag_frac=0.3)
    Q = rng.permutation(n).astype(np.int32)
    S = dense_pattern(n, Ap, Ai)[:, Q].astype(int)
    AtA = (S.T @ S) > 0
    np.testing.assert_array_equal(gblu.column_etree(n, Ap, Ai, Q), brute_etree_of(AtA))


def test_restart_set_golden_and_brute_force():
    g = load_golden("restart_recompute_3x3.txt")
    parent = gblu.column_etree(g["n"], g["Ap"], g["Ai"], g["Q"])
    np.testing.assert_array_equal(parent, g["etree_parent"])
    finished = np.array([0, 1, 1], dtype=np.uint8)   # column 0 failed, 1 and 2 finished
    rs = gblu.restart_set(parent, finished)
    np.testing.assert_array_equal(np.nonzero(rs)[0], g["restart_set"])
    rng = np.random.default_rng(0)
    for trial in range(200):
        n = int(rng.integers(1, 30))
        parent = np.array([rng.integers(k + 1, n + 1) if k < n - 1 else n for k in range(n)])
        parent = np.where(parent >= n, -1, parent).astype(np.int32)
        finished = (rng.random(n) < 0.7).astype(np.uint8)
        expect = np.zeros(n, bool)
        for k in range(n):
            if not finished[k]:
                j = k
                while j != -1:
                    expect[j] = True
                    j = parent[j]
        np.testing.assert_array_equal(gblu.restart_set(parent, finished), expect)


def test_levels_are_longest_path():
    rng = np.random.default_rng(1)
    for trial in range(50):
        n = int(rng.integers(1, 40))
        Up = [0]
        Ui = []
        deps = []
        for k in range(n):
            d = sorted(set(rng.integers(0, k, size=int(rng.integers(0, 4))).tolist())) if k else []
            deps.append(d)
            Ui += d + [k]
            Up.append(len(Ui))
        lv, nl = gblu.levels(n, np.array(Up), np.array(Ui))
        expect = np.zeros(n, int)
        for k in range(n):
            expect[k] = max([expect[j] + 1 for j in deps[k]], default=0)
        np.testing.assert_array_equal(lv, expect)
        assert nl == expect.max() + 1


def symbolic_fill(n, Ap, Ai, Q):
    """nnz(L+U) of A(Q,Q)+A(Q,Q)^T with diagonal pivots (brute force)."""
    S = dense_pattern(n, Ap, Ai)
    S = S | S.T
    S = S[np.ix_(Q, Q)]
    np.fill_diagonal(S, True)
    for k in range(n):
        rows = np.nonzero(S[k + 1:, k])[0] + k + 1
        S[np.ix_(rows, rows)] = True
    return int(S.sum())


def test_mindeg_is_permutation_and_reduces_fill():
    ckt = inputs.mna_grid2d(12, 12, n_vsrc=3)
    n, Ap, Ai, _ = ckt.csc()
    perm = gblu.order_mindeg(n, Ap, Ai)
    assert sorted(perm.tolist()) == list(range(n))
    fill_md = symbolic_fill(n, Ap, Ai, perm)
    fill_nat = symbolic_fill(n, Ap, Ai, np.arange(n))
    assert fill_md < 0.8 * fill_nat


def test_mindeg_on_arrow_matrix_orders_hub_last():
    n = 30
    A = np.eye(n)
    A[0, :] = 1
    A[:, 0] = 1
    _, Ap, Ai, _ = inputs.dense_to_csc(A)
    perm = gblu.order_mindeg(n, Ap, Ai)
    assert perm[-1] == 0 or perm[-2] == 0   # the dense hub is eliminated (nearly) last


def test_invalid_patterns_rejected_on_host():
    with pytest.raises(gblu.GbluError):
        gblu.column_etree(2, np.array([0, 1, 2]), np.array([0, 5]))   # row out of range
    with pytest.raises(gblu.GbluError):
        gblu.column_etree(2, np.array([0, 2, 2]), np.array([1, 1]))   # duplicate
    with pytest.raises(gblu.GbluError):
        gblu.order_mindeg(2, np.array([1, 1, 2]), np.array([0, 1]))   # Ap[0] != 0


def test_server_argument_errors_without_a_device():
    """Host-side argument checks of the solve server (no device needed)."""
    import ctypes
    lib = gblu.load()
    s = ctypes.c_void_p()
    assert lib.gblu_server_create(ctypes.byref(s), 0, 0, 4, None) == gblu.ERR_INVALID_INPUT
    assert lib.gblu_server_create(ctypes.byref(s), 0, 1 << 30, 0, None) == gblu.ERR_INVALID_INPUT
    assert lib.gblu_server_create(ctypes.byref(s), 999, 1 << 30, 4, None) == gblu.ERR_CUDA
    assert b"not available" in lib.gblu_server_last_error()
    assert lib.gblu_server_submit(None, 0, None, None, None, 0, None) == gblu.ERR_INVALID_INPUT
    lib.gblu_server_destroy(None)


def test_nested_dissection_order():
    """gblu_order_nd: a deterministic permutation whose symmetric fill on a
    mesh is close to the coordinate bisection of the generator and well
    below minimum degree; on a path graph it is the optimum-fill family
    (separators last, no fill at all)."""
    ckt = inputs.rc_mesh3d(40, 40, 4, seed=3, n_fet=80)
    n, Ap, Ai, _ = ckt.csc()
    q1 = gblu.order_nd(n, Ap, Ai)
    q2 = gblu.order_nd(n, Ap, Ai)
    assert np.array_equal(q1, q2)
    assert sorted(q1.tolist()) == list(range(n))
    f_nd = gblu.symmetric_fill(n, Ap, Ai, q1)
    f_geo = gblu.symmetric_fill(n, Ap, Ai, inputs.grid_nd_order(ckt))
    f_md = gblu.symmetric_fill(n, Ap, Ai, gblu.order_mindeg(n, Ap, Ai))
    assert f_nd <= 1.3 * f_geo and f_nd <= 1.2 * f_md
    # tridiagonal (a path): any order from dissection keeps the fill at n-1
    m = 3000
    rows = [np.array([j - 1, j, j + 1]) for j in range(m)]
    rows = [r[(r >= 0) & (r < m)] for r in rows]
    Ap2 = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    Ai2 = np.concatenate(rows).astype(np.int32)
    q = gblu.order_nd(m, Ap2, Ai2)
    assert sorted(q.tolist()) == list(range(m))
    assert gblu.symmetric_fill(m, Ap2, Ai2, q) <= 2 * (m - 1)


def test_default_options_match_the_header():
    """gblu_default_opts fills the structure the binding declares: the last
    fields land where the library writes them."""
    import ctypes
    lib = gblu.load()
    o = gblu.Opts()
    lib.gblu_default_opts(ctypes.byref(o))
    assert o.pivot_tol == 1e-3 and o.alpha == 2.0 and o.spin_limit == 1 << 24
    assert o.solve_dense_density == 0.9 and o.solve_slices == 8
    assert o.warp_column_max == 640 and o.speculate_first == 2
    # an out-of-range switch is rejected before any device work
    o.speculate_first = 3
    h = ctypes.c_void_p()
    assert lib.gblu_create(ctypes.byref(h), 0, ctypes.byref(o)) == gblu.ERR_INVALID_INPUT


def brute_cost(n, Ap, Ai, Q):
    """(strict lower entries, flops sum_j 2 c_j^2) of the symbolic Cholesky
    factor of (A + A^T)(Q,Q), by dense boolean elimination."""
    S = dense_pattern(n, Ap, Ai)
    S = S | S.T
    S = S[np.ix_(Q, Q)]
    np.fill_diagonal(S, True)
    counts = np.zeros(n, np.int64)
    for k in range(n):
        rows = np.nonzero(S[k + 1:, k])[0] + k + 1
        counts[k] = len(rows)
        S[np.ix_(rows, rows)] = True
    return int(counts.sum()), float(2 * (counts.astype(float) ** 2).sum())


def test_symmetric_cost_against_brute_force():
    rng = np.random.default_rng(17)
    for trial in range(30):
        n = int(rng.integers(1, 60))
        _, Ap, Ai, _ = inputs.random_sparse(n, rng.uniform(0.02, 0.2), rng)
        Q = rng.permutation(n).astype(np.int32)
        fill, flops = gblu.symmetric_cost(n, Ap, Ai, Q)
        bf, bfl = brute_cost(n, Ap, Ai, Q)
        assert fill == bf and flops == bfl
        assert gblu.symmetric_fill(n, Ap, Ai, Q) == bf
    with pytest.raises(gblu.GbluError):
        gblu.symmetric_cost(3, np.array([0, 1, 2, 3]), np.array([0, 1, 2]), np.array([0, 0, 1]))


def boolean_lu(B):
    """Pattern of the LU factors of the square boolean matrix B (diagonal
    set) without row exchanges: dense boolean right-looking elimination."""
    B = B.copy()
    np.fill_diagonal(B, True)
    n = len(B)
    for k in range(n):
        rows = np.nonzero(B[k + 1:, k])[0] + k + 1
        cols = np.nonzero(B[k, k + 1:])[0] + k + 1
        B[np.ix_(rows, cols)] = True
    return B


def structure_pattern(n, LUp, LUi, nU):
    """Dense boolean L + U of a structure in step numbering; also checks the
    column layout: U rows ascending, the diagonal last, L rows ascending."""
    M = np.zeros((n, n), dtype=bool)
    for k in range(n):
        col = LUi[LUp[k]:LUp[k + 1]]
        u, low = col[:nU[k]], col[nU[k]:]
        assert u[-1] == k and np.all(np.diff(u) > 0) and np.all(u < k + 1)
        assert np.all(np.diff(low) > 0) and np.all(low > k)
        M[col, k] = True
    return M


def test_predicted_first_structure():
    """gblu_symmetric_structure (the structure the first factorization
    predicts) is the Cholesky pattern of (A + A^T)(Q,Q) for L and U^T,
    found here by dense boolean elimination; it contains the pattern of the
    LU factors of A(Q,Q) without row exchanges and equals it when A is
    structurally symmetric."""
    rng = np.random.default_rng(29)
    for trial in range(40):
        n = int(rng.integers(1, 60))
        _, Ap, Ai, _ = inputs.random_sparse(n, rng.uniform(0.02, 0.2), rng)
        if trial % 2:   # structurally symmetric
            _, Ap, Ai, _ = inputs.dense_to_csc(np.ones((n, n)), (lambda m: m | m.T)(dense_pattern(n, Ap, Ai)))
        Q = rng.permutation(n).astype(np.int32)
        LUp, LUi, nU = gblu.symmetric_structure(n, Ap, Ai, Q)
        M = structure_pattern(n, LUp, LUi, nU)
        A = dense_pattern(n, Ap, Ai)
        chol = boolean_lu((A | A.T)[np.ix_(Q, Q)])
        assert np.array_equal(M, chol)
        assert np.array_equal(M, M.T)
        exact = boolean_lu(A[np.ix_(Q, Q)])
        assert not np.any(exact & ~M)
        if trial % 2:
            assert np.array_equal(M, exact)
    with pytest.raises(gblu.GbluError):
        gblu.symmetric_structure(3, np.array([0, 1, 2, 3]), np.array([0, 1, 2]), np.array([0, 0, 1]))


def test_predicted_structure_holds_the_oracle_factors():
    """On diagonally dominant values the oracle keeps every diagonal row
    (Algorithm 1 with the threshold rule), and its L and U lie inside the
    predicted structure."""
    from oracle import oracle as O
    rng = np.random.default_rng(31)
    for trial in range(10):
        n = int(rng.integers(5, 80))
        _, Ap, Ai, Ax = inputs.random_sparse(n, rng.uniform(0.03, 0.15), rng, dominance=4.0 * n)
        Q = rng.permutation(n).astype(np.int32)
        lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
        assert lu.status == O.OK and np.array_equal(lu.piv, Q)
        M = structure_pattern(n, *gblu.symmetric_structure(n, Ap, Ai, Q))
        for part in ("L", "U"):
            p, i = np.asarray(getattr(lu, part + "p"), np.int64), getattr(lu, part + "i")
            cols = np.repeat(np.arange(n), np.diff(p))
            assert np.all(M[i, cols]), part


def test_predicted_structure_for_given_rows():
    """gblu_predicted_structure with pivot rows piv (the structure a restart
    predicts after pivot exchanges) is the Cholesky pattern of B + B^T for
    B = A(piv, Q), found by dense boolean elimination; it contains the
    pattern of B's LU factors without row exchanges, also where B has
    structurally zero diagonal entries (fill makes them nonzero), and the
    oracle's factors whenever the oracle keeps the rows piv (Algorithm 1
    with those rows preferred and a tiny threshold).  piv = Q is
    gblu_symmetric_structure."""
    from oracle import oracle as O
    rng = np.random.default_rng(37)
    kept = kept_zero = zero_diag = 0
    for trial in range(120):
        n = int(rng.integers(2, 50))
        _, Ap, Ai, Ax = inputs.random_sparse(n, rng.uniform(0.05, 0.3), rng, dominance=2.0)
        Q = rng.permutation(n).astype(np.int32)
        piv = Q.copy()
        for _ in range(int(rng.integers(1, 4))):   # a few exchanges of two steps' rows
            a, b = rng.choice(n, 2, replace=False)
            piv[a], piv[b] = piv[b], piv[a]
        M = structure_pattern(n, *gblu.predicted_structure(n, Ap, Ai, Q, piv))
        A = dense_pattern(n, Ap, Ai)
        B = A[np.ix_(piv, Q)]
        zd = bool(np.any(~np.diag(B)))
        zero_diag += zd
        assert np.array_equal(M, boolean_lu(B | B.T))
        assert not np.any(boolean_lu(B) & ~M)
        lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-12, prefer=piv)
        if lu.status == O.OK and np.array_equal(lu.piv, piv):
            kept += 1
            kept_zero += zd
            for part in ("L", "U"):
                p, i = np.asarray(getattr(lu, part + "p"), np.int64), getattr(lu, part + "i")
                cols = np.repeat(np.arange(n), np.diff(p))
                assert np.all(M[i, cols]), part
    assert kept >= 25 and kept_zero >= 15 and zero_diag >= 80
    _, Ap, Ai, _ = inputs.random_sparse(30, 0.1, rng)
    Q = rng.permutation(30).astype(np.int32)
    for got, want in zip(gblu.predicted_structure(30, Ap, Ai, Q, None), gblu.symmetric_structure(30, Ap, Ai, Q)):
        assert np.array_equal(got, want)
    with pytest.raises(gblu.GbluError):
        gblu.predicted_structure(3, np.array([0, 1, 2, 3]), np.array([0, 1, 2]), np.arange(3), np.array([0, 0, 1]))


def test_levels_of_predicted_structures_are_tree_heights():
    """On a Cholesky-pattern structure (gblu_predicted_structure, with or
    without pivot exchanges) the EGraph level of a column (gblu_levels over
    its U rows) is its height in the elimination tree, the tree's parent of
    j being the first L row of column j: the schedule computes the levels of
    predicted structures that way."""
    rng = np.random.default_rng(41)
    for trial in range(40):
        n = int(rng.integers(1, 120))
        _, Ap, Ai, _ = inputs.random_sparse(n, rng.uniform(0.01, 0.2), rng)
        Q = rng.permutation(n).astype(np.int32)
        piv = None
        if trial % 2:
            piv = Q.copy()
            a, b = rng.choice(n, 2) if n > 1 else (0, 0)
            piv[a], piv[b] = piv[b], piv[a]
        LUp, LUi, nU = gblu.predicted_structure(n, Ap, Ai, Q, piv)
        Up = np.zeros(n + 1, np.int64)
        Up[1:] = np.cumsum(nU)
        Ui = np.concatenate([LUi[LUp[k]:LUp[k] + nU[k]] for k in range(n)]).astype(np.int32)
        lv, nl = gblu.levels(n, Up, Ui)
        height = np.zeros(n, np.int64)
        for j in range(n):
            if LUp[j] + nU[j] < LUp[j + 1]:
                p = LUi[LUp[j] + nU[j]]
                height[p] = max(height[p], height[j] + 1)
        assert np.array_equal(lv, height) and nl == height.max() + 1


def test_constrained_minimum_degree():
    """gblu_order_cmd: one group gives plain minimum degree; with groups the
    elimination order never goes back to a lower group, and a group
    overrides degree (the hubs of two stars, put in the first group, come
    first although every leaf has a lower degree)."""
    ckt = inputs.mna_grid2d(12, 12, n_vsrc=3)
    n, Ap, Ai, _ = ckt.csc()
    assert np.array_equal(gblu.order_cmd(n, Ap, Ai, np.zeros(n, np.int32)), gblu.order_mindeg(n, Ap, Ai))
    rng = np.random.default_rng(5)
    group = rng.integers(0, 5, n).astype(np.int32)
    perm = gblu.order_cmd(n, Ap, Ai, group)
    assert sorted(perm.tolist()) == list(range(n))
    assert np.all(np.diff(group[perm]) >= 0)
    # two stars (hubs 0 and 6, five leaves each) in group 0, nothing else
    m = 12
    A = np.eye(m)
    for hub, leaves in ((0, range(1, 6)), (6, range(7, 12))):
        for v in leaves:
            A[hub, v] = A[v, hub] = 1
    _, Ap2, Ai2, _ = inputs.dense_to_csc(A)
    p = gblu.order_cmd(m, Ap2, Ai2, np.zeros(m, np.int32))
    assert p[0] not in (0, 6)   # a leaf (degree 1) goes first without groups
    g = np.ones(m, np.int32)
    g[[0, 6]] = 0
    p = gblu.order_cmd(m, Ap2, Ai2, g)
    assert set(p[:2].tolist()) == {0, 6}
    with pytest.raises(gblu.GbluError):
        gblu.order_cmd(m, Ap2, Ai2, -np.ones(m, np.int32))


def test_constrained_nested_dissection_and_automatic_choice():
    """gblu_order_cnd orders a mesh with no more flops than plain nested
    dissection on it (the measured gain of Section III-A's constrained pass:
    0.550 against 0.565 GFLOP on this 60x60x4 mesh); gblu_order_auto returns
    the candidate of fewest flops and says which."""
    ckt = inputs.workload_mesh(nx=60, ny=60)
    n, Ap, Ai, _ = ckt.csc()
    q_nd = gblu.order_nd(n, Ap, Ai)
    q_cnd = gblu.order_cnd(n, Ap, Ai)
    assert sorted(q_cnd.tolist()) == list(range(n))
    assert np.array_equal(q_cnd, gblu.order_cnd(n, Ap, Ai))
    costs = {"mindeg": gblu.symmetric_cost(n, Ap, Ai, gblu.order_mindeg(n, Ap, Ai))[1],
             "amf": gblu.symmetric_cost(n, Ap, Ai, gblu.order_amf(n, Ap, Ai))[1],
             "nd": gblu.symmetric_cost(n, Ap, Ai, q_nd)[1],
             "cnd": gblu.symmetric_cost(n, Ap, Ai, q_cnd)[1]}
    assert costs["cnd"] <= costs["nd"]
    q, method = gblu.order_auto(n, Ap, Ai)
    assert costs[method] == min(costs.values())
    assert gblu.symmetric_cost(n, Ap, Ai, q)[1] == costs[method]
    # small circuit: the minimum-degree family is a candidate too
    ckt = inputs.workload_small()
    n, Ap, Ai, _ = ckt.csc()
    q, method = gblu.order_auto(n, Ap, Ai)
    best = min(gblu.symmetric_cost(n, Ap, Ai, f(n, Ap, Ai))[1]
               for f in (gblu.order_mindeg, gblu.order_amf, gblu.order_nd, gblu.order_cnd))
    assert gblu.symmetric_cost(n, Ap, Ai, q)[1] == best


def test_minimum_deficiency_order():
    """gblu_order_amf: a deterministic permutation that, on the C1 grid and
    on the bordered grid, costs fewer flops than minimum degree (measured:
    2.4 against 2.8 and 205 against 236 MFLOP), and on a path adds no fill."""
    for ckt in (inputs.workload_small(), inputs.bordered_grid()):
        n, Ap, Ai, _ = ckt.csc()
        q = gblu.order_amf(n, Ap, Ai)
        assert sorted(q.tolist()) == list(range(n))
        assert np.array_equal(q, gblu.order_amf(n, Ap, Ai))
        assert gblu.symmetric_cost(n, Ap, Ai, q)[1] < gblu.symmetric_cost(n, Ap, Ai, gblu.order_mindeg(n, Ap, Ai))[1]
    m = 500
    rows = [np.array([j - 1, j, j + 1]) for j in range(m)]
    rows = [r[(r >= 0) & (r < m)] for r in rows]
    Ap2 = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    Ai2 = np.concatenate(rows).astype(np.int32)
    q = gblu.order_amf(m, Ap2, Ai2)
    assert gblu.symmetric_fill(m, Ap2, Ai2, q) == m - 1


def test_every_order_is_a_permutation_on_random_patterns():
    """All ordering entry points on random patterns from 1 to 400 unknowns,
    unsymmetric, with empty rows and columns off the diagonal: each returns a
    permutation, and the automatic choice is the cheapest candidate."""
    rng = np.random.default_rng(31)
    fns = {"mindeg": gblu.order_mindeg, "amf": gblu.order_amf, "nd": gblu.order_nd, "cnd": gblu.order_cnd}
    for trial in range(40):
        n = int(rng.integers(1, 400))
        _, Ap, Ai, _ = inputs.random_sparse(n, rng.uniform(0.0, 0.05), rng)
        costs = {}
        for name, fn in fns.items():
            q = fn(n, Ap, Ai)
            assert sorted(q.tolist()) == list(range(n)), name
            costs[name] = gblu.symmetric_cost(n, Ap, Ai, q)[1]
        q, method = gblu.order_auto(n, Ap, Ai)
        assert sorted(q.tolist()) == list(range(n))
        assert costs[method] == min(costs.values())


def test_orders_of_degenerate_patterns():
    """One unknown, a diagonal matrix, a matrix with an empty column and a
    dense block: every order is a permutation and the estimate is exact."""
    cases = [(1, np.array([0, 1]), np.array([0])),
             (5, np.arange(6), np.arange(5)),
             (4, np.array([0, 2, 2, 4, 5]), np.array([0, 3, 1, 2, 3]))]
    m = 12
    _, Ap, Ai, _ = inputs.dense_to_csc(np.ones((m, m)))
    cases.append((m, Ap, Ai))
    for n, Ap, Ai in cases:
        for fn in (gblu.order_mindeg, gblu.order_amf, gblu.order_nd, gblu.order_cnd,
                   lambda n, Ap, Ai: gblu.order_auto(n, Ap, Ai)[0]):
            q = fn(n, np.asarray(Ap), np.asarray(Ai))
            assert sorted(q.tolist()) == list(range(n))
            assert gblu.symmetric_cost(n, Ap, Ai, q) == brute_cost(n, np.asarray(Ap), np.asarray(Ai), q)
    # a dense block fills completely whatever the order
    fill, flops = gblu.symmetric_cost(m, Ap, Ai, np.arange(m))
    assert fill == m * (m - 1) // 2 and flops == sum(2 * c * c for c in range(m))


def test_header_is_plain_c_and_links(tmp_path):
    """include/gblu.h is a C ABI: a C99 program that includes it compiles
    without warnings, links against the library and calls a host entry
    point."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = gblu.load()
    libdir = os.path.dirname(lib._name)
    src = tmp_path / "use_gblu.c"
    src.write_text('#include "gblu.h"\n'
                   "int main(void) {\n"
                   "    gblu_opts o;\n"
                   "    int32_t Ap[3] = {0, 2, 3}, Ai[3] = {0, 1, 1}, perm[2];\n"
                   "    gblu_default_opts(&o);\n"
                   "    if (o.pivot_tol != 1e-3) return 1;\n"
                   "    return gblu_order_mindeg(2, Ap, Ai, perm) == GBLU_OK ? 0 : 2;\n"
                   "}\n")
    exe = tmp_path / "use_gblu"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lgblu",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    assert subprocess.run([str(exe)]).returncode == 0


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: without the built library the binding raises."""
    monkeypatch.setattr(gblu, "_lib", None)
    monkeypatch.setattr(gblu._build, "LIB", os.path.join(ROOT, "no_such_dir", "libgblu.so"))
    with pytest.raises(OSError):
        gblu.load(build_if_missing=False)


def test_solve_partition_rule():
    """Section V-A's split of a triangle, on synthetic count profiles.

    Paper rule: P0 is the largest p whose trailing block [p, n) holds at
    least 70% of the entries and at least min_entries; density rule: the
    longest trailing block whose density stays at least the threshold.
    Slices: P0 and n included, consecutive, at most max_piece rows, each
    (but the last) closed at the first row where its entries reach an equal
    share of the block's."""
    rng = np.random.default_rng(12)
    for trial in range(200):
        n = int(rng.integers(2, 400))
        # per-column strict counts growing toward the end (a dense-ish tail)
        strict = np.minimum(np.arange(n)[::-1], rng.integers(0, 4, n) + (np.arange(n) > n * rng.uniform(0.3, 0.9)) * n)
        strict = np.minimum(strict, n - 1 - np.arange(n))
        count_from = np.concatenate([np.cumsum(strict[::-1])[::-1], [0]]).astype(np.int64)
        rowlen = (rng.integers(0, 5, n) + strict).astype(np.int64)
        total = count_from[0]
        min_entries = int(rng.integers(0, max(1, total)))
        slices = int(rng.integers(1, 9))
        max_piece = int(rng.integers(1, 60))
        # paper's rule
        p0, cut = gblu.solve_partition(count_from, rowlen, 0.0, 0.7, min_entries, slices, max_piece)
        want = n
        if total > 0:
            for p in range(n - 1, -1, -1):
                if count_from[p] >= 0.7 * total and count_from[p] >= min_entries:
                    want = p
                    break
        assert p0 == want
        if p0 < n:
            assert cut[0] == p0 and cut[-1] == n and np.all(np.diff(cut) > 0)
            assert np.all(np.diff(cut) <= max_piece)
            per = rowlen[p0:].sum() / slices
            for a, b in zip(cut[:-2], cut[1:-1]):
                acc = np.cumsum(rowlen[a:b])
                # closed at the first row reaching the share, or at max_piece rows
                assert acc[-1] >= per or b - a == max_piece
                assert len(acc) == 1 or acc[-2] < per
        else:
            assert len(cut) == 0
        # density rule
        d = float(rng.uniform(0.3, 1.0))
        p0, _ = gblu.solve_partition(count_from, rowlen, d, 0.7, min_entries, slices, max_piece)
        want = n
        for p in range(n - 2, -1, -1):
            m = n - p
            if count_from[p] < d * m * (m - 1) / 2:
                break
            want = p
        if want < n and count_from[want] < min_entries:
            want = n
        assert p0 == want


def test_solve_partition_hand_worked_profiles():
    """Section V-A's rule on profiles worked out by hand (not by a copy of
    the loops): P0, then the slice cuts, including the edge cases P0 = n-2,
    an empty triangle and a minimum count above the total.

    Profile: strict per-column counts [0, 1, 1, 2, 1, 0] give
    count_from = [5, 5, 4, 3, 1, 0, 0]; 70% of 5 is 3.5, so scanning p from
    n-1 down, p = 2 (4 entries) is the first position that holds enough.
    With min_entries 5 it is p = 1; with min_entries 6 no block qualifies."""
    cf = np.array([5, 5, 4, 3, 1, 0, 0], np.int64)
    rowlen = np.array([1, 2, 3, 1, 2, 1], np.int64)
    # rows 2..5 hold 3 + 1 + 2 + 1 = 7 entries; two slices of 3.5: the first
    # closes at row 3 (3, then 4 >= 3.5), the last runs to the end
    assert_p0_cut(cf, rowlen, 0.0, 4, 2, 10, 2, [2, 4, 6])
    # at most one row per slice
    assert_p0_cut(cf, rowlen, 0.0, 4, 2, 1, 2, [2, 3, 4, 5, 6])
    assert_p0_cut(cf, rowlen, 0.0, 5, 1, 10, 1, [1, 6])
    assert_p0_cut(cf, rowlen, 0.0, 6, 2, 10, 6, [])
    # an empty triangle has no trailing block
    assert_p0_cut(np.zeros(7, np.int64), rowlen, 0.0, 0, 2, 10, 6, [])
    # density rule, P0 = n - 2: strict counts [0, 0, 0, 1, 0] give
    # count_from = [1, 1, 1, 1, 0, 0]; the 2-row block [3, 5) has its one
    # entry (density 1), the 3-row block [2, 5) would need 3
    cf2 = np.array([1, 1, 1, 1, 0, 0], np.int64)
    rl2 = np.array([0, 0, 1, 1, 1], np.int64)
    assert_p0_cut(cf2, rl2, 1.0, 1, 8, 10, 3, [3, 4, 5])
    assert_p0_cut(cf2, rl2, 1.0, 2, 8, 10, 5, [])   # below the minimum count


def assert_p0_cut(count_from, rowlen, density, min_entries, slices, max_piece, p0_want, cut_want):
    p0, cut = gblu.solve_partition(count_from, rowlen, density, 0.7, min_entries, slices, max_piece)
    assert p0 == p0_want
    assert list(cut) == cut_want
