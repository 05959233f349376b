"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (FP64): factor entries to 1e-10 relative to the column's
inf-norm, identical pivot sequences, relative residual
||b - A x||_inf / (||A||_inf ||x||_inf) <= 1e-12 for every solve.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_14082_gb300 import gblu, inputs
from tests.factor_compare import compare_factors
from tests.golden_io import dense_lu, load

pytestmark = pytest.mark.gpu

DEV = 0
RTOL = 1e-10
RESID = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(f"cuda:{DEV}")


def solve_and_check(s, n, Ap, Ai, Ax, Axd, rng):
    b = inputs.rhs(n, rng)
    x = s.solve(dev(b))
    res = s.residual(Axd, dev(b), x).cpu().numpy()
    xh = x.cpu().numpy()
    assert res[0] <= RESID, f"device residual {res[0]:.3e}"
    assert O.residual(n, Ap, Ai, Ax, xh, b) <= RESID
    return xh, b


@pytest.mark.parametrize("name", ["mna_vsource_3x3.txt", "refactor_fail_col2_4x4.txt",
                                  "restart_recompute_3x3.txt"])
def test_golden_examples_on_gpu(name):
    g = load(name)
    n = g["n"]
    s = gblu.Solver(DEV, pivot_tol=g["eps"])
    s.analyze(n, g["Ap"], g["Ai"], g["Q"])
    if "Ax0" in g:
        s.factorize(dev(g["Ax0"]))
        assert np.array_equal(s.export_factors()["piv"], g["prefer"])
        rc, rep = s.refactorize(dev(g["Ax"]))
        assert rc == gblu.REPIVOTED and rep
    else:
        s.factorize(dev(g["Ax"]))
    f = s.export_factors()
    np.testing.assert_array_equal(f["piv"], g["piv"])
    L = np.eye(n)
    U = np.zeros((n, n))
    for k in range(n):
        L[f["Li"][f["Lp"][k]:f["Lp"][k + 1]], k] = f["Lx"][f["Lp"][k]:f["Lp"][k + 1]]
        U[f["Ui"][f["Up"][k]:f["Up"][k + 1]], k] = f["Ux"][f["Up"][k]:f["Up"][k + 1]]
    Lg, Ug = dense_lu(g)
    np.testing.assert_allclose(L, Lg, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(U, Ug, rtol=1e-15, atol=1e-15)
    if "x" in g:
        x = s.solve(dev(g["b"])).cpu().numpy()
        np.testing.assert_allclose(x, g["x"], rtol=1e-15)
    if name == "restart_recompute_3x3.txt":
        st = s.stats()
        assert st["n_restart_cols"] == len(g["restart_set"]) and st["last_first_bad"] == 0


def well_conditioned(n, Ap, Ai, Ax, limit=1e12):
    """Pivot choices among rounding noise are arbitrary: compare only
    matrices whose condition number is far from 1/eps_machine."""
    A = np.zeros((n, n))
    for c in range(n):
        A[Ai[Ap[c]:Ap[c + 1]], c] = Ax[Ap[c]:Ap[c + 1]]
    return np.linalg.cond(A) < limit


@pytest.mark.parametrize("sched", ["auto", "level", "syncfree"])
def test_random_small_matrices_factorize_and_refactorize(sched):
    rng = np.random.default_rng(42)
    for trial in range(60):
        n = int(rng.integers(1, 80))
        _, Ap, Ai, Ax = inputs.random_sparse(n, rng.uniform(0.02, 0.3), rng,
                                             zero_diag_frac=rng.uniform(0, 0.3), dominance=1.0)
        Q = rng.permutation(n).astype(np.int32)
        if not well_conditioned(n, Ap, Ai, Ax):
            continue
        lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
        s = gblu.Solver(DEV, sched_mode=sched, solve_mode=sched)
        s.analyze(n, Ap, Ai, Q)
        if lu.status == O.ERR_SINGULAR:
            with pytest.raises(gblu.GbluError) as ei:
                s.factorize(dev(Ax))
            assert ei.value.code == gblu.ERR_SINGULAR
            continue
        Axd = dev(Ax)
        s.factorize(Axd)
        compare_factors(s.export_factors(), lu, RTOL)
        solve_and_check(s, n, Ap, Ai, Ax, Axd, rng)
        for it in range(3):
            Ax2 = inputs.perturb_entries(Ax, rng, frac=0.3, sigma=1.0)
            if not well_conditioned(n, Ap, Ai, Ax2):
                break
            lu2 = O.refactorize(lu, Ap, Ai, Ax2)
            Axd2 = dev(Ax2)
            if lu2.status != O.OK:
                with pytest.raises(gblu.GbluError):
                    s.refactorize(Axd2)
                break
            rc, rep = s.refactorize(Axd2)
            assert rep == (lu2.n_rejected > 0)
            compare_factors(s.export_factors(), lu2, RTOL)
            solve_and_check(s, n, Ap, Ai, Ax2, Axd2, rng)
            lu = lu2


def test_column_scaled_ill_conditioned_matrices():
    """Random matrices with their columns scaled by 10^U(-13, 0): condition
    numbers far above the 1e12 the random tests above keep, yet the pivot
    sequence is that of the unscaled matrix (the threshold test compares
    entries of one column, and the factors of A D are L and U D), so the
    factors must still equal the oracle's."""
    rng = np.random.default_rng(43)
    seen = 0
    for trial in range(60):
        n = int(rng.integers(2, 60))
        _, Ap, Ai, Ax = inputs.random_sparse(n, rng.uniform(0.05, 0.3), rng,
                                             zero_diag_frac=rng.uniform(0, 0.3), dominance=1.0)
        if not well_conditioned(n, Ap, Ai, Ax):
            continue
        scale = 10.0 ** rng.uniform(-13, 0, n)
        Ax = Ax * np.repeat(scale, np.diff(Ap))
        seen += not well_conditioned(n, Ap, Ai, Ax, limit=1e12)
        Q = rng.permutation(n).astype(np.int32)
        lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
        if lu.status != O.OK:
            continue
        s = gblu.Solver(DEV)
        s.analyze(n, Ap, Ai, Q)
        Axd = dev(Ax)
        s.factorize(Axd)
        compare_factors(s.export_factors(), lu, RTOL)
        solve_and_check(s, n, Ap, Ai, Ax, Axd, rng)
    assert seen >= 20


def test_small_mna_workload_sequence():
    """n = 2,020 MNA grid with voltage sources: 1 factorize, then 10
    refactorizations with 5% of the element conductances perturbed
    (log-normal, sigma 0.3), each followed by a solve."""
    ckt = inputs.workload_small()
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    rng = np.random.default_rng(inputs.BASE_SEED)
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    Axd = dev(Ax)
    s.factorize(Axd)
    recs = [compare_factors(s.export_factors(), lu, RTOL)]
    solve_and_check(s, n, Ap, Ai, Ax, Axd, rng)
    dx = []
    for it in range(10):
        ckt = inputs.perturb_elements(ckt, rng)
        Ax = ckt.values()
        Axd = dev(Ax)
        lu = O.refactorize(lu, Ap, Ai, Ax)
        s.refactorize(Axd)
        recs.append(compare_factors(s.export_factors(), lu, RTOL))
        xg, b = solve_and_check(s, n, Ap, Ai, Ax, Axd, rng)
        xo = O.solve(lu, b)
        dx.append(np.abs(xg - xo).max() / np.abs(xo).max())
        assert dx[-1] <= 1e-10
    print(f"\nC1 sequence (11 factorizations): componentwise error "
          f"{max(r['componentwise'] for r in recs):.3e}, strict per-column error "
          f"{max(r['strict_above_floor'] for r in recs):.3e} above the floor "
          f"({min(r['l_cols_checked'] for r in recs)}/{recs[0]['l_cols']} L and "
          f"{min(r['u_cols_checked'] for r in recs)}/{recs[0]['u_cols']} U columns), "
          f"{max(r['strict_all'] for r in recs):.3e} over all columns; "
          f"x vs oracle {max(dx):.3e}")
    # the raw-entry perturbation fires the pivot check more often
    for it in range(5):
        Ax = inputs.perturb_entries(ckt.values(), rng, frac=0.05, sigma=0.3)
        Axd = dev(Ax)
        lu = O.refactorize(lu, Ap, Ai, Ax)
        s.refactorize(Axd)
        compare_factors(s.export_factors(), lu, RTOL)
        solve_and_check(s, n, Ap, Ai, Ax, Axd, rng)


def mesh_small(seed=7):
    return inputs.rc_mesh3d(40, 40, 4, seed=seed, n_fet=100)


def test_ill_conditioned_mesh_factors_match_oracle():
    """The ill-conditioned mesh variant (every conductance log-uniform in
    [1e-9, 1e4]; 1-norm condition number about 2e11 at 40x40x4), with no
    condition-number filter: the first
    factorization and three re-factorizations with redrawn transistor values
    equal the oracle's factors within the tolerance, and every solve meets
    the residual bound (a backward error, so conditioning does not enter)."""
    ckt = inputs.rc_mesh3d(40, 40, 4, seed=11, n_fet=100, g_range=(1e-9, 1e4))
    n, Ap, Ai, Ax = ckt.csc()
    A = np.zeros((n, n))
    for c in range(n):
        A[Ai[Ap[c]:Ap[c + 1]], c] = Ax[Ap[c]:Ap[c + 1]]
    assert np.linalg.cond(A, 1) > 1e11
    Q = inputs.grid_nd_order(ckt)
    rng = np.random.default_rng(12)
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    Axd = dev(Ax)
    s.factorize(Axd)
    compare_factors(s.export_factors(), lu, RTOL)
    solve_and_check(s, n, Ap, Ai, Ax, Axd, rng)
    for it in range(3):
        Ax = inputs.redraw_transistors(ckt, rng).values()
        Axd = dev(Ax)
        lu = O.refactorize(lu, Ap, Ai, Ax)
        s.refactorize(Axd)
        compare_factors(s.export_factors(), lu, RTOL)
        solve_and_check(s, n, Ap, Ai, Ax, Axd, rng)


def test_schedules_give_bitwise_identical_results():
    ckt = mesh_small()
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    b = dev(inputs.rhs(n, np.random.default_rng(1)))
    outs = []
    for mode in ("auto", "level", "syncfree"):
        s = gblu.Solver(DEV, sched_mode=mode, solve_mode=mode)
        s.analyze(n, Ap, Ai, Q)
        s.factorize(dev(Ax))
        Ax2 = inputs.redraw_transistors(ckt, np.random.default_rng(3)).values()
        s.refactorize(dev(Ax2))
        f = s.export_factors()
        outs.append((f["Lx"], f["Ux"], s.solve(b).cpu().numpy()))
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert np.array_equal(a, c)


def test_forced_repivot_protocol_matches_oracle():
    """Section VI-A general case: runs forced to re-pivot at a random column.
    The pivot entry of A for step k is shifted so that the updated pivot
    x(k) becomes 1e-9 of its value, far below pivot_tol times the largest
    entry of L(:,k), so the check must fail at step k (or earlier)."""
    ckt = mesh_small(seed=11)
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    rng = np.random.default_rng(5)
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    s.factorize(dev(Ax))
    compare_factors(s.export_factors(), lu, RTOL)

    def slot(r, c):
        rows = Ai[Ap[c]:Ap[c + 1]]
        hit = np.nonzero(rows == r)[0]
        return Ap[c] + hit[0] if len(hit) else None

    done = 0
    while done < 6:
        Ax2 = inputs.redraw_transistors(ckt, rng).values()
        ref = O.refactorize(lu, Ap, Ai, Ax2)
        k = int(rng.integers(0, n))
        p = slot(lu.piv[k], Q[k])
        if ref.n_rejected or p is None or ref.Lp[k + 1] == ref.Lp[k]:
            continue
        Ax2[p] -= ref.Ux[ref.Up[k + 1] - 1] * (1.0 - 1e-9)
        lu2 = O.refactorize(lu, Ap, Ai, Ax2)
        assert lu2.n_rejected > 0
        Axd2 = dev(Ax2)
        rc, rep = s.refactorize(Axd2)
        assert rc == gblu.REPIVOTED and rep
        st = s.stats()
        assert 0 <= st["last_first_bad"] <= k
        compare_factors(s.export_factors(), lu2, RTOL)
        solve_and_check(s, n, Ap, Ai, Ax2, Axd2, rng)
        # the next plain refactorization runs on the new pattern
        Ax3 = inputs.redraw_transistors(ckt, rng).values()
        lu3 = O.refactorize(lu2, Ap, Ai, Ax3)
        rc, rep = s.refactorize(dev(Ax3))
        assert rep == (lu3.n_rejected > 0)
        compare_factors(s.export_factors(), lu3, RTOL)
        lu = lu3
        done += 1


def test_dense_block_uses_long_column_path():
    """Columns longer than the shared-memory work vector (1,024 entries)
    are updated in place in global memory."""
    rng = np.random.default_rng(3)
    n = 1200
    A = rng.normal(size=(n, n))
    A[np.arange(n), np.arange(n)] += 40.0
    _, Ap, Ai, Ax = inputs.dense_to_csc(A, np.ones((n, n), bool))
    Q = np.arange(n, dtype=np.int32)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    Axd = dev(Ax)
    s.factorize(Axd)
    compare_factors(s.export_factors(), lu, RTOL)
    solve_and_check(s, n, Ap, Ai, Ax, Axd, rng)
    # and through the pivoting tail: flip the first diagonal
    Ax2 = Ax.copy()
    Ax2[0] = 1e-9
    lu2 = O.refactorize(lu, Ap, Ai, Ax2)
    s.refactorize(dev(Ax2))
    compare_factors(s.export_factors(), lu2, RTOL)


def rails_grid():
    """130x130 grid with 9 rails of growing coverage: its factor columns
    span every task kind and memory mode of the refactorization kernel
    (short columns one per warp, medium columns in pairs, long columns in
    shared memory, longer ones with only their rows in shared memory, and
    one beyond that, updated entirely in global memory)."""
    return inputs.bordered_grid(130, 130, n_rails=9,
                                density=[0.0005, 0.002, 0.004, 0.01, 0.02, 0.05, 0.1, 0.3, 0.95])


@pytest.mark.parametrize("sched", ["auto", "level", "syncfree"])
def test_every_column_task_kind(sched):
    ckt = rails_grid()
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    rng = np.random.default_rng(17)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    ln = np.diff(lu.Lp) + np.diff(lu.Up)
    # one warp up to 640 entries; half a CTA up to 2,560; a whole CTA with
    # its work vector in shared memory up to 5,120, its rows alone there up
    # to 15,360, and beyond that in global memory
    kinds = [(ln <= 640).sum(), ((ln > 640) & (ln <= 2560)).sum(),
             ((ln > 2560) & (ln <= 5120)).sum(), ((ln > 5120) & (ln <= 15360)).sum(),
             (ln > 15360).sum()]
    assert min(kinds) >= 1 and kinds[3] >= 2, kinds
    s = gblu.Solver(DEV, sched_mode=sched, solve_mode=sched)
    s.analyze(n, Ap, Ai, Q)
    s.factorize(dev(Ax))
    # the rails are wide columns: most of their dependencies go row by row
    assert s.stats()["wide_cols"] >= 4
    compare_factors(s.export_factors(), lu, RTOL)
    for it in range(3):
        ckt = inputs.perturb_elements(ckt, rng, frac=0.2)
        Ax = ckt.values()
        Axd = dev(Ax)
        lu = O.refactorize(lu, Ap, Ai, Ax)
        rc, rep = s.refactorize(Axd)
        assert rep == (lu.n_rejected > 0)
        compare_factors(s.export_factors(), lu, RTOL)
        solve_and_check(s, n, Ap, Ai, Ax, Axd, rng)
    # force a restart at the first rail: every longer column is recomputed
    k = n - 9
    c = Q[k]
    rows = Ai[Ap[c]:Ap[c + 1]]
    p = Ap[c] + np.nonzero(rows == lu.piv[k])[0][0]
    Ax2 = Ax.copy()
    Ax2[p] -= lu.Ux[lu.Up[k + 1] - 1] * (1.0 - 1e-9)
    lu2 = O.refactorize(lu, Ap, Ai, Ax2)
    assert lu2.n_rejected > 0
    Axd2 = dev(Ax2)
    rc, rep = s.refactorize(Axd2)
    assert rc == gblu.REPIVOTED and rep
    compare_factors(s.export_factors(), lu2, RTOL)
    solve_and_check(s, n, Ap, Ai, Ax2, Axd2, rng)
    lu3 = O.refactorize(lu2, Ap, Ai, Ax)
    rc, rep = s.refactorize(Axd)
    assert rep == (lu3.n_rejected > 0)
    compare_factors(s.export_factors(), lu3, RTOL)


def test_dense_tail_block():
    """The trailing dense block factored as a dense matrix (dense tail) agrees
    with the oracle and with the column kernels alone, and a pivot that fails
    inside the block restarts exactly like one that fails in a sparse column."""
    ckt = mesh_small(seed=13)
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    rng = np.random.default_rng(23)
    lu = O.factorize(n, Ap, Ai, Ax, Q, 1e-3)
    sd = gblu.Solver(DEV, dense_min_rows=128)
    sc = gblu.Solver(DEV, dense_min_rows=0)
    for s in (sd, sc):
        s.analyze(n, Ap, Ai, Q)
        s.factorize(dev(Ax))
    assert sd.stats()["dense_rows"] >= 128 and sc.stats()["dense_rows"] == 0
    m = sd.stats()["dense_rows"]
    for it in range(3):
        Ax = inputs.redraw_transistors(ckt, rng).values()
        Axd = dev(Ax)
        lu = O.refactorize(lu, Ap, Ai, Ax)
        for s in (sd, sc):
            rc, rep = s.refactorize(Axd)
            assert rep == (lu.n_rejected > 0)
            compare_factors(s.export_factors(), lu, RTOL)
            solve_and_check(s, n, Ap, Ai, Ax, Axd, rng)
    # force the check to fail at a column inside the block
    k = n - m + m // 3
    c = Q[k]
    rows = Ai[Ap[c]:Ap[c + 1]]
    hit = np.nonzero(rows == lu.piv[k])[0]
    assert len(hit)
    Ax2 = Ax.copy()
    Ax2[Ap[c] + hit[0]] -= lu.Ux[lu.Up[k + 1] - 1] * (1.0 - 1e-9)
    lu2 = O.refactorize(lu, Ap, Ai, Ax2)
    assert lu2.n_rejected > 0
    Axd2 = dev(Ax2)
    rc, rep = sd.refactorize(Axd2)
    assert rc == gblu.REPIVOTED and rep
    assert n - m <= sd.stats()["last_first_bad"] <= k
    compare_factors(sd.export_factors(), lu2, RTOL)
    solve_and_check(sd, n, Ap, Ai, Ax2, Axd2, rng)
    # and back to a normal step on the repacked structure
    lu3 = O.refactorize(lu2, Ap, Ai, Ax)
    rc, rep = sd.refactorize(dev(Ax))
    assert rep == (lu3.n_rejected > 0)
    compare_factors(sd.export_factors(), lu3, RTOL)


def test_edge_cases():
    # n = 1
    s = gblu.Solver(DEV)
    s.analyze(1, np.array([0, 1]), np.array([0]), None)
    s.factorize(dev([4.0]))
    assert s.solve(dev([2.0])).cpu().item() == 0.5
    # structurally singular (empty column)
    s = gblu.Solver(DEV)
    s.analyze(2, np.array([0, 2, 2]), np.array([0, 1]), np.array([0, 1]))
    with pytest.raises(gblu.GbluError) as ei:
        s.factorize(dev([1.0, 2.0]))
    assert ei.value.code == gblu.ERR_SINGULAR
    # numerically singular
    s = gblu.Solver(DEV)
    s.analyze(2, np.array([0, 2, 4]), np.array([0, 1, 0, 1]), np.array([0, 1]))
    with pytest.raises(gblu.GbluError):
        s.factorize(dev([1.0, 2.0, 2.0, 4.0]))
    # invalid input
    s = gblu.Solver(DEV)
    with pytest.raises(gblu.GbluError) as ei:
        s.analyze(2, np.array([0, 2, 2]), np.array([1, 1]))
    assert ei.value.code == gblu.ERR_INVALID_INPUT
    with pytest.raises(gblu.GbluError) as ei:
        s.solve(dev([1.0, 2.0]))
    assert ei.value.code == gblu.ERR_NOT_ANALYZED


def test_bounded_wait_returns_timeout_and_context_survives():
    """Every device wait has an iteration limit: with a limit of one
    iteration the sync-free kernels give up on the first unfinished
    predecessor and the call returns GBLU_ERR_DEVICE_TIMEOUT; the context
    stays usable."""
    ckt = mesh_small(seed=2)
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    s = gblu.Solver(DEV, sched_mode="syncfree", solve_mode="syncfree", spin_limit=1)
    s.analyze(n, Ap, Ai, Q)
    codes = []
    for attempt in range(4):   # a wait must occur at least once; it then gives up
        try:
            if attempt == 0 or not codes:
                s.factorize(dev(Ax))
            s.refactorize(dev(Ax))
            s.solve(dev(np.ones(n)))
            torch.cuda.synchronize()
        except gblu.GbluError as e:
            codes.append(e.code)
            break
    assert codes == [gblu.ERR_DEVICE_TIMEOUT]
    torch.cuda.synchronize()
    s2 = gblu.Solver(DEV)
    s2.analyze(n, Ap, Ai, Q)
    Axd = dev(Ax)
    s2.factorize(Axd)
    solve_and_check(s2, n, Ap, Ai, Ax, Axd, np.random.default_rng(0))


def test_library_ordering_when_no_q_given():
    ckt = inputs.workload_small()
    n, Ap, Ai, Ax = ckt.csc()
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, None)
    Axd = dev(Ax)
    s.factorize(Axd)
    f = s.export_factors()
    assert np.array_equal(f["q"], gblu.order_auto(n, Ap, Ai)[0])
    lu = O.factorize(n, Ap, Ai, Ax, f["q"], 1e-3)
    compare_factors(f, lu, RTOL)
    solve_and_check(s, n, Ap, Ai, Ax, Axd, np.random.default_rng(0))


@pytest.mark.parametrize("slices", [1, 3, 8])
def test_structure_adaptive_solve(slices):
    """Section V: trailing block L(P0:n, P0:n) split off by the 70% rule
    (the entry minimum lowered so that a test-sized mesh qualifies), cut into
    trapezoid slices; the solution must match the oracle's residual bound,
    agree with the unsplit solve, and be identical across schedules."""
    ckt = mesh_small(seed=4)
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    rng = np.random.default_rng(8)
    b = inputs.rhs(n, rng)
    Axd = dev(Ax)
    ref = gblu.Solver(DEV, solve_slices=0)
    ref.analyze(n, Ap, Ai, Q)
    ref.factorize(Axd)
    assert ref.stats()["solve_p0_l"] == n
    x_ref = ref.solve(dev(b)).cpu().numpy()
    outs = []
    for mode in ("auto", "level", "syncfree"):
        s = gblu.Solver(DEV, sched_mode=mode, solve_mode=mode, solve_dense_min=1000,
                        solve_slices=slices, solve_dense_density=0.0)
        s.analyze(n, Ap, Ai, Q)
        s.factorize(Axd)
        st = s.stats()
        f = s.export_factors()
        # P0: the largest position whose trailing block holds >= 70% of nnz(L)
        counts = np.diff(f["Lp"])
        suffix = np.cumsum(counts[::-1])[::-1]
        ok = np.nonzero((suffix >= 0.7 * counts.sum()) & (suffix >= 1000))[0]
        assert st["solve_p0_l"] == ok.max()
        assert 1 <= st["solve_slices_l"] <= slices + 1 and st["solve_p0_u"] < n
        x = s.solve(dev(b))
        res = s.residual(Axd, dev(b), x).cpu().numpy()[0]
        assert res <= RESID
        xh = x.cpu().numpy()
        np.testing.assert_allclose(xh, x_ref, rtol=1e-9, atol=1e-12 * np.abs(x_ref).max())
        assert O.residual(n, Ap, Ai, Ax, xh, b) <= RESID
        outs.append(xh)
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
    # GPU rule: the longest trailing block that is at least half dense
    s = gblu.Solver(DEV, solve_dense_min=100, solve_slices=slices, solve_dense_density=0.5)
    s.analyze(n, Ap, Ai, Q)
    s.factorize(Axd)
    f = s.export_factors()
    counts = np.diff(f["Lp"])
    suffix = np.cumsum(counts[::-1])[::-1]
    m = n - np.arange(n, dtype=float)
    dense = suffix[:-1] >= 0.5 * m[:-1] * (m[:-1] - 1) / 2
    p0 = n
    for p in range(n - 2, -1, -1):
        if not dense[p]:
            break
        p0 = p
    assert s.stats()["solve_p0_l"] == (p0 if p0 < n and suffix[p0] >= 100 else n)
    x = s.solve(dev(b)).cpu().numpy()
    np.testing.assert_allclose(x, x_ref, rtol=1e-9, atol=1e-12 * np.abs(x_ref).max())


def test_library_ordering_on_meshes():
    """gblu_analyze without Q on meshes (its automatic choice among minimum
    degree, minimum deficiency and the two dissections): the factors of the
    first factorization and of a re-factorization equal the oracle's on the
    order the library chose."""
    for ckt in (inputs.rc_mesh3d(16, 16, 4, seed=9, n_fet=40), inputs.rc_mesh3d(30, 30, 4, seed=10, n_fet=60)):
        n, Ap, Ai, Ax = ckt.csc()
        s = gblu.Solver(DEV)
        s.analyze(n, Ap, Ai, None)
        Axd = dev(Ax)
        s.factorize(Axd)
        f = s.export_factors()
        assert np.array_equal(f["q"], gblu.order_auto(n, Ap, Ai)[0])
        lu = O.factorize(n, Ap, Ai, Ax, f["q"], 1e-3)
        compare_factors(f, lu, RTOL)
        Ax2 = inputs.redraw_transistors(ckt, np.random.default_rng(4)).values()
        lu2 = O.refactorize(lu, Ap, Ai, Ax2)
        Axd2 = dev(Ax2)
        rc, rep = s.refactorize(Axd2)
        assert rep == (lu2.n_rejected > 0)
        compare_factors(s.export_factors(), lu2, RTOL)
        solve_and_check(s, n, Ap, Ai, Ax2, Axd2, np.random.default_rng(0))
