"""Batches of value sets on one structure (gblu_refactorize_batch,
gblu_solve_batch): each set's result is bit-for-bit the result of the
single-matrix path on the same values (same kernels, same order), a set
whose pivot check fails is reported alone, and the oracle agrees."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_14082_gb300 import gblu, inputs
from tests.factor_compare import compare_factors

pytestmark = pytest.mark.gpu

DEV = 0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(f"cuda:{DEV}")


def value_sets(ckt, nsets, seed):
    rng = np.random.default_rng(seed)
    return [inputs.perturb_elements(ckt, rng, frac=0.05, sigma=0.2).values() for _ in range(nsets)]


def singles(n, Ap, Ai, Q, Ax0, sets, rhs):
    """x of each set through the one-matrix path (fresh factorization each,
    so every set starts from the same structure), and whether it repivoted."""
    xs, reps = [], []
    for Ax, b in zip(sets, rhs):
        s = gblu.Solver(DEV)
        s.analyze(n, Ap, Ai, Q)
        s.factorize(dev(Ax0))
        _, rep = s.refactorize(dev(Ax))
        xs.append(s.solve(dev(b)).cpu().numpy())
        reps.append(rep)
    return xs, reps


def batch_case(case):
    if case == "small_mna":
        return inputs.workload_small()
    if case == "rails":   # six rails, each a wide column (its dependencies applied row by row)
        return inputs.bordered_grid(60, 60, n_rails=6, density=0.2)
    return inputs.rc_mesh3d(40, 40, 4, seed=5, n_fet=100)


@pytest.mark.parametrize("case", ["small_mna", "mesh", "rails"])
def test_batch_equals_single_path_bitwise(case):
    ckt = batch_case(case)
    n, Ap, Ai, Ax0 = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    nsets = 6
    sets = value_sets(ckt, nsets, 31)
    rng = np.random.default_rng(7)
    rhs = [inputs.rhs(n, rng) for _ in range(nsets)]
    x_single, reps = singles(n, Ap, Ai, Q, Ax0, sets, rhs)
    sb = gblu.Solver(DEV)
    sb.analyze(n, Ap, Ai, Q)
    sb.factorize(dev(Ax0))
    if case == "rails":
        assert sb.stats()["wide_cols"] == 6
    LUx, failed = sb.refactorize_batch(dev(np.stack(sets)))
    assert np.array_equal(failed.astype(bool), np.array(reps))
    x = sb.solve_batch(LUx, dev(np.stack(rhs))).cpu().numpy()
    lu0 = O.factorize(n, Ap, Ai, Ax0, Q, 1e-3)
    for s_ in range(nsets):
        if failed[s_]:
            continue
        assert np.array_equal(x[s_], x_single[s_]), f"set {s_} differs from the single path"
        assert O.residual(n, Ap, Ai, sets[s_], x[s_], rhs[s_]) <= 1e-12
        lu = O.refactorize(lu0, Ap, Ai, sets[s_])
        assert lu.n_rejected == 0


def test_batch_reports_the_failing_set_alone():
    ckt = inputs.workload_small()
    n, Ap, Ai, Ax0 = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    nsets = 5
    sets = value_sets(ckt, nsets, 41)
    lu0 = O.factorize(n, Ap, Ai, Ax0, Q, 1e-3)
    # set 2: the pivot of step k becomes 1e-9 of its value, so its check fails
    bad = 2
    ref = O.refactorize(lu0, Ap, Ai, sets[bad])
    k = n // 2
    while True:
        c = Q[k]
        rows = Ai[Ap[c]:Ap[c + 1]]
        hit = np.nonzero(rows == lu0.piv[k])[0]
        if len(hit) and ref.Lp[k + 1] > ref.Lp[k]:
            break
        k += 1
    sets[bad] = sets[bad].copy()
    sets[bad][Ap[c] + hit[0]] -= ref.Ux[ref.Up[k + 1] - 1] * (1.0 - 1e-9)
    assert O.refactorize(lu0, Ap, Ai, sets[bad]).n_rejected > 0
    rng = np.random.default_rng(9)
    rhs = [inputs.rhs(n, rng) for _ in range(nsets)]
    x_single, reps = singles(n, Ap, Ai, Q, Ax0, sets, rhs)
    assert reps[bad]
    sb = gblu.Solver(DEV)
    sb.analyze(n, Ap, Ai, Q)
    sb.factorize(dev(Ax0))
    LUx, failed = sb.refactorize_batch(dev(np.stack(sets)))
    assert failed[bad] == 1 and failed.sum() == 1 + sum(reps[i] for i in range(nsets) if i != bad)
    x = sb.solve_batch(LUx, dev(np.stack(rhs))).cpu().numpy()
    for s_ in range(nsets):
        if not failed[s_]:
            assert np.array_equal(x[s_], x_single[s_])
    # the handle's own factors are untouched by the batch
    f = sb.export_factors()
    compare_factors(f, lu0, 1e-10)


def test_batch_argument_errors():
    ckt = inputs.workload_small()
    n, Ap, Ai, Ax0 = ckt.csc()
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, inputs.grid_nd_order(ckt))
    with pytest.raises(gblu.GbluError):   # not factorized yet
        s.refactorize_batch(dev(np.stack([Ax0, Ax0])))
    s.factorize(dev(Ax0))
    with pytest.raises(ValueError):
        s.refactorize_batch(dev(Ax0))     # not [nsets, nnz]
    LUx, failed = s.refactorize_batch(dev(np.stack([Ax0])))
    assert failed.tolist() == [0]
    with pytest.raises(ValueError):
        s.solve_batch(LUx, dev(np.zeros((2, n))))


def multi_cases():
    out = []
    for (nx, ny, seed) in ((10, 12, 1), (20, 25, 2), (30, 30, 3), (40, 50, 4), (16, 60, 5)):
        ckt = inputs.mna_grid2d(nx, ny, seed=seed)
        n, Ap, Ai, Ax0 = ckt.csc()
        out.append((ckt, n, Ap, Ai, Ax0, inputs.grid_nd_order(ckt)))
    ckt = inputs.rc_mesh3d(14, 14, 3, seed=6, n_fet=30)
    n, Ap, Ai, Ax0 = ckt.csc()
    out.append((ckt, n, Ap, Ai, Ax0, inputs.grid_nd_order(ckt)))
    # and one with wide columns (four rails), beside patterns without any
    ckt = inputs.bordered_grid(50, 50, n_rails=4, density=0.3)
    n, Ap, Ai, Ax0 = ckt.csc()
    out.append((ckt, n, Ap, Ai, Ax0, inputs.grid_nd_order(ckt)))
    return out


def test_multi_pattern_batch_equals_single_handles():
    cases = multi_cases()
    rng = np.random.default_rng(21)

    def handles():
        hs = []
        for ckt, n, Ap, Ai, Ax0, Q in cases:
            s = gblu.Solver(DEV)
            s.analyze(n, Ap, Ai, Q)
            s.factorize(dev(Ax0))
            hs.append(s)
        return hs

    multi, single = handles(), handles()
    lus = [O.factorize(c[1], c[2], c[3], c[4], c[5], 1e-3) for c in cases]
    for step in range(3):
        vals = [inputs.perturb_elements(c[0], rng, frac=0.05, sigma=0.2).values() for c in cases]
        rhs = [inputs.rhs(c[1], rng) for c in cases]
        if step == 2:
            # pattern 3 gets a pivot that fails its check (the others do not)
            ckt, n, Ap, Ai, Ax0, Q = cases[3]
            ref = O.refactorize(lus[3], Ap, Ai, vals[3])
            k = n // 2
            while True:
                c = Q[k]
                rows = Ai[Ap[c]:Ap[c + 1]]
                hit = np.nonzero(rows == lus[3].piv[k])[0]
                if len(hit) and ref.Lp[k + 1] > ref.Lp[k]:
                    break
                k += 1
            vals[3] = vals[3].copy()
            vals[3][Ap[c] + hit[0]] -= ref.Ux[ref.Up[k + 1] - 1] * (1.0 - 1e-9)
        reps = gblu.refactorize_multi(multi, [dev(v) for v in vals])
        xm = [x.cpu().numpy() for x in gblu.solve_multi(multi, [dev(b) for b in rhs])]
        for i, (c, s) in enumerate(zip(cases, single)):
            _, rep = s.refactorize(dev(vals[i]))
            assert rep == reps[i]
            xs = s.solve(dev(rhs[i])).cpu().numpy()
            if rep:   # the restart set depends on timing: equal within rounding
                np.testing.assert_allclose(xm[i], xs, rtol=1e-10, atol=1e-12 * np.abs(xs).max())
            else:
                assert np.array_equal(xs, xm[i]), f"pattern {i} differs from its single handle"
            lus[i] = O.refactorize(lus[i], c[2], c[3], vals[i])
            compare_factors(multi[i].export_factors(), lus[i], 1e-10)
            assert O.residual(c[1], c[2], c[3], vals[i], xm[i], rhs[i]) <= 1e-12
        if step == 2:
            assert reps[3] and sum(reps) == 1 + sum(reps[i] for i in range(len(cases)) if i != 3)
    with pytest.raises(gblu.GbluError):
        gblu.refactorize_multi([multi[0], multi[0]], [dev(cases[0][4])] * 2)
