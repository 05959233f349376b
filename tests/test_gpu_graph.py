"""Graph replay of a Newton step (gblu_step): the same results as
gblu_refactorize + gblu_solve, bit for bit, and across a step whose check
fails (restart, new structure, new capture).  On the restarting step itself
the two runs may differ in the last bits: which columns were finished when
the check failed depends on timing, and the restart recomputes the others
in its own order, so that step is compared within rounding."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_14082_gb300 import gblu, inputs

pytestmark = pytest.mark.gpu

DEV = 0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(f"cuda:{DEV}")


@pytest.mark.parametrize("case", ["small_mna", "mesh"])
def test_step_equals_refactorize_and_solve(case):
    ckt = inputs.workload_small() if case == "small_mna" else inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)
    n, Ap, Ai, Ax0 = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    g, p = gblu.Solver(DEV), gblu.Solver(DEV)
    for s in (g, p):
        s.analyze(n, Ap, Ai, Q)
        s.factorize(dev(Ax0))
    lu = O.factorize(n, Ap, Ai, Ax0, Q, 1e-3)
    rng = np.random.default_rng(17)
    for it in range(6):
        ckt = inputs.perturb_elements(ckt, rng) if case == "small_mna" else inputs.redraw_transistors(ckt, rng)
        Ax = ckt.values()
        if it == 3:
            # a pivot that fails its check: the replay restarts and solves again
            ref = O.refactorize(lu, Ap, Ai, Ax)
            k = n // 2
            while True:
                c = Q[k]
                rows = Ai[Ap[c]:Ap[c + 1]]
                hit = np.nonzero(rows == lu.piv[k])[0]
                if len(hit) and ref.Lp[k + 1] > ref.Lp[k]:
                    break
                k += 1
            Ax = Ax.copy()
            Ax[Ap[c] + hit[0]] -= ref.Ux[ref.Up[k + 1] - 1] * (1.0 - 1e-9)
        b = inputs.rhs(n, rng)
        xg, rep_g = g.step(dev(Ax), dev(b))
        _, rep_p = p.refactorize(dev(Ax))
        xp = p.solve(dev(b))
        assert rep_g == rep_p
        if it == 3:
            assert rep_g
        if rep_g:
            torch.testing.assert_close(xg, xp, rtol=1e-10, atol=1e-12 * xp.abs().max().item())
        else:
            assert torch.equal(xg, xp)
        lu = O.refactorize(lu, Ap, Ai, Ax)
        assert O.residual(n, Ap, Ai, Ax, xg.cpu().numpy(), b) <= 1e-12
    st = g.stats()
    assert st["n_refactor"] == 6 and st["kernel_launches"] > 0


def test_autotune_keeps_results():
    """The autotuner only changes the schedule: the factors of the same
    values are bit for bit the same, and the solve still meets the residual."""
    ckt = inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)
    n, Ap, Ai, Ax0 = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    s.factorize(dev(Ax0))
    rng = np.random.default_rng(4)
    Ax = inputs.redraw_transistors(ckt, rng).values()
    b = inputs.rhs(n, rng)
    s.refactorize(dev(Ax))
    f0 = s.export_factors()
    chosen, tr, ts = s.autotune(dev(Ax), dev(b), reps=2)
    assert chosen["alpha"] in (0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0) and tr > 0 and ts > 0
    assert s.opts()["alpha"] == chosen["alpha"]
    s.refactorize(dev(Ax))
    f1 = s.export_factors()
    for k in f0:
        assert np.array_equal(f0[k], f1[k]), k
    x = s.solve(dev(b)).cpu().numpy()
    assert O.residual(n, Ap, Ai, Ax, x, b) <= 1e-12
    with pytest.raises(gblu.GbluError):
        s.set_opts(alpha=-1.0)


def test_step_batch_replay_equals_eager_batch():
    """gblu_step_batch (graph replay after the first call) gives the factor
    values, solutions and failed flags of gblu_refactorize_batch followed
    by gblu_solve_batch, bit for bit, over several calls whose values change
    in the same buffers; one call has a set whose check fails."""
    ckt = inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)
    n, Ap, Ai, Ax0 = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    g, p = gblu.Solver(DEV), gblu.Solver(DEV)
    for s in (g, p):
        s.analyze(n, Ap, Ai, Q)
        s.factorize(dev(Ax0))
    lu = O.factorize(n, Ap, Ai, Ax0, Q, 1e-3)
    nsets = 12
    rng = np.random.default_rng(23)
    st = g.stats()
    nlu = st["nnz_l"] + st["nnz_u"]
    Ax = torch.empty((nsets, len(Ai)), dtype=torch.float64, device=f"cuda:{DEV}")
    b = torch.empty((nsets, n), dtype=torch.float64, device=f"cuda:{DEV}")
    LUg = torch.empty((nsets, nlu), dtype=torch.float64, device=f"cuda:{DEV}")
    xg = torch.empty_like(b)
    launches = []
    for call in range(4):
        vals = np.stack([inputs.scale_values(Ax0, rng, 0.02) for _ in range(nsets)])
        if call == 2:
            # set 5: the pivot of one step is made to fail its check
            ref = O.refactorize(lu, Ap, Ai, vals[5])
            k = (2 * n) // 3
            c = Q[k]
            hit = np.nonzero(Ai[Ap[c]:Ap[c + 1]] == lu.piv[k])[0][0]
            vals[5, Ap[c] + hit] -= ref.Ux[ref.Up[k + 1] - 1] * (1.0 - 1e-9)
        Ax.copy_(torch.from_numpy(vals))
        b.copy_(torch.from_numpy(np.stack([inputs.rhs(n, rng) for _ in range(nsets)])))
        l0 = g.stats()["kernel_launches"]
        fg = g.step_batch(Ax, LUg, b, xg)
        launches.append(g.stats()["kernel_launches"] - l0)
        LUp, fp = p.refactorize_batch(Ax)
        xp = p.solve_batch(LUp, b)
        assert np.array_equal(fg, fp)
        if call == 2:
            assert fg[5]
        ok = fg == 0
        assert torch.equal(LUg[torch.from_numpy(ok).to(LUg.device)], LUp[torch.from_numpy(ok).to(LUg.device)])
        assert torch.equal(xg[torch.from_numpy(ok).to(xg.device)], xp[torch.from_numpy(ok).to(xg.device)])
    # replays launch the same kernels as the eager first call
    assert launches[1] == launches[2] == launches[3] > 0
