"""The allocation-free solve entry point against the handle's solve.

Callers that cannot allocate device memory (a simulator on its own fixed
pool, code running during graph capture) keep the factors in their own
buffers and call gblu_solve_factors_noalloc, whose scratch is a static
device array.  This file is collected last on purpose.  The test exports
the factors of a handle, lays them out row-wise in buffers the caller owns,
and checks two calls in a row against gblu_solve on the same factors.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from paper_2411_14082_gb300 import gblu, inputs

pytestmark = pytest.mark.gpu

DEV = 0
RTOL = 1e-12


def row_wise(f, n):
    """CSR copies (strict lower L, strict upper U, diag U) of exported factors."""
    L = sp.csc_matrix((f["Lx"], f["Li"], f["Lp"]), shape=(n, n)).tocsr()
    U = sp.csc_matrix((f["Ux"], f["Ui"], f["Up"]), shape=(n, n))
    d = U.diagonal().copy()
    Us = sp.triu(U, k=1, format="csr")
    L.sort_indices()
    Us.sort_indices()
    dev = f"cuda:{DEV}"
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)
    return dict(Lrp=t(L.indptr, np.int64), Lcol=t(L.indices, np.int32), Lval=t(L.data, np.float64),
                Urp=t(Us.indptr, np.int64), Ucol=t(Us.indices, np.int32), Uval=t(Us.data, np.float64),
                Udiag=t(d, np.float64), piv=t(f["piv"], np.int32), q=t(f["q"], np.int32))


@pytest.mark.parametrize("case", ["small_mna", "mesh_40x40x4"])
def test_noalloc_solve_matches_handle_solve_twice(case):
    ckt = inputs.workload_small() if case == "small_mna" else inputs.rc_mesh3d(40, 40, 4, seed=7, n_fet=100)
    n, Ap, Ai, Ax = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, Q)
    Axd = torch.from_numpy(Ax).cuda(DEV)
    s.factorize(Axd)
    R = row_wise(s.export_factors(), n)
    rng = np.random.default_rng(3)
    status = torch.full((1,), -77, dtype=torch.int32, device=f"cuda:{DEV}")
    for call in range(2):
        b = torch.from_numpy(inputs.rhs(n, rng)).cuda(DEV)
        x_ref = s.solve(b)
        x = torch.full_like(b, float("nan"))
        gblu.solve_factors_noalloc(n, R["Lrp"], R["Lcol"], R["Lval"], R["Urp"], R["Ucol"],
                                   R["Uval"], R["Udiag"], R["piv"], R["q"], b, x, status)
        torch.cuda.synchronize()
        assert status.item() == 0
        xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
        assert np.all(np.isfinite(xn))
        np.testing.assert_allclose(xn, xr, rtol=RTOL, atol=RTOL * np.abs(xr).max())
        res = s.residual(Axd, b, x).cpu().numpy()
        assert res[0] <= 1e-12


def test_noalloc_rejects_sizes_beyond_the_maximum():
    z64 = torch.zeros(2, dtype=torch.int64, device=f"cuda:{DEV}")
    z32 = torch.zeros(1, dtype=torch.int32, device=f"cuda:{DEV}")
    zd = torch.zeros(1, dtype=torch.float64, device=f"cuda:{DEV}")
    zd2 = torch.zeros(1, dtype=torch.float64, device=f"cuda:{DEV}")
    with pytest.raises(gblu.GbluError) as ei:
        gblu.solve_factors_noalloc(gblu.NOALLOC_MAX_N + 1, z64, z32, zd, z64, z32, zd, zd,
                                   z32, z32, zd, zd2)
    assert ei.value.code == gblu.ERR_INVALID_INPUT
    assert "GBLU_NOALLOC_MAX_N" in str(ei.value)


def test_noalloc_wait_limit_reports_timeout_and_context_survives():
    """With a wait limit of one poll, a row that needs a value not yet
    published gives up at once: status_dev receives GBLU_ERR_DEVICE_TIMEOUT
    (the only place a caller can see it; the call itself returned when the
    kernels were queued).  A later call with the default limit on the same
    device solves correctly, so the context is intact."""
    ckt = inputs.rc_mesh3d(40, 40, 4, seed=7, n_fet=100)
    n, Ap, Ai, Ax = ckt.csc()
    s = gblu.Solver(DEV)
    s.analyze(n, Ap, Ai, inputs.grid_nd_order(ckt))
    s.factorize(torch.from_numpy(Ax).cuda(DEV))
    R = row_wise(s.export_factors(), n)
    b = torch.from_numpy(inputs.rhs(n, np.random.default_rng(4))).cuda(DEV)
    status = torch.full((1,), -77, dtype=torch.int32, device=f"cuda:{DEV}")
    seen = []
    for call in range(3):
        x = torch.zeros_like(b)
        gblu.solve_factors_noalloc(n, R["Lrp"], R["Lcol"], R["Lval"], R["Urp"], R["Ucol"],
                                   R["Uval"], R["Udiag"], R["piv"], R["q"], b, x, status,
                                   spin_limit=1)
        torch.cuda.synchronize()
        seen.append(status.item())
    assert gblu.ERR_DEVICE_TIMEOUT in seen and set(seen) <= {0, gblu.ERR_DEVICE_TIMEOUT}
    x = torch.full_like(b, float("nan"))
    gblu.solve_factors_noalloc(n, R["Lrp"], R["Lcol"], R["Lval"], R["Urp"], R["Ucol"],
                               R["Uval"], R["Udiag"], R["piv"], R["q"], b, x, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    xr = s.solve(b).cpu().numpy()
    np.testing.assert_allclose(x.cpu().numpy(), xr, rtol=RTOL, atol=RTOL * np.abs(xr).max())
