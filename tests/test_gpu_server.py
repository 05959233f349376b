"""Solve server (gblu_server_*): requests of several patterns submitted
together give bit-for-bit the results they give alone and through the
single-matrix path; a request whose pivot check fails is redone with
pivoting; admission respects the device-memory budget."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_14082_gb300 import gblu, inputs

pytestmark = pytest.mark.gpu

DEV = 0


def pattern_cases():
    out = []
    for ckt in (inputs.workload_small(), inputs.rc_mesh3d(24, 24, 4, seed=5, n_fet=60)):
        n, Ap, Ai, Ax0 = ckt.csc()
        Q = inputs.grid_nd_order(ckt)
        out.append((ckt, n, Ap, Ai, Ax0, Q))
    return out


def clean_requests(case, count, seed):
    """Value sets whose checked re-factorization keeps every pivot (oracle)."""
    ckt, n, Ap, Ai, Ax0, Q = case
    lu0 = O.factorize(n, Ap, Ai, Ax0, Q, 1e-3)
    rng = np.random.default_rng(seed)
    reqs = []
    while len(reqs) < count:
        Ax = inputs.perturb_elements(ckt, rng, frac=0.05, sigma=0.2).values()
        if O.refactorize(lu0, Ap, Ai, Ax).n_rejected == 0:
            reqs.append((Ax, inputs.rhs(n, rng)))
    return reqs


def test_mix_equals_alone_and_single_path():
    import torch
    cases = pattern_cases()
    reqs = [clean_requests(c, 40, 11 + i) for i, c in enumerate(cases)]
    mix = gblu.Server(DEV, hbm_budget=4 << 30, max_batch=16)
    alone = gblu.Server(DEV, hbm_budget=4 << 30, max_batch=16)
    pids_m = [mix.add_pattern(c[1], c[2], c[3], c[5], c[4])[0] for c in cases]
    pids_a = [alone.add_pattern(c[1], c[2], c[3], c[5], c[4])[0] for c in cases]
    ids = []
    for j in range(40):                     # interleaved, all in flight at once
        for p in range(len(cases)):
            ids.append((p, j, mix.submit(pids_m[p], *reqs[p][j])))
    got = {}
    for p, j, rid in ids:
        x, r = mix.wait(rid)
        assert r["status"] == gblu.OK and r["repivoted"] == 0
        assert r["berr"] <= 1e-12
        got[p, j] = x
    st = mix.stats()
    assert st["completed"] == st["submitted"] == 80 and st["max_batch_seen"] >= 2
    for p, c in enumerate(cases):
        _, n, Ap, Ai, Ax0, Q = c
        for j in range(40):
            x, r = alone.wait(alone.submit(pids_a[p], *reqs[p][j]))
            assert r["batch_size"] == 1
            assert np.array_equal(x, got[p, j]), f"pattern {p} request {j}: mix differs from alone"
            assert O.residual(n, Ap, Ai, reqs[p][j][0], x, reqs[p][j][1]) <= 1e-12
        # the single-matrix path on a fresh handle
        s = gblu.Solver(DEV)
        s.analyze(n, Ap, Ai, Q)
        s.factorize(torch.from_numpy(Ax0).cuda(DEV))
        for j in (0, 17, 39):
            s.refactorize(torch.from_numpy(reqs[p][j][0]).cuda(DEV))
            xs = s.solve(torch.from_numpy(reqs[p][j][1]).cuda(DEV)).cpu().numpy()
            assert np.array_equal(xs, got[p, j])
    mix.close()
    alone.close()


def test_failing_request_is_redone_with_pivoting():
    case = pattern_cases()[0]
    ckt, n, Ap, Ai, Ax0, Q = case
    reqs = clean_requests(case, 12, 5)
    lu0 = O.factorize(n, Ap, Ai, Ax0, Q, 1e-3)
    Axb, bb = reqs[6]
    ref = O.refactorize(lu0, Ap, Ai, Axb)
    k = n // 2
    while True:
        c = Q[k]
        rows = Ai[Ap[c]:Ap[c + 1]]
        hit = np.nonzero(rows == lu0.piv[k])[0]
        if len(hit) and ref.Lp[k + 1] > ref.Lp[k]:
            break
        k += 1
    Axb = Axb.copy()
    Axb[Ap[c] + hit[0]] -= ref.Ux[ref.Up[k + 1] - 1] * (1.0 - 1e-9)
    assert O.refactorize(lu0, Ap, Ai, Axb).n_rejected > 0
    reqs[6] = (Axb, bb)
    srv = gblu.Server(DEV, hbm_budget=2 << 30, max_batch=8)
    pid, _ = srv.add_pattern(n, Ap, Ai, Q, Ax0)
    ids = [srv.submit(pid, *r) for r in reqs]
    for j, rid in enumerate(ids):
        x, r = srv.wait(rid)
        assert r["status"] in (gblu.OK, gblu.REPIVOTED)
        assert O.residual(n, Ap, Ai, reqs[j][0], x, reqs[j][1]) <= 1e-12
        assert r["berr"] <= 1e-12
        if j == 6:
            assert r["repivoted"] == 1 and r["status"] == gblu.REPIVOTED
    assert srv.stats()["repivots"] >= 1
    srv.close()


def test_admission_by_device_memory():
    cases = pattern_cases()
    _, n, Ap, Ai, Ax0, Q = cases[1]
    with pytest.raises(gblu.GbluError) as e:
        gblu.Server(DEV, hbm_budget=1 << 20).add_pattern(n, Ap, Ai, Q, Ax0)
    assert e.value.code == gblu.ERR_NOMEM
    probe = gblu.Server(DEV, hbm_budget=4 << 30, max_batch=3)
    pid, slots = probe.add_pattern(n, Ap, Ai, Q, Ax0)
    fp3 = probe.pattern_info(pid)["footprint_bytes"]
    assert slots == 3
    probe.close()
    # a budget of about that footprint admits the pattern with at most 3
    # slots and then has no room for a second copy
    srv = gblu.Server(DEV, hbm_budget=fp3 + (1 << 20), max_batch=64)
    pid, slots = srv.add_pattern(n, Ap, Ai, Q, Ax0)
    info = srv.pattern_info(pid)
    st = srv.stats()
    assert 1 <= slots <= 3 and info["footprint_bytes"] <= st["budget_bytes"]
    assert st["reserved_bytes"] == info["footprint_bytes"]
    with pytest.raises(gblu.GbluError) as e:
        srv.add_pattern(n, Ap, Ai, Q, Ax0)
    assert e.value.code == gblu.ERR_NOMEM
    # the admitted pattern still serves
    rng = np.random.default_rng(2)
    b = inputs.rhs(n, rng)
    x, r = srv.wait(srv.submit(pid, Ax0, b))
    assert r["status"] == gblu.OK and O.residual(n, Ap, Ai, Ax0, x, b) <= 1e-12
    with pytest.raises(gblu.GbluError):
        srv.wait(10 ** 9)                    # unknown request
    srv.close()


def test_single_precision_requests():
    """Mode 1 requests (single-precision factors, refinement in double)
    reach the double-precision backward error, mixed with mode 0 ones."""
    case = pattern_cases()[1]
    ckt, n, Ap, Ai, Ax0, Q = case
    reqs = clean_requests(case, 10, 9)
    srv = gblu.Server(DEV, hbm_budget=2 << 30, max_batch=8)
    pid, _ = srv.add_pattern(n, Ap, Ai, Q, Ax0)
    ids = [(j, srv.submit(pid, *r, mixed=(j % 2 == 1))) for j, r in enumerate(reqs)]
    for j, rid in ids:
        x, r = srv.wait(rid)
        assert r["status"] in (gblu.OK, gblu.REPIVOTED)
        assert r["berr"] <= 1e-12 and O.residual(n, Ap, Ai, reqs[j][0], x, reqs[j][1]) <= 1e-12
        if j % 2 == 1:
            assert r["batch_size"] == 1 and r["refine_iters"] != 0 or r["berr"] <= 1e-12
    srv.close()
