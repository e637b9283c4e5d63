"""Continuous-batching server: results are the same alone and in the mix; admission by budget.

Tolerance: 1e-12 relative per state on FP64 plans.  Batching changes only which launch a
state column rides in; the small-batch implicit solve uses an affine-scan evaluation
order, so results agree to rounding rather than bit for bit.  On split-precision plans the
batch width selects the Legendre and implicit-solve kernels: alone and in the mix agree
within the split-precision tolerance (full height field 1e-6, fields 1e-5).
"""
import numpy as np
import pytest

from paper_2306_09497_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def plans():
    from paper_2306_09497_gb300 import swe
    p31 = swe.Plan(31, 48, 96)
    p21 = swe.Plan(21, 32, 64)
    yield swe, p31, p21
    p31.close()
    p21.close()


def _run(swe, server, reqs, arrivals):
    """reqs: list of submit-kwargs; arrivals: step index at which each request is submitted."""
    ids = {}
    step = 0
    pending = set(range(len(reqs)))
    done = {}
    while pending or len(done) < len(reqs):
        for i in sorted(pending):
            if arrivals[i] == step:
                ids[i] = server.submit(**reqs[i])
                pending.discard(i)
        a, q, dn = server.step()
        step += 1
        for i, rid in list(ids.items()):
            if i in done:
                continue
            try:
                done[i] = server.result(rid)
            except swe.SWEError:
                pass
        assert step < 100
    return done


def test_results_same_alone_and_in_mix(plans):
    swe, p31, p21 = plans
    fine = swe.stepper(swe.SWE_IMEX, 600.0, 3)
    coarse = swe.stepper(swe.SWE_IMEX, 1800.0, 1, 2, 1e5)
    U = inputs.random_state(31, 4, seed=61)
    reqs = [
        dict(fine_plan=p31, coarse_plan=p31, method=swe.SWE_METHOD_PARAREAL, fine=fine, coarse=coarse, S=4, iters=3,
             U0_host=U[0]),
        dict(fine_plan=p31, coarse_plan=p21, method=swe.SWE_METHOD_PARAREAL, fine=fine, coarse=coarse, S=6, iters=2,
             U0_host=U[1]),
        dict(fine_plan=p31, coarse_plan=p31, method=swe.SWE_METHOD_MGRIT2, fine=swe.stepper(swe.SWE_IMEX, 600.0, 1),
             coarse=swe.stepper(swe.SWE_IMEX, 1200.0, 1, 2, 1e5), S=4, cf=2, iters=2, U0_host=U[2]),
        dict(fine_plan=p31, coarse_plan=p31, method=swe.SWE_METHOD_PARAREAL, fine=fine, coarse=coarse, S=5, iters=2,
             U0_host=U[3]),
    ]
    alone = []
    for r in reqs:
        srv = swe.Server(1 << 34, 8)
        alone.append(_run(swe, srv, [r], [0])[0][0])
        srv.close()
    srv = swe.Server(1 << 34, 8)
    mixed = _run(swe, srv, reqs, [0, 1, 0, 1])     # requests 1 and 3 arrive while 0 and 2 run
    srv.close()
    for i in range(len(reqs)):
        got = mixed[i][0]
        for n in range(got.shape[0]):
            for f in range(3):
                assert _rel(got[n, f], alone[i][n, f]) < 1e-12, (i, n, f)
    # a Parareal request equals the stand-alone Parareal driver
    pr = swe.Parareal(p31, p31, fine, coarse, 4)
    U0 = torch.from_numpy(U[0].view(np.float64).copy()).cuda()
    pr.init(U0)
    pr.iterate(3)
    sol = torch.empty(5, 3, p31.nc * 2, dtype=torch.float64, device="cuda")
    pr.solution(sol)
    ref = sol.cpu().numpy().view(np.complex128).reshape(5, 3, -1)
    for n in range(5):
        for f in range(3):
            assert _rel(alone[0][n, f], ref[n, f]) < 1e-12
    pr.close()


def test_admission_by_budget(plans):
    swe, p31, _ = plans
    fine = swe.stepper(swe.SWE_IMEX, 600.0, 2)
    coarse = swe.stepper(swe.SWE_IMEX, 1200.0, 1)
    U = inputs.random_state(31, 2, seed=62)
    per_req = swe.Server.request_bytes(p31, p31, swe.SWE_METHOD_PARAREAL, fine, coarse, 4)
    # charged: state, staging and workspace, more than the state alone
    assert per_req > (3 * 4 + 1) * 3 * p31.nc * 16
    srv = swe.Server(int(per_req * 1.5), 8)          # room for one request at a time
    a = srv.submit(p31, p31, swe.SWE_METHOD_PARAREAL, fine, coarse, 4, 2, U[0])
    b = srv.submit(p31, p31, swe.SWE_METHOD_PARAREAL, fine, coarse, 4, 2, U[1])
    active, queued, _ = srv.step()
    assert active == 1 and queued == 1
    active, queued, done = srv.step()
    assert done == 1
    srv.result(a)                                     # frees its memory: b can be admitted
    for _ in range(3):
        srv.step()
    _, lat, qwait, iters = srv.result(b)
    assert iters == 2 and qwait > 0.0 and lat >= qwait
    srv.close()


def _full_err(a, b, phibar, m):
    w = np.where(m == 0, 1.0, 2.0)
    x, y = a.copy(), b.copy()
    x[0] += np.sqrt(2.0) * phibar
    y[0] += np.sqrt(2.0) * phibar
    return np.sqrt(np.sum(w * np.abs(x - y) ** 2) / np.sum(w * np.abs(y) ** 2))


def test_split_results_same_alone_and_in_mix_across_lanes():
    """Split-precision plans, two truncations with plans of their own (two lanes that run
    concurrently), Parareal requests batched in groups and MGRIT requests, arrivals while
    others run: each result against the same request served alone."""
    from paper_2306_09497_gb300 import swe
    P = swe.SWE_SPLIT_BF16X3
    p63, p31c = swe.Plan(63, 96, 192, prec=P), swe.Plan(31, 48, 96, prec=P)
    p31, p21c = swe.Plan(31, 48, 96, prec=P), swe.Plan(21, 32, 64, prec=P)
    m63, _ = inputs.mn_arrays(63)
    m31, _ = inputs.mn_arrays(31)
    def par(pf, pc, seed, S, iters):
        U = inputs.random_state(pf.M, 1, seed=seed)[0]
        return dict(fine_plan=pf, coarse_plan=pc, method=swe.SWE_METHOD_PARAREAL,
                    fine=swe.stepper(swe.SWE_IMEX, 300.0, 4), coarse=swe.stepper(swe.SWE_IMEX, 600.0, 2, 4, 1e16),
                    S=S, iters=iters, U0_host=U)
    def mg(pf, pc, seed, S):
        U = inputs.random_state(pf.M, 1, seed=seed)[0]
        return dict(fine_plan=pf, coarse_plan=pc, method=swe.SWE_METHOD_MGRIT2,
                    fine=swe.stepper(swe.SWE_IMEX, 300.0, 1), coarse=swe.stepper(swe.SWE_IMEX, 1200.0, 1, 2, 1e6),
                    S=S, cf=4, iters=2, U0_host=U)
    reqs = [par(p63, p31c, 71, 8, 3), par(p31, p21c, 72, 6, 2), mg(p63, p31c, 73, 6), par(p63, p31c, 74, 12, 2),
            par(p63, p31c, 75, 4, 3), mg(p31, p21c, 76, 8)]
    alone = []
    for r in reqs:
        srv = swe.Server(1 << 34, 8)
        alone.append(_run(swe, srv, [r], [0])[0][0])
        srv.close()
    srv = swe.Server(1 << 34, 8)
    mixed = _run(swe, srv, reqs, [0, 0, 0, 1, 1, 2])
    srv.close()
    worst_full, worst = 0.0, 0.0
    for i, r in enumerate(reqs):
        m = m63 if r["fine_plan"] is p63 else m31
        got, ref = mixed[i][0], alone[i]
        for n in range(1, got.shape[0]):
            worst_full = max(worst_full, _full_err(got[n, 0], ref[n, 0], p63.phibar, m))
            for f in range(3):
                if np.linalg.norm(ref[n, f]) > 0:
                    worst = max(worst, _rel(got[n, f], ref[n, f]))
    assert worst_full < 1e-6 and worst < 1e-5, (worst_full, worst)
    for p in (p63, p31c, p31, p21c):
        p.close()
