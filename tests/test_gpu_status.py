"""Failure detection and checkpoint/resume through the C ABI (GPU).

No test here faults, traps or hangs the GPU: failures are made on the host (a NaN in the
input state, bits injected into a plan's status word) or by a bounded wait on an
mbarrier that nothing completes, which gives up after a few polls and reports.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2306_09497_gb300 import inputs, swe  # noqa: E402


@pytest.fixture(scope="module")
def plans():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    p64 = swe.Plan(31, 48, 96)
    pmx = swe.Plan(63, 96, 192, prec=swe.SWE_SPLIT_BF16X3)
    yield p64, pmx
    p64.close()
    pmx.close()


def test_injected_timeout_is_reported_once(plans):
    for p in plans:
        assert p.check() == swe.SWE_OK
        p.inject_status(2)
        assert p.check() == swe.SWE_ETIMEOUT
        assert p.check() == swe.SWE_OK


def test_injected_nonfinite_is_reported_and_timeout_wins(plans):
    p = plans[0]
    p.inject_status(1)
    assert p.check() == swe.SWE_EUNSTABLE
    p.inject_status(1)
    p.inject_status(2)
    assert p.check() == swe.SWE_ETIMEOUT
    assert p.check() == swe.SWE_OK
    with pytest.raises(swe.SWEError):
        p.inject_status(4)


@pytest.mark.parametrize("polls", [1, 64, 4096])
def test_bounded_wait_gives_up_and_reports(plans, polls):
    """An mbarrier wait that nothing completes returns after at most `polls` polls and the
    timeout reaches the host as SWE_ETIMEOUT; the context stays usable."""
    p = plans[1]
    p.wait_selftest(polls)
    assert p.check() == swe.SWE_ETIMEOUT
    # the plan still computes correctly afterwards
    coef = torch.from_numpy(inputs.random_coeffs(p.M, 16, seed=2).view(np.float64).copy()).cuda()
    grid = torch.empty((16, p.nlat, p.nlon), dtype=torch.float32, device="cuda")
    back = torch.empty_like(coef)
    p.sht_inverse(coef, grid, 16)
    p.sht_forward(grid, back, 16)
    assert p.check() == swe.SWE_OK
    c = coef.cpu().numpy().view(np.complex128)
    b = back.cpu().numpy().view(np.complex128)
    m, _ = inputs.mn_arrays(p.M)
    c[:, m == 0] = c[:, m == 0].real
    assert np.max(np.abs(b - c)) < 1e-5 * np.max(np.abs(c))


def test_real_tensor_core_work_leaves_status_clear(plans):
    p = plans[1]
    S = 40   # above the narrow-batch limit: the tcgen05 kernels run
    U = torch.from_numpy(inputs.random_state(p.M, S, seed=4).view(np.float64).copy()).cuda()
    N = torch.empty_like(U)
    p.nonlinear(U, N, S)
    assert p.check() == swe.SWE_OK


def test_nan_in_initial_state_returns_unstable(plans):
    p = plans[0]
    U0 = inputs.random_state(p.M, 1, seed=9)[0]
    U0[1, 5] = np.nan
    U0d = torch.from_numpy(U0.view(np.float64).copy()).cuda()
    fine = swe.stepper(swe.SWE_IMEX, 600.0, 3)
    coarse = swe.stepper(swe.SWE_IMEX, 1800.0, 1, 2, 1e5)
    it = swe.Parareal(p, p, fine, coarse, 4, use_graphs=False)
    it.init(U0d)
    with pytest.raises(swe.SWEError) as ei:
        it.iterate(2)
    assert ei.value.status == swe.SWE_EUNSTABLE
    it.close()
    assert p.check() == swe.SWE_OK     # the iteration consumed the word


def test_mgrit_nan_returns_unstable(plans):
    p = plans[0]
    U0 = inputs.random_state(p.M, 1, seed=9)[0]
    U0[0, 3] = np.inf
    U0d = torch.from_numpy(U0.view(np.float64).copy()).cuda()
    steps = [swe.stepper(swe.SWE_IMEX, 600.0, 1), swe.stepper(swe.SWE_IMEX, 1800.0, 1, 2, 1e5)]
    g = swe.MGRIT([p, p], steps, 12, 3, 0, cycle=1)
    g.init(U0d)
    with pytest.raises(swe.SWEError) as ei:
        g.cycle(2)
    assert ei.value.status == swe.SWE_EUNSTABLE
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_checkpoint_resume_reproduces_the_iterate(plans, prec):
    """swe_pint_save after k iterations, swe_pint_load into a fresh solver, one more
    iteration: the same iterate as continuing the original solver."""
    p = plans[0] if prec == "fp64" else plans[1]
    S = 6
    U0 = torch.from_numpy(inputs.random_state(p.M, 1, seed=13).view(np.float64).copy()).cuda()
    fine = swe.stepper(swe.SWE_IMEX, 300.0, 4)
    coarse = swe.stepper(swe.SWE_IMEX, 1200.0, 1, 2, 1e5)
    a = swe.Parareal(p, p, fine, coarse, S)
    a.init(U0)
    a.iterate(2)
    per = 3 * p.nc * 2
    Uh = torch.empty((S + 1) * per, dtype=torch.float64, pin_memory=True)
    Gh = torch.empty(S * per, dtype=torch.float64, pin_memory=True)
    a.save_state(Uh, Gh)
    torch.cuda.synchronize()
    a.iterate(1)
    ua = torch.empty((S + 1) * per, dtype=torch.float64, device="cuda")
    a.solution(ua)
    b = swe.Parareal(p, p, fine, coarse, S)
    b.init(U0)
    b.load_state(Uh, Gh)
    b.iterate(1)
    ub = torch.empty_like(ua)
    b.solution(ub)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)
    # and without the saved coarse results (recomputed serially on load)
    c = swe.Parareal(p, p, fine, coarse, S)
    c.init(U0)
    c.load_state(Uh)
    c.iterate(1)
    uc = torch.empty_like(ua)
    c.solution(uc)
    torch.cuda.synchronize()
    assert torch.equal(ua, uc)
    for x in (a, b, c):
        x.close()
