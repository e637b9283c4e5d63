"""Parity of the configurations that the benchmark runs, against the FP64 oracle.

* The SL-SI-SETTLS coarse levels of the T255 MGRIT workload run on T127 (192 x 384) in split
  precision: level 1 relaxes 456 C-intervals at once with the one-step scheme (Delta t =
  4 Delta t_0 = 236.84 s), level 2 is the serial coarsest level with the two-step scheme
  (Delta t = 16 Delta t_0 = 947.37 s, one state); both with nu = 1e7 m^2/s, q = 2.
  State k of the 456 is the balanced base state rotated by k grid columns in longitude: the
  Gaussian grid is uniform in longitude, f = 2 Omega mu does not depend on it, and a shift by
  whole columns commutes with the FFT, the grid products, the departure-point search and the
  interpolation stencils, so one oracle run serves every state (each compared after the same
  rotation of the oracle result).
* Parareal with a spatially coarser coarse propagator (G = P phi_c R, R spectral truncation,
  P zero padding) in split precision, against the oracle's Parareal with the same transfers.
* The FP64 plain path (the denominator of the mixed/FP64 ratio) at T255.

Split-precision bounds (Parseval-weighted relative L2): full height field 1e-6 (the stated
height bound); Phi' and xi 1e-5 (every SL step re-synthesises the state from FP32 grid
values); delta 1e-4: the balanced initial states have no divergence, so after a few steps
delta is 3 to 4 orders of magnitude below the other fields while the FP32 rounding of the
synthesis scales with the whole state (measured at T127: 1.3e-5 and 3.8e-5; the same bound as
for the MGRIT iterates).  FP64: 1e-10.
"""
import numpy as np
import pytest

from oracle import pint
from oracle.sphere import Sphere
from oracle.swe import SWE, to_dense, to_packed
from paper_2306_09497_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT0 = 432000.0 / 7296.0


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()


def _err(a, b, m):
    w = np.where(m == 0, 1.0, 2.0)
    return np.sqrt(np.sum(w * np.abs(a - b) ** 2) / np.sum(w * np.abs(b) ** 2))


def _full(x, phibar):
    y = x.copy()
    y[0] += np.sqrt(2.0) * phibar           # Phi_bar on P_0^0 = 1/sqrt(2)
    return y


def _balanced(s, sw, seed):
    xi, noise = inputs.initial_fields(s.M, seed)
    xd = s.unpack(xi)
    return to_packed(s, (sw.balanced_geopotential(xd) + s.unpack(noise), xd, np.zeros_like(xd)))


@pytest.fixture(scope="module")
def t127():
    s = Sphere(127, 192, 384)
    sw = SWE(s)
    return s, sw, _balanced(s, sw, 3)


def _check_all(got, ref_base, m, nlon, phibar, tol_f, tol_delta=1e-4):
    shift = lambda U, k: U * np.exp(-1j * m * (2.0 * np.pi * k / nlon))[None, :]
    worst = np.zeros(4)
    for k in range(got.shape[0]):
        ref = shift(ref_base, k)
        worst[0] = max(worst[0], _err(_full(got[k, 0], phibar), _full(ref[0], phibar), m))
        for f in range(3):
            worst[1 + f] = max(worst[1 + f], _err(got[k, f], ref[f], m))
    assert worst[0] < 1e-6 and worst[1] < tol_f and worst[2] < tol_f and worst[3] < tol_delta, worst
    return worst


def test_split_sl_one_step_level1_batch_of_456(t127):
    """Level-1 relaxation launch: 456 states, 2 one-step SL-SI-SETTLS steps of 236.84 s."""
    from paper_2306_09497_gb300 import swe
    s, sw, base = t127
    M, nlat, nlon, S, nsteps, dt = 127, 192, 384, 456, 2, 4 * DT0
    m, _ = inputs.mn_arrays(M)
    U0 = np.stack([base * np.exp(-1j * m * (2.0 * np.pi * k / nlon))[None, :] for k in range(S)])
    plan = swe.Plan(M, nlat, nlon, prec=swe.SWE_SPLIT_BF16X3)
    out = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.propagate(swe.stepper(swe.SWE_SLSI_SETTLS_1STEP, dt, nsteps, 2, 1e7), _dev(U0), out, S)
    assert plan.check() == swe.SWE_OK
    got = out.cpu().numpy().view(np.complex128).reshape(S, 3, -1)
    U = to_dense(s, base)
    for _ in range(nsteps):
        U = sw.sl_si_settls_step(U, None, dt, nu=1e7, q=2)
    _check_all(got, to_packed(s, U), m, nlon, plan.phibar, 1e-5)
    plan.close()


def test_split_sl_two_step_coarsest_chain(t127):
    """Level-2 serial chain: one state, 4 two-step SL-SI-SETTLS steps of 947.37 s (the first
    one-step)."""
    from paper_2306_09497_gb300 import swe
    s, sw, base = t127
    M, nlat, nlon, nsteps, dt = 127, 192, 384, 4, 16 * DT0
    m, _ = inputs.mn_arrays(M)
    plan = swe.Plan(M, nlat, nlon, prec=swe.SWE_SPLIT_BF16X3)
    out = torch.empty((1, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.propagate(swe.stepper(swe.SWE_SLSI_SETTLS, dt, nsteps, 2, 1e7), _dev(base[None]), out, 1)
    got = out.cpu().numpy().view(np.complex128).reshape(1, 3, -1)
    U, prev = to_dense(s, base), None
    for k in range(nsteps):
        nxt = sw.sl_si_settls_step(U, prev if k > 0 else None, dt, nu=1e7, q=2)
        prev, U = U, nxt
    _check_all(got, to_packed(s, U), m, nlon, plan.phibar, 1e-5)
    plan.close()


def _trunc(Mb):
    def f(U):
        out = []
        for x in U:
            y = np.zeros((Mb + 1, Mb + 1), dtype=complex)
            k = min(x.shape[0], Mb + 1)
            y[:k, :k] = x[:k, :k]
            out.append(y)
        return tuple(out)
    return f


@pytest.mark.parametrize("S,K", [(4, 3), (12, 2)])
def test_split_parareal_with_spatial_coarsening(S, K):
    """T63 fine (IMEX, 4 x 240 s per slice) / T31 coarse (IMEX, 2 x 480 s, q = 4, nu = 1e16
    scaled), split precision: every slice boundary after every iteration against the oracle's
    Parareal with G = P phi_c R."""
    from paper_2306_09497_gb300 import swe
    sf, sc = Sphere(63, 96, 192), Sphere(31, 48, 96)
    swf, swc = SWE(sf), SWE(sc)
    U0 = _balanced(sf, swf, 61)
    pf = swe.Plan(63, 96, 192, prec=swe.SWE_SPLIT_BF16X3)
    pc = swe.Plan(31, 48, 96, prec=swe.SWE_SPLIT_BF16X3)
    nu_c = 1e16 * (127.0 / 31.0) ** 4
    fine = swe.stepper(swe.SWE_IMEX, 240.0, 4)
    coarse = swe.stepper(swe.SWE_IMEX, 480.0, 2, 4, nu_c)
    pr = swe.Parareal(pf, pc, fine, coarse, S)
    pr.init(_dev(U0[None]))
    f_prop = lambda U: pint.serial(U, lambda X: swf.imex_step(X, 240.0), 4)
    R, P = _trunc(31), _trunc(63)
    g_prop = lambda U: P(pint.serial(R(U), lambda X: swc.imex_step(X, 480.0, nu=nu_c, q=4), 2))
    hist = pint.parareal(to_dense(sf, U0), f_prop, g_prop, S, K)
    m, _ = inputs.mn_arrays(63)
    sol = torch.empty((S + 1, 3, pf.nc * 2), dtype=torch.float64, device="cuda")
    worst = np.zeros(4)
    for k in range(K + 1):
        if k > 0:
            pr.iterate(1)
        pr.solution(sol)
        got = sol.cpu().numpy().view(np.complex128).reshape(S + 1, 3, -1)
        for n in range(1, S + 1):
            ref = to_packed(sf, hist[k][n])
            worst[0] = max(worst[0], _err(_full(got[n, 0], pf.phibar), _full(ref[0], pf.phibar), m))
            for f in range(3):
                worst[1 + f] = max(worst[1 + f], _err(got[n, f], ref[f], m))
    assert worst[0] < 1e-6 and worst[1] < 1e-5 and worst[2] < 1e-5 and worst[3] < 1e-4, worst
    pr.close()
    pf.close()
    pc.close()


def test_fp64_imex_t255_matches_oracle():
    """The FP64 plain path at the benchmark's truncation: two states, one IMEX step of
    Delta t_0, 1e-10 per field."""
    from paper_2306_09497_gb300 import swe
    M, nlat, nlon = 255, 384, 768
    s = Sphere(M, nlat, nlon)
    sw = SWE(s)
    base = _balanced(s, sw, 3)
    m, _ = inputs.mn_arrays(M)
    U0 = np.stack([base, base * np.exp(-1j * m * (2.0 * np.pi * 5 / nlon))[None, :]])
    plan = swe.Plan(M, nlat, nlon)
    out = torch.empty((2, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.propagate(swe.stepper(swe.SWE_IMEX, DT0, 1), _dev(U0), out, 2)
    got = out.cpu().numpy().view(np.complex128).reshape(2, 3, -1)
    ref = to_packed(s, sw.imex_step(to_dense(s, base), DT0))
    refs = [ref, ref * np.exp(-1j * m * (2.0 * np.pi * 5 / nlon))[None, :]]
    for k in range(2):
        for f in range(3):
            assert _err(got[k, f], refs[k][f], m) < 1e-10, (k, f, _err(got[k, f], refs[k][f], m))
    plan.close()
