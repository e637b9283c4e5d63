"""Advective form of the geopotential tendency (Eq. 1 as written, -V.grad(Phi') - Phi' delta)
on the GPU against the oracle's advective form, through the C ABI.  On grids that satisfy the
3/2 rule the two forms are the same projection to rounding; below it they alias differently.

FP64: one nonlinear evaluation 1e-11 per field, IMEX trajectories 1e-10.  Split precision:
the bounds of the flux-form nonlinear evaluation (Phi 5e-5, xi 1e-5, delta 4e-6 M; FP32 grid
values through products) for states with a divergent part, at a narrow batch (FP32 SIMT
contractions) and a batch above 8 columns (tcgen05 GEMMs).
"""
import numpy as np
import pytest

from oracle.sphere import Sphere
from oracle.swe import SWE, to_dense, to_packed
from paper_2306_09497_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()


def _err(a, b, m):
    w = np.where(m == 0, 1.0, 2.0)
    return np.sqrt(np.sum(w * np.abs(a - b) ** 2) / np.sum(w * np.abs(b) ** 2))


def _states(s, sw, S, seed):
    out = []
    for b in range(S):
        xi, noise = inputs.initial_fields(s.M, seed + b)
        xd = s.unpack(xi)
        de = 0.1 * s.unpack(inputs.initial_fields(s.M, seed + 50 + b)[0])
        out.append(to_packed(s, (sw.balanced_geopotential(xd) + s.unpack(noise), xd, de)))
    return np.stack(out)


@pytest.mark.parametrize("M,nlat,nlon", [(31, 36, 96), (31, 48, 96), (63, 96, 192)])
def test_advective_nonlinear_fp64(M, nlat, nlon):
    """On the 3/2-rule grids both forms give the same projection (to rounding); T31 on 36
    latitudes is below the rule, where the two forms alias differently, so there the test also
    sees that the advective path ran."""
    from paper_2306_09497_gb300 import swe
    plan = swe.Plan(M, nlat, nlon)
    plan.set_nphi_form(swe.SWE_NPHI_ADVECTIVE)
    s = Sphere(M, nlat, nlon)
    sw = SWE(s, nphi_form="advective")
    S = 3
    U = _states(s, SWE(s), S, 80)
    out = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.nonlinear(_dev(U), out, S)
    got = out.cpu().numpy().view(np.complex128).reshape(S, 3, -1)
    m, _ = inputs.mn_arrays(M)
    flux = to_packed(s, SWE(s).nonlinear(to_dense(s, U[0])))
    for b in range(S):
        ref = to_packed(s, sw.nonlinear(to_dense(s, U[b])))
        for f in range(3):
            assert _err(got[b, f], ref[f], m) < 1e-11, (b, f, _err(got[b, f], ref[f], m))
    if nlat < (3 * M + 1) / 2:
        assert _err(got[0, 0], flux[0], m) > 1e-6          # the advective path ran
    else:
        assert _err(got[0, 0], flux[0], m) < 1e-11         # same projection as the flux form
    plan.close()


@pytest.mark.parametrize("S", [2, 12])
def test_advective_nonlinear_split(S):
    from paper_2306_09497_gb300 import swe
    M, nlat, nlon = 63, 96, 192
    plan = swe.Plan(M, nlat, nlon, prec=swe.SWE_SPLIT_BF16X3)
    plan.set_nphi_form(swe.SWE_NPHI_ADVECTIVE)
    s = Sphere(M, nlat, nlon)
    sw = SWE(s, nphi_form="advective")
    U = _states(s, SWE(s), S, 90)
    out = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.nonlinear(_dev(U), out, S)
    got = out.cpu().numpy().view(np.complex128).reshape(S, 3, -1)
    m, _ = inputs.mn_arrays(M)
    bound = (5e-5, 1e-5, 4e-6 * M)
    for b in (0, S - 1):
        ref = to_packed(s, sw.nonlinear(to_dense(s, U[b])))
        for f in range(3):
            assert _err(got[b, f], ref[f], m) < bound[f], (b, f, _err(got[b, f], ref[f], m))
    plan.close()


def test_advective_imex_fp64_trajectory():
    """12 IMEX steps with the advective form (4th-order hyperviscosity) against the oracle, on
    T31 with 36 latitudes (below the 3/2 rule, where the two forms differ)."""
    from paper_2306_09497_gb300 import swe
    M, nlat, nlon, S, dt, nsteps = 31, 36, 96, 2, 600.0, 12
    plan = swe.Plan(M, nlat, nlon)
    plan.set_nphi_form(swe.SWE_NPHI_ADVECTIVE)
    s = Sphere(M, nlat, nlon)
    sw = SWE(s, nphi_form="advective")
    U0 = _states(s, SWE(s), S, 100)
    out = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.propagate(swe.stepper(swe.SWE_IMEX, dt, nsteps, 4, 1e16), _dev(U0), out, S)
    got = out.cpu().numpy().view(np.complex128).reshape(S, 3, -1)
    m, _ = inputs.mn_arrays(M)
    for b in range(S):
        U = to_dense(s, U0[b])
        for _ in range(nsteps):
            U = sw.imex_step(U, dt, nu=1e16, q=4)
        ref = to_packed(s, U)
        for f in range(3):
            assert _err(got[b, f], ref[f], m) < 1e-10, (b, f, _err(got[b, f], ref[f], m))
    # switching back gives the flux form again
    plan.set_nphi_form(swe.SWE_NPHI_FLUX)
    N = torch.empty_like(out)
    plan.nonlinear(_dev(U0), N, S)
    flux = to_packed(s, SWE(s).nonlinear(to_dense(s, U0[0])))
    got_n = N.cpu().numpy().view(np.complex128).reshape(S, 3, -1)
    assert _err(got_n[0, 0], flux[0], m) < 1e-11
    plan.close()
