"""Gaussian-bumps test case (§5.1) on the GPU against the oracle.

The initial geopotential is the analytic three-bump field sampled at each side's own Gauss
nodes and transformed by each side's own forward transform; Phi_bar = g * 29400 m and the
velocity is zero.  Checks: the spectral initial state (1e-12), and two-level MGRIT with IMEX
on a spatially coarsened level (the paper's convergence-study setting, at T63 / T31) in FP64
against the oracle's MGRIT (1e-10 per field), including the KE spectrum of the final iterate.
"""
import numpy as np
import pytest

from oracle import norms, pint
from oracle.sphere import Sphere
from oracle.swe import SWE, Physics, to_dense, to_packed
from paper_2306_09497_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

G = inputs.GRAVITY
PHIBAR = G * inputs.BUMPS_HBAR


def _gpu_bumps(plan):
    """[1][3][2 NC] bumps state from the library's own nodes and forward transform."""
    mu, _ = plan.gauss()
    lon = 2.0 * np.pi * np.arange(plan.nlon) / plan.nlon
    phi = inputs.gaussian_bumps_phi(np.arcsin(mu), lon)
    grid = torch.from_numpy(phi[None].copy()).cuda()
    spec = torch.empty((1, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.sht_forward(grid, spec, 1)
    U0 = torch.zeros((1, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    U0[0, 0] = spec[0]
    return U0


def _oracle_bumps(s):
    phi = inputs.gaussian_bumps_phi(np.arcsin(s.mu), s.lon)
    P = s.real_m0(s.grid_to_sh(phi))
    return (P, np.zeros_like(P), np.zeros_like(P))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_bumps_initial_state_matches_oracle():
    from paper_2306_09497_gb300 import swe
    M, nlat, nlon = 63, 96, 192
    plan = swe.Plan(M, nlat, nlon, phibar=PHIBAR)
    got = _gpu_bumps(plan).cpu().numpy().view(np.complex128).reshape(3, -1)
    s = Sphere(M, nlat, nlon)
    ref = to_packed(s, _oracle_bumps(s))
    assert _rel(got[0], ref[0]) < 1e-12
    assert np.all(got[1:] == 0.0)
    plan.close()


def test_bumps_two_level_mgrit_spatial_coarsening_matches_oracle():
    from paper_2306_09497_gb300 import swe
    sf, sc = Sphere(63, 96, 192), Sphere(31, 48, 96)
    phys = Physics(phibar=PHIBAR)
    swf, swc = SWE(sf, phys), SWE(sc, phys)
    pf = swe.Plan(63, 96, 192, phibar=PHIBAR)
    pc = swe.Plan(31, 48, 96, phibar=PHIBAR)
    dt0, cf, N0, cycles, nu_c = 240.0, 2, 16, 2, 1e6
    steps = [swe.stepper(swe.SWE_IMEX, dt0, 1), swe.stepper(swe.SWE_IMEX, cf * dt0, 1, 2, nu_c)]
    g = swe.MGRIT([pf, pc], steps, N0, cf, 0, cycle=1)
    g.init(_gpu_bumps(pf))

    def trunc(Mb):
        def f(U):
            out = []
            for x in U:
                y = np.zeros((Mb + 1, Mb + 1), dtype=complex)
                k = min(x.shape[0], Mb + 1)
                y[:k, :k] = x[:k, :k]
                out.append(y)
            return tuple(out)
        return f
    m = pint.MGRIT([lambda U, p: swf.imex_step(U, dt0), lambda U, p: swc.imex_step(U, cf * dt0, nu=nu_c, q=2)],
                   N0=N0, cf=cf, nu=0, restrict_space=[trunc(31), None], prolong_space=[trunc(63), None])
    hist = m.run(_oracle_bumps(sf), cycles)
    Nc = N0 // cf
    out = torch.empty((Nc + 1, 3, pf.nc * 2), dtype=torch.float64, device="cuda")
    for k in range(cycles + 1):
        if k > 0:
            g.cycle(1)
        g.cpoints(out)
        got = out.cpu().numpy().view(np.complex128).reshape(Nc + 1, 3, -1)
        for i in range(1, Nc + 1):
            ref = to_packed(sf, hist[k][i])
            for f in range(3):
                assert _rel(got[i, f], ref[f]) < 1e-10, (k, i, f, _rel(got[i, f], ref[f]))
    # KE spectrum of the final iterate at t = T
    E = torch.empty((1, 64), dtype=torch.float64, device="cuda")
    pf.ke_spectrum(out[Nc:Nc + 1], 1, E)
    ref_E = norms.ke_spectrum(hist[cycles][Nc][1], hist[cycles][Nc][2], pf.a)
    assert np.max(np.abs(E.cpu().numpy()[0] - ref_E)) <= 1e-9 * np.max(ref_E)
    g.close()
    pf.close()
    pc.close()
