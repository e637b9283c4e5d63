"""T511 (768 x 1536) in the launch configuration of the T511 Parareal workload's fine sweep:
split precision, 256 states propagated by one IMEX step of 3 days / 256 / 34 = 29.78 s
(propagate_F, which cuts the 256 columns into workspace-sized chunks, so a chunk boundary is
crossed), against the FP64 oracle.

The base state is the balanced k^-3 flow with height noise plus a localised 120 m Gaussian
height bump (the workload's initial condition); state k is the base shifted by k grid columns
in longitude, which commutes with every step of the method on a Gaussian grid (f = 2 Omega mu
does not depend on longitude), so one oracle step serves all 256 states, each compared after
the same phase shift.  Bounds as at T255: Phi' 1e-6, xi and delta 1e-5 (Parseval-weighted
relative L2).  Also the split-precision scalar transforms at T511 at a narrow and a wide batch.
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


def test_split_imex_t511_parareal_fine_sweep_batch():
    from paper_2306_09497_gb300 import swe
    M, nlat, nlon, S = 511, 768, 1536, 256
    dt = 3 * 86400.0 / 256 / 34
    s = Sphere(M, nlat, nlon)
    sw = SWE(s)
    xi, noise = inputs.initial_fields(M, 4)
    xd = s.unpack(xi)
    bump = s.grid_to_sh(inputs.single_bump_phi(np.arcsin(s.mu), s.lon))
    base = to_packed(s, (sw.balanced_geopotential(xd) + s.unpack(noise) + bump, xd, np.zeros_like(xd)))
    m, _ = inputs.mn_arrays(M)
    shift = lambda U, k: U * np.exp(-1j * m * (2.0 * np.pi * k / nlon))[None, :]
    U0 = np.stack([shift(base, k) for k in range(S)])
    plan = swe.Plan(M, nlat, nlon, prec=swe.SWE_SPLIT_BF16X3)
    out = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.propagate(swe.stepper(swe.SWE_IMEX, dt, 1), _dev(U0), out, S)
    got = out.cpu().numpy().view(np.complex128).reshape(S, 3, -1)
    plan.close()
    ref_base = to_packed(s, sw.imex_step(to_dense(s, base), dt))
    w = np.where(m == 0, 1.0, 2.0)
    worst = np.zeros(3)
    for k in range(S):
        ref = shift(ref_base, k)
        for f in range(3):
            e = np.sqrt(np.sum(w * np.abs(got[k, f] - ref[f]) ** 2) / np.sum(w * np.abs(ref[f]) ** 2))
            worst[f] = max(worst[f], e)
    assert worst[0] < 1e-6 and worst[1] < 1e-5 and worst[2] < 1e-5, worst


@pytest.fixture(scope="module")
def t511():
    from paper_2306_09497_gb300 import swe
    plan = swe.Plan(511, 768, 1536, prec=swe.SWE_SPLIT_BF16X3)
    yield plan, Sphere(511, 768, 1536)
    plan.close()


# 6 fields: narrow FP32 contraction; 20: tcgen05 GEMMs.  Both take the two-warp lane-group
# longitude transforms of nlon = 1536.  Bounds twice those at T255: the FP32 rounding of the
# Fourier data and of the sums grows with the number of terms summed, sqrt(nlat nlon) for the
# white-noise forward input (twice T255's).
@pytest.mark.parametrize("B", [6, 20])
def test_split_sht_inverse_t511(t511, B):
    plan, s = t511
    coef = inputs.random_coeffs(s.M, B, seed=23)
    grid = torch.empty((B, s.nlat, s.nlon), dtype=torch.float32, device="cuda")
    plan.sht_inverse(_dev(coef), grid, B)
    got = grid.cpu().numpy().astype(np.float64)
    for b in (0, B - 1):
        ref = s.sh_to_grid(s.unpack(coef[b]))
        assert np.max(np.abs(got[b] - ref)) < 2e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("B", [5, 20])
def test_split_sht_forward_t511(t511, B):
    plan, s = t511
    g = inputs.random_grid(s.nlat, s.nlon, B, seed=24)
    spec = torch.empty((B, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.sht_forward(torch.from_numpy(g.astype(np.float32)).cuda(), spec, B)
    got = spec.cpu().numpy().view(np.complex128).reshape(B, -1)
    for b in (0, B - 1):
        ref = s.pack(s.grid_to_sh(g[b].astype(np.float32).astype(np.float64)))
        assert np.max(np.abs(got[b] - ref)) < 1e-5 * np.max(np.abs(ref))
