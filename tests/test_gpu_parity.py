"""GPU parity of the FP64 path against the oracle, through the C ABI.

Tolerance: FP64 paths must agree with the oracle to 1e-10 relative L2 per field
(area-weighted L2 = Parseval norm of the spectral coefficients); single
transforms and operators are held to tighter bounds derived from their
rounding (a handful of Legendre/DFT sums of length <= nlon: 1e-12).
"""
import numpy as np
import pytest

from oracle.sphere import Sphere
from oracle.swe import SWE, to_dense, to_packed
from paper_2306_09497_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def _swe():
    from paper_2306_09497_gb300 import swe
    return swe


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()


def _host_c(t, shape):
    return t.cpu().numpy().view(np.complex128).reshape(shape)


def _relL2(a, b, m=None):
    """Area-weighted relative L2 (Parseval) of packed coefficient vectors."""
    w = 1.0 if m is None else np.where(m == 0, 1.0, 2.0)
    num = np.sqrt(np.sum(w * np.abs(a - b) ** 2))
    den = np.sqrt(np.sum(w * np.abs(b) ** 2))
    if den == 0.0:
        return 0.0 if num == 0.0 else np.inf
    return num / den


GRIDS = [(31, 48, 96), (63, 96, 192)]


@pytest.fixture(scope="module", params=GRIDS, ids=lambda g: f"T{g[0]}")
def pair(request):
    M, nlat, nlon = request.param
    swe = _swe()
    plan = swe.Plan(M, nlat, nlon)
    s = Sphere(M, nlat, nlon)
    yield plan, s, SWE(s)
    plan.close()


def test_gauss_grid_matches_oracle(pair):
    plan, s, _ = pair
    mu, w = plan.gauss()
    assert np.max(np.abs(mu - s.mu)) < 1e-15
    assert np.max(np.abs(w - s.w) / s.w) < 1e-12     # both sides ~1e-13 near the poles


def test_sht_inverse_matches_oracle(pair):
    plan, s, _ = pair
    B = 5
    coef = inputs.random_coeffs(s.M, B, seed=1)
    grid = torch.empty((B, s.nlat, s.nlon), dtype=torch.float64, device="cuda")
    plan.sht_inverse(_dev(coef), grid, B)
    got = grid.cpu().numpy()
    for b in range(B):
        ref = s.sh_to_grid(s.unpack(coef[b]))
        assert np.max(np.abs(got[b] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_sht_forward_matches_oracle(pair):
    plan, s, _ = pair
    B = 3   # odd batch: exercises the unpaired FFT column
    g = inputs.random_grid(s.nlat, s.nlon, B, seed=2)
    spec = torch.empty((B, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.sht_forward(torch.from_numpy(g).cuda(), spec, B)
    got = _host_c(spec, (B, plan.nc))
    for b in range(B):
        ref = s.pack(s.grid_to_sh(g[b]))
        assert np.max(np.abs(got[b] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_sht_roundtrip_on_gpu(pair):
    plan, s, _ = pair
    B = 4
    coef = inputs.random_coeffs(s.M, B, seed=3)
    coef[:, : s.M + 1] = coef[:, : s.M + 1].real     # m = 0 row real
    grid = torch.empty((B, s.nlat, s.nlon), dtype=torch.float64, device="cuda")
    spec = torch.empty((B, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.sht_inverse(_dev(coef), grid, B)
    plan.sht_forward(grid, spec, B)
    got = _host_c(spec, (B, plan.nc))
    assert np.max(np.abs(got - coef)) / np.max(np.abs(coef)) < 1e-12


def _state(s, S, seed):
    return inputs.random_state(s.M, S, seed)


def test_linear_operator_matches_oracle(pair):
    plan, s, sw = pair
    S = 3
    U = _state(s, S, 4)
    out = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.linear(_dev(U), out, S)
    got = _host_c(out, (S, 3, plan.nc))
    m, _ = inputs.mn_arrays(s.M)
    for b in range(S):
        ref = to_packed(s, sw.linear(to_dense(s, U[b])))
        for f in range(3):
            assert _relL2(got[b, f], ref[f], m) < 1e-13


def test_implicit_solve_matches_oracle(pair):
    plan, s, sw = pair
    S = 3
    R = _state(s, S, 5)
    out = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    alpha = 450.0
    plan.implicit_solve(alpha, _dev(R), out, S)
    got = _host_c(out, (S, 3, plan.nc))
    m, _ = inputs.mn_arrays(s.M)
    for b in range(S):
        Rd = list(to_dense(s, R[b]))
        Rd[1][0, 0] = 0.0
        Rd[2][0, 0] = 0.0
        ref = to_packed(s, sw.implicit_solve(tuple(Rd), alpha))
        for f in range(3):
            assert _relL2(got[b, f], ref[f], m) < 1e-13


def test_nonlinear_matches_oracle(pair):
    plan, s, sw = pair
    S = 3
    U = _state(s, S, 6)
    out = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.nonlinear(_dev(U), out, S)
    got = _host_c(out, (S, 3, plan.nc))
    m, _ = inputs.mn_arrays(s.M)
    for b in range(S):
        ref = to_packed(s, sw.nonlinear(to_dense(s, U[b])))
        for f in range(3):
            # sums of O(nlat) products with a steeply decaying spectrum: 1e-11
            assert _relL2(got[b, f], ref[f], m) < 1e-11


def test_balanced_init_matches_oracle(pair):
    plan, s, sw = pair
    S = 2
    raw = [inputs.initial_fields(s.M, seed) for seed in (10, 11)]
    xi = np.stack([r[0] for r in raw])
    noise = np.stack([r[1] for r in raw])
    out = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.balance(_dev(xi), _dev(noise), out, S)
    got = _host_c(out, (S, 3, plan.nc))
    m, _ = inputs.mn_arrays(s.M)
    for b in range(S):
        xd = s.unpack(xi[b])
        phi = sw.balanced_geopotential(xd) + s.unpack(noise[b])
        assert _relL2(got[b, 0], s.pack(phi), m) < 1e-12
        assert _relL2(got[b, 1], xi[b], m) < 1e-15
        assert np.max(np.abs(got[b, 2])) == 0.0


@pytest.mark.parametrize("nsteps", [1, 12])
def test_imex_propagation_matches_oracle(pair, nsteps):
    plan, s, sw = pair
    swe = _swe()
    S = 3
    raw = [inputs.initial_fields(s.M, seed) for seed in (20, 21, 22)]
    U0 = []
    for xi, noise in raw:
        xd = s.unpack(xi)
        U0.append(to_packed(s, (sw.balanced_geopotential(xd) + s.unpack(noise), xd, np.zeros_like(xd))))
    U0 = np.stack(U0)
    dt, nu, q = 600.0, 1e14, 4
    out = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
    plan.propagate(swe.stepper(swe.SWE_IMEX, dt, nsteps, q, nu), _dev(U0), out, S)
    got = _host_c(out, (S, 3, plan.nc))
    m, _ = inputs.mn_arrays(s.M)
    for b in range(S):
        U = to_dense(s, U0[b])
        for _ in range(nsteps):
            U = sw.imex_step(U, dt, nu=nu, q=q)
        ref = to_packed(s, U)
        for f in range(3):
            assert _relL2(got[b, f], ref[f], m) < FP64_TOL


def test_propagate_edge_cases():
    swe = _swe()
    plan = swe.Plan(15, 24, 48)
    st = swe.stepper(swe.SWE_IMEX, 300.0, 0)
    U = torch.randn(2, 3, plan.nc * 2, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(U)
    plan.propagate(st, U, out, 2)                     # zero steps = copy
    assert torch.equal(out, U)
    with pytest.raises(swe.SWEError):
        plan.propagate(st, U, out, 0)                 # empty batch rejected
    with pytest.raises(swe.SWEError):
        plan.propagate(swe.stepper(swe.SWE_IMEX, -1.0, 1), U, out, 2)
    with pytest.raises(swe.SWEError):
        swe.Plan(31, 47, 96)                          # odd nlat rejected
    with pytest.raises(swe.SWEError):
        swe.Plan(31, 48, 100)                         # nlon not 2^a 3^b
    plan.close()
