"""Pins of the oracle's SWE operators and steppers (§2, App. A) against closed forms and invariants."""
import numpy as np
import pytest

from oracle.sphere import Sphere
from oracle.swe import SWE, Physics, to_dense
from paper_2306_09497_gb300 import inputs


@pytest.fixture(scope="module")
def t31():
    s = Sphere(31, 48, 96)
    return s, SWE(s)


def _rand_state(s, seed):
    U = inputs.random_state(s.M, 1, seed)[0]
    return to_dense(s, U)


def test_coriolis_spectral_equals_grid_products(t31):
    s, sw = t31
    U = _rand_state(s, 11)
    a = sw.coriolis_grid(U)
    b = sw.coriolis_spectral(U)
    for f in (1, 2):
        assert np.max(np.abs(a[f] - b[f])) / np.max(np.abs(a[f])) < 1e-13


def test_cn_gravity_wave_factor():
    """With Omega = 0 a gravity-wave eigenmode is multiplied by (4 + xi)/(4 - xi), xi = lambda dt (§4.1.1)."""
    s = Sphere(31, 48, 96)
    phys = Physics(omega=0.0)
    sw = SWE(s, phys)
    dt = 600.0
    for (m, n) in [(0, 1), (3, 7), (10, 31)]:
        for sign in (+1, -1):
            lam = sign * 1j * np.sqrt(n * (n + 1) * phys.phibar) / phys.a
            U = [np.zeros((32, 32), dtype=complex) for _ in range(3)]
            U[2][m, n] = 1.0
            U[0][m, n] = -phys.phibar / lam
            out = sw.cn_step(tuple(U), dt / 4.0)
            xi = lam * dt
            fac = (4 + xi) / (4 - xi)
            for f in (0, 2):
                assert abs(out[f][m, n] - fac * U[f][m, n]) < 1e-14 * abs(U[f][m, n])
            assert np.max(np.abs(out[1])) == 0.0


def test_cn_solve_residual_with_grid_coriolis(t31):
    """(I - alpha L) U* = (I + alpha L) U, with L_C applied by grid products, to 1e-13."""
    s, sw = t31
    U = _rand_state(s, 12)
    alpha = 300.0

    def L_grid(X):
        _, cx, cd = sw.coriolis_grid(X)
        return (-sw.p.phibar * X[2], cx, -s.lap(X[0]) + cd)

    Us = sw.cn_step(U, alpha)
    lhs = tuple(Us[f] - alpha * L_grid(Us)[f] for f in range(3))
    rhs = tuple(U[f] + alpha * L_grid(U)[f] for f in range(3))
    for f in range(3):
        assert np.max(np.abs(lhs[f] - rhs[f])) / np.max(np.abs(rhs[f])) < 1e-13


def test_viscosity_damping_factor(t31):
    """Backward Euler viscosity multiplies mode n by [1 + dt nu (n(n+1)/a^2)^{q/2}]^{-1} (App. A)."""
    s, sw = t31
    U = _rand_state(s, 13)
    for q, nu in [(2, 1e5), (4, 1e14), (6, 1e25)]:
        out = sw.viscosity(U, 120.0, nu, q)
        n = s.n
        fac = 1.0 / (1.0 + 120.0 * nu * (n * (n + 1) / sw.p.a ** 2) ** (q / 2))
        for f in range(3):
            assert np.allclose(out[f], U[f] * fac, rtol=1e-15, atol=0)


def _solid_body(s, sw, u0=20.0):
    xi = np.zeros((s.M + 1, s.M + 1), dtype=complex)
    # psi = -a u0 mu  =>  xi = lap psi = (2/a^2) a u0 mu = (2 u0 / a) sqrt(2/3) P_1^0
    xi[0, 1] = 2.0 * u0 / sw.p.a / np.sqrt(1.5)
    return xi


def test_balanced_solid_body_matches_closed_form(t31):
    """Nonlinear balance of u = u0 cos(lat): Phi' = -(a Omega u0 + u0^2/2) mu^2 + const."""
    s, sw = t31
    u0 = 20.0
    xi = _solid_body(s, sw, u0)
    phi = sw.balanced_geopotential(xi)
    g = s.sh_to_grid(phi)
    ref = -(sw.p.a * sw.p.omega * u0 + 0.5 * u0 ** 2) * s.mu[:, None] ** 2 * np.ones((1, s.nlon))
    # Phi'_00 = 0: compare with the closed form minus its area mean
    d = g - (ref - np.sum(s.w * ref[:, 0]) / 2.0)
    assert np.max(np.abs(d)) < 1e-10 * np.max(np.abs(ref))


def test_balanced_zonal_flow_is_discrete_steady_state(t31):
    """The balanced solid-body flow has zero total tendency L U + N(U) in the semi-discrete system."""
    s, sw = t31
    xi = _solid_body(s, sw)
    U0 = (sw.balanced_geopotential(xi), xi, np.zeros_like(xi))
    N = sw.nonlinear(U0)
    L = sw.linear(U0)
    u0 = 20.0
    scale = (np.max(np.abs(U0[0])) * u0 / sw.p.a,        # geopotential tendency scale
             np.max(np.abs(L[2])), np.max(np.abs(L[2])))   # vorticity/divergence tendency scale
    for f in range(3):
        assert np.max(np.abs(L[f] + N[f])) <= 1e-12 * scale[f]


def test_imex_drift_from_balanced_flow_is_second_order(t31):
    """Strang splitting (Eq. 3) leaves the balanced state with an O(dt^2) drift over a fixed horizon."""
    s, sw = t31
    xi = _solid_body(s, sw)
    U0 = (sw.balanced_geopotential(xi), xi, np.zeros_like(xi))
    drift = []
    for dt in (240.0, 120.0, 60.0):
        U = U0
        for _ in range(int(6000.0 / dt)):
            U = sw.imex_step(U, dt)
        drift.append(np.max(np.abs(U[0] - U0[0])) / np.max(np.abs(U0[0])))
    assert 3.9 < drift[0] / drift[1] < 4.1
    assert 3.9 < drift[1] / drift[2] < 4.1


def test_mass_conserved_by_imex(t31):
    s, sw = t31
    xi, noise = inputs.initial_fields(s.M, 5)
    xi = s.unpack(xi)
    phi = sw.balanced_geopotential(xi) + s.unpack(noise)
    phi[0, 0] = 123.0
    U = (phi, xi, np.zeros_like(xi))
    for _ in range(20):
        U = sw.imex_step(U, 120.0, nu=1e5, q=2)
    assert abs(U[0][0, 0] - 123.0) < 1e-12 * np.max(np.abs(phi))


def test_imex_linear_limit_is_cn_squared():
    """For an infinitesimal state N is negligible and one IMEX step equals two CN(dt/4) steps."""
    s = Sphere(15, 24, 48)
    sw = SWE(s)
    U = _rand_state(s, 14)
    U = tuple(x * 1e-9 for x in U)
    a = sw.imex_step(U, 300.0)
    b = sw.cn_step(sw.cn_step(U, 75.0), 75.0)
    for f in range(3):
        assert np.max(np.abs(a[f] - b[f])) < 1e-6 * np.max(np.abs(b[f]))


# ---------------- semi-Lagrangian pieces ----------------
def test_sl_interpolation_exact_at_nodes_and_smooth_fields(t31):
    s, sw = t31
    lat = np.arcsin(s.mu)
    lon = s.lon
    LAT, LON = np.meshgrid(lat, lon, indexing="ij")
    # Cartesian coordinate fields are smooth on the sphere, including across the poles
    fx = np.cos(LAT) * np.cos(LON)
    fz = np.sin(LAT)
    got = sw._interp([fx], LAT, LON)[0]
    assert np.max(np.abs(got - fx)) < 1e-14
    rng = np.random.default_rng(4)
    pl = np.arcsin(rng.uniform(-1, 1, 2000))
    pl[:50] = rng.uniform(lat[0], np.pi / 2, 50)              # inside the polar caps
    pl[50:100] = rng.uniform(-np.pi / 2, lat[-1], 50)
    po = rng.uniform(0, 2 * np.pi, 2000)
    gx, gz = sw._interp([fx, fz], pl, po)
    assert np.max(np.abs(gx - np.cos(pl) * np.cos(po))) < 2e-5
    assert np.max(np.abs(gz - np.sin(pl))) < 2e-5


def test_sl_departure_points_solid_body(t31):
    """Solid-body rotation about the axis: departures lie upstream by u0 dt / a along the latitude circle."""
    s, sw = t31
    u0 = 20.0
    xi = _solid_body(s, sw, u0)
    z = np.zeros_like(xi)
    vel = sw._cart_velocity((z, xi, z))
    dt = 1800.0
    latd, lond = sw.departure_points(vel, vel, dt)
    lat = np.arcsin(s.mu)[:, None]
    dlon = np.mod(s.lon[None, :] - lond + np.pi, 2 * np.pi) - np.pi
    ang = u0 * dt / sw.p.a
    assert np.max(np.abs(dlon - ang)) < 1e-3 * ang
    assert np.max(np.abs(latd - lat)) < 1e-3 * ang


def test_sl_step_without_wind_is_crank_nicolson():
    """With V = 0 and N_R = 0 the departure points are the arrival points and Eq. 7 is CN with alpha = dt/2."""
    s = Sphere(31, 48, 96)
    sw = SWE(s)
    U = _rand_state(s, 15)
    U = (U[0], np.zeros_like(U[1]), np.zeros_like(U[2]))
    a = sw.sl_si_settls_step(U, None, 900.0)
    b = sw.cn_step(U, 450.0)
    for f in range(3):
        assert np.max(np.abs(a[f] - b[f])) < 1e-12 * max(np.max(np.abs(b[f])), 1e-300) + 1e-300


def test_nonlinear_terms_are_exactly_quadratic(t31):
    """N of Eq. 1 (flux forms of N_Phi, N_xi, N_delta) is homogeneous of degree 2 in the state:
    N(eps U) = eps^2 N(U).  A linear term left inside N (Phi_bar in the mass flux, f in the
    vorticity flux; both belong to L) breaks this."""
    s, sw = t31
    U = (_rand_state(s, 41)[0], _rand_state(s, 42)[1], _rand_state(s, 43)[2])
    N1 = sw.nonlinear(U)
    for eps in (0.5, 3.0):
        Ne = sw.nonlinear(tuple(eps * x for x in U))
        for f in range(3):
            assert np.max(np.abs(Ne[f] - eps ** 2 * N1[f])) <= 1e-12 * eps ** 2 * np.max(np.abs(N1[f]))


def test_rigid_rotation_advects_geopotential_exactly(t31):
    """u = u0 cos(lat), delta = 0: N_Phi = -div(Phi' V) = -(u0 / a) dPhi'/dlambda, i.e. -(i m u0 / a)
    Phi'_mn, exactly on the 3/2 grid (Phi' u cos(lat) / cos^2(lat) = u0 Phi' is band-limited);
    the zonal vorticity is not advected (N_xi = 0)."""
    s, sw = t31
    u0 = 20.0
    xi = _solid_body(s, sw, u0)
    phi = _rand_state(s, 44)[0]
    N = sw.nonlinear((phi, xi, np.zeros_like(xi)))
    ref = -1j * s.m * u0 / sw.p.a * phi * s.mask
    assert np.max(np.abs(N[0] - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(N[1])) <= 1e-12 * u0 / sw.p.a * np.max(np.abs(xi)) * s.M


def test_zonal_flow_has_no_mass_or_vorticity_flux_divergence(t31):
    """A zonal state (m = 0 only, delta = 0) has purely zonal fluxes Phi' V and xi V, whose
    divergence is a lambda-derivative of a lambda-independent field: N_Phi = N_xi = 0, while
    N_delta (the balance forcing) is not zero."""
    s, sw = t31
    R = _rand_state(s, 45)
    phi = np.zeros_like(R[0])
    xi = np.zeros_like(R[1])
    phi[0, :] = R[0][0, :].real
    xi[0, 1:] = R[1][0, 1:].real
    N = sw.nonlinear((phi, xi, np.zeros_like(xi)))
    scale = np.max(np.abs(N[2]))
    assert scale > 0.0
    assert np.max(np.abs(N[0])) <= 1e-12 * np.max(np.abs(phi)) * np.max(np.abs(xi)) * s.M
    assert np.max(np.abs(N[1])) <= 1e-12 * scale


# ---------------------------------------------------------------------------------------
# advective form of the geopotential tendency (Eq. 1 as written): -V.grad(Phi') - Phi' delta
def test_advective_nphi_rigid_rotation_is_exact():
    """Solid-body rotation u = u0 cos(lat), v = 0: V.grad(Phi') = (u0/a) dPhi'/dlambda exactly,
    delta = 0, so N_Phi = -i m (u0/a) Phi'_mn for any band-limited Phi'."""
    s = Sphere(31, 48, 96)
    sw = SWE(s, nphi_form="advective")
    u0 = 30.0
    xi = np.zeros((32, 32), dtype=complex)
    xi[0, 1] = 2.0 * u0 / sw.p.a * np.sqrt(2.0 / 3.0)
    Phi = s.unpack(inputs.random_state(31, 1, seed=17)[0, 0])
    N = sw.nphi_advective((Phi, xi, np.zeros_like(xi)))
    ref = -1j * s.m * (u0 / sw.p.a) * Phi
    assert np.max(np.abs(N - s.real_m0(ref))) < 1e-12 * np.max(np.abs(ref))


def test_advective_nphi_equals_flux_form_on_an_oversampled_grid():
    """-V.grad(Phi') - Phi' delta = -div(Phi' V) analytically; with both integrands resolved
    (an oversampled Gaussian grid) the two discrete forms agree to quadrature accuracy.  A
    sign, a factor a or a swapped wind component in either form breaks the agreement."""
    M = 10
    s = Sphere(M, 64, 128)
    U = tuple(s.unpack(x) for x in inputs.random_state(M, 1, seed=23, scale=(1e3, 1e-5, 4e-6))[0])
    Na = SWE(s, nphi_form="advective").nonlinear(U)[0]
    Nf = SWE(s, nphi_form="flux").nonlinear(U)[0]
    assert np.max(np.abs(Na - Nf)) < 1e-9 * np.max(np.abs(Nf))


def test_advective_and_flux_forms_agree_on_the_three_halves_grid():
    """On a grid that satisfies the 3/2 rule every integrand of either form is a polynomial in
    mu (the (1 - mu^2) denominators cancel against the factors of U, V and P_n^m), so both are
    exact projections of the same expression and agree to rounding; mass is conserved."""
    M = 31
    s = Sphere(M, 48, 96)
    U = tuple(s.unpack(x) for x in inputs.random_state(M, 1, seed=29, scale=(1e3, 1e-5, 4e-6))[0])
    Na = SWE(s, nphi_form="advective").nonlinear(U)[0]
    Nf = SWE(s, nphi_form="flux").nonlinear(U)[0]
    assert np.max(np.abs(Na - Nf)) < 1e-12 * np.max(np.abs(Nf))
    assert abs(Nf[0, 0]) < 1e-12 * np.max(np.abs(Nf))         # no mass tendency
    assert abs(Na[0, 0]) < 1e-12 * np.max(np.abs(Nf))


def test_advective_and_flux_forms_differ_below_the_three_halves_rule():
    """With too few latitudes (T31 on 36 instead of 48) the products alias, differently in the
    two forms: the advective form is a computation of its own."""
    M = 31
    s = Sphere(M, 36, 96)
    U = tuple(s.unpack(x) for x in inputs.random_state(M, 1, seed=29, scale=(1e3, 1e-5, 4e-6))[0])
    Na = SWE(s, nphi_form="advective").nonlinear(U)[0]
    Nf = SWE(s, nphi_form="flux").nonlinear(U)[0]
    d = np.max(np.abs(Na - Nf)) / np.max(np.abs(Nf))
    assert 1e-5 < d < 1e-1
