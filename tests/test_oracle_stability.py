"""Pins of the scalar test-ODE schemes and the PinT stability functions of §4."""
import numpy as np
import pytest

from oracle import pint, stability as st


XI_T = 2.5e-4j    # xi_L tilde as printed in §4.1


@pytest.mark.parametrize("xiL", [0.0, 5e3 * XI_T, 1e4 * XI_T, -2.5e4 * XI_T, 0.3 + 0.1j])
@pytest.mark.parametrize("xiN", [0.1j, -0.5 + 0.3j, 1.2j, 0.05])
def test_imex_scalar_amplification(xiL, xiN):
    got = st.imex_step(1.0 + 0j, xiL, xiN)
    assert abs(got - st.A_imex(xiL, xiN)) < 1e-14 * max(1.0, abs(got))
    # the printed A_IMEX-E is the increment of the explicit stage: 1 + printed = implemented
    assert abs(st.A_imex_implicit(xiL) ** 2 * (1 + st.A_imex_explicit_printed(xiN)) - got) < 1e-14 * max(1, abs(got))


def test_imex_implicit_factor_unimodular_on_imaginary_axis():
    for xiL in [1j, 10j, -3j]:
        assert abs(abs(st.A_imex_implicit(xiL)) - 1.0) < 1e-15


@pytest.mark.parametrize("kappa_s", [0.0, np.pi / 10, np.pi / 2, 1.7 * np.pi])
@pytest.mark.parametrize("xiL,xiN", [(1e4 * XI_T, 0.3j), (0.0, -0.2 + 0.5j), (2.5e4 * XI_T, 0.05)])
def test_sl_scalar_recurrence_matches_quadratic_roots(kappa_s, xiL, xiN):
    """The two-step SL-SI-SETTLS recurrence is a combination of r+^n and r-^n, r the roots of Eq. 13."""
    r = st.sl_roots(xiL, xiN, kappa_s)
    u = [1.0 + 0j, 0.7 - 0.2j]
    for _ in range(12):
        u.append(st.sl_step(u[-1], u[-2], xiL, xiN, kappa_s))
    c = np.linalg.solve(np.array([[1, 1], [r[0], r[1]]]), np.array(u[:2]))
    for k, uk in enumerate(u):
        ref = c[0] * r[0] ** k + c[1] * r[1] ** k
        assert abs(uk - ref) < 1e-12 * max(1.0, abs(ref))


def _scalar_prop(A, N):
    return lambda u: u * A ** N


@pytest.mark.parametrize("k", [0, 1, 3, 6])
def test_parareal_scalar_matches_stability_function(k):
    """Brute-force Parareal on u' = (lL + lN) u equals Eq. 17 (§4.2)."""
    n = 12
    xiL, xiN = 1e4 * XI_T / 2, 0.4j / 2
    Af = st.A_imex(xiL / 2, xiN / 2)        # fine: dt/2, two steps per slice
    Ac = st.A_imex(xiL, xiN)                # coarse: one step
    hist = pint.parareal(1.0 + 0j, _scalar_prop(Af, 2), _scalar_prop(Ac, 1), n, k)
    got = hist[k][n]
    ref = st.A_parareal(n, k, Ac, Af ** 2 - Ac)
    assert abs(got - ref) < 1e-12 * max(1.0, abs(ref))


def test_parareal_finite_termination_scalar():
    n = 8
    Af, Ac = 0.97 + 0.2j, 0.9 + 0.3j
    hist = pint.parareal(1.0 + 0j, _scalar_prop(Af, 1), _scalar_prop(Ac, 1), n, n)
    for k in range(n + 1):
        for j in range(k + 1):
            assert abs(hist[k][j] - Af ** j) < 1e-14


def _mgrit_scalar(F, G, n, cf, nu, iters):
    """Two-level MGRIT on the scalar ODE: one fine step = F^(1/cf) is not needed; we set the
    fine level step to f with f^cf = F and the coarse step to G."""
    f = F ** (1.0 / cf)
    m = pint.MGRIT([lambda u, p: u * f, lambda u, p: u * G], N0=n * cf, cf=cf, nu=nu)
    return m.run(1.0 + 0j, iters)


@pytest.mark.parametrize("k", [0, 1, 2, 5])
def test_two_level_mgrit_nu0_is_parareal(k):
    n, cf = 10, 2
    F, G = (0.95 + 0.25j), (0.9 + 0.3j)
    got = _mgrit_scalar(F, G, n, cf, 0, k)[k][n]
    ref = st.A_parareal(n, k, G, F - G)
    assert abs(got - ref) < 1e-12


@pytest.mark.parametrize("nu", [1, 2, 3])
def test_two_level_mgrit_finite_termination(nu):
    """Exact after N_0 / ((nu+1) cf) iterations (§3.2.3)."""
    n, cf = 12, 2
    F, G = (0.95 + 0.25j), (0.9 + 0.3j)
    iters = -(-n // (nu + 1))
    hist = _mgrit_scalar(F, G, n, cf, nu, iters)
    for j in range(n + 1):
        assert abs(hist[iters][j] - F ** j) < 1e-12


@pytest.mark.parametrize("nu", [1, 2])
@pytest.mark.parametrize("k", [1, 2, 4])
def test_two_level_mgrit_matches_recurrence_eq19_interior(nu, k):
    """Brute-force MGRIT follows u^k_n = G u^k_{n-1} + F^nu (F - G) u^{k-1}_{n-nu-1} (Eq. 19);
    its first nu C-points after t = 0 are exact from iteration 1 on (F(CF)^nu relaxation)."""
    n, cf = 14, 2
    F, G = (0.95 + 0.25j), (0.9 + 0.3j)
    hist = _mgrit_scalar(F, G, n, cf, nu, k)
    S = F ** nu * (F - G)
    prev = hist[k - 1]
    cur = hist[k]
    for j in range(nu + 1, n + 1):
        assert abs(cur[j] - (G * cur[j - 1] + S * prev[j - nu - 1])) < 1e-12
    for j in range(1, nu + 1):
        assert abs(cur[j] - F ** j) < 1e-12


@pytest.mark.parametrize("nu", [0, 1, 2, 3])
@pytest.mark.parametrize("k", [0, 1, 3, 5, 10])
def test_mgrit_path_count_closed_form(nu, k):
    """The binomial sum with upper limit min(k, n/(nu+1)) equals the recurrence of Eq. 19; the
    printed limit floor(k/(nu+1)) agrees only when nu = 0 or k = 0 (reading of Eq. 20)."""
    n = 100
    F, G = 0.999 + 0.02j, 0.995 + 0.03j
    rec = st.recurrence_eq19(n, k, nu, F, G)
    pc = st.A_mgrit_pathcount(n, k, nu, F, G)
    assert abs(rec - pc) < 1e-10 * max(1.0, abs(rec))
    pr = st.A_mgrit_printed(n, k, nu, F, G)
    if nu == 0 or k == 0:
        assert abs(pr - pc) < 1e-10 * max(1.0, abs(pc))
    else:
        assert abs(pr - pc) > 1e-8


def test_printed_constants(tmp_path):
    """Physical constants as printed (§4.1, §5.1); see tests/golden/paper_constants.txt."""
    import os
    from paper_2306_09497_gb300 import inputs
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
    vals = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    assert vals["a"] == inputs.EARTH_RADIUS
    assert vals["omega"] == inputs.EARTH_OMEGA
    assert vals["g"] == inputs.GRAVITY
    assert vals["phibar_stability"] == inputs.PHI_BAR
    # the printed xi_L tilde ~ 2.5e-4 does not equal sqrt(phibar)/a (~4.96e-5); recorded as a garble
    assert abs(np.sqrt(vals["phibar_stability"]) / vals["a"] - 4.963e-5) < 1e-8
    assert vals["xiL_tilde_printed"] == 2.5e-4
