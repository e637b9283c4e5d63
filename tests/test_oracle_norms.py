"""Pins of the oracle's §5 diagnostics: error norms (Eq. 21, area-weighted L2) and the KE
spectrum of §5.1."""
import numpy as np
import pytest

from oracle import norms
from oracle.sphere import Sphere
from paper_2306_09497_gb300 import inputs

A = 6371.22e3


def _dense(s, M, seed, n=1, scale=(1.0e3, 1.0e-5, 1.0e-6)):
    U = inputs.random_state(M, n, seed=seed, scale=scale)
    return [tuple(s.unpack(U[k, f]) for f in range(3)) for k in range(n)]


def test_parseval_l2_equals_gauss_quadrature_of_grid_fields():
    """Band-limited T_M fields: the squared difference has degree <= 2M, which Gauss
    quadrature on nlat >= M+1 latitudes and the DFT on nlon > 2M longitudes integrate exactly."""
    s = Sphere(31, 48, 96)
    a, b = _dense(s, 31, 3, 2)
    for f in range(3):
        ga, gb = s.sh_to_grid(a[f]), s.sh_to_grid(b[f])
        wq = s.w[:, None] / (2.0 * s.nlon)            # area weights, sum 1
        ref = np.sqrt(np.sum(wq * (ga - gb) ** 2) / np.sum(wq * gb ** 2))
        assert abs(norms.parseval_l2_error(a[f], b[f]) - ref) < 1e-12 * ref


def test_spectral_error_respects_R_norm():
    s = Sphere(31, 48, 96)
    ref = _dense(s, 31, 4)[0][1]
    psi = ref.copy()
    psi[3, 20] += 1e-3 * np.max(np.abs(ref))          # beyond R = 16: invisible there
    assert norms.spectral_error(psi, ref, 16) == 0.0
    assert norms.spectral_error(psi, ref, 20) > 0.0
    psi2 = ref.copy()
    psi2[2, 5] += 1e-4
    e = norms.spectral_error(psi2, ref, 16)
    assert abs(e - 1e-4 / np.max(np.abs(ref[:17, :17]))) < 1e-12 * e


def test_ke_spectrum_solid_body_closed_form():
    """u = u0 cos(lat): xi = 2 u0 mu / a = (2 u0 / a) sqrt(2/3) P_1^0, so E(1) = u0^2 / 3 (the area
    mean of u^2 / 2) and E(n) = 0 for n >= 2."""
    M, u0 = 21, 25.0
    xi = np.zeros((M + 1, M + 1), dtype=complex)
    xi[0, 1] = 2.0 * u0 / A * np.sqrt(2.0 / 3.0)
    E = norms.ke_spectrum(xi, np.zeros_like(xi), A)
    assert abs(E[1] - u0 ** 2 / 3.0) < 1e-12 * u0 ** 2
    assert np.all(E[2:] == 0.0) and E[0] == 0.0


@pytest.mark.parametrize("M", [15, 31])
def test_ke_spectrum_sums_to_mean_kinetic_energy(M):
    """sum_n E(n) equals the area mean of (u^2 + v^2)/2 of the grid wind, integrated with an
    oversampled Gauss grid (u^2 + v^2 is smooth but not a polynomial in mu)."""
    s = Sphere(M, 8 * (M + 1), 4 * (M + 1) + 8)
    U = _dense(s, M, 7 + M, scale=(1.0e3, 1.0e-5, 3.0e-6))[0]
    Ug, Vg = s.uv_to_grid(s.inv_lap(U[1]), s.inv_lap(U[2]))
    ke = 0.5 * (Ug ** 2 + Vg ** 2) / s.coslat2[:, None]
    mean = np.sum(s.w[:, None] * ke) / (2.0 * s.nlon)
    E = norms.ke_spectrum(U[1], U[2], A)
    assert abs(E.sum() - mean) < 1e-10 * mean


def test_ke_spectrum_invariant_under_rotation_in_longitude():
    M = 31
    s = Sphere(M, 48, 96)
    U = _dense(s, M, 8)[0]
    ph = np.exp(1j * 0.7 * np.arange(M + 1))[:, None]
    E0 = norms.ke_spectrum(U[1], U[2], A)
    E1 = norms.ke_spectrum(U[1] * ph, U[2] * ph, A)
    assert np.max(np.abs(E0 - E1)) < 1e-13 * np.max(E0)
