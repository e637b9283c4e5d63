"""Pins of the oracle's spherical-harmonic machinery (§2.2) against independent references."""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss
from scipy.special import gammaln, lpmv

from oracle.sphere import Sphere, dlegendre_table, gauss_legendre, legendre_table


@pytest.mark.parametrize("nlat", [4, 48, 192, 384])
def test_gauss_nodes_match_numpy(nlat):
    x, w = gauss_legendre(nlat)
    xr, wr = leggauss(nlat)
    order = np.argsort(x)
    assert np.all(np.diff(x) < 0)                     # north to south
    assert np.max(np.abs(x[order] - xr)) < 1e-15
    assert np.max(np.abs(w[order] - wr) / wr) < 1e-9     # numpy's own weights are good to ~4e-10
    assert abs(w.sum() - 2.0) < 1e-13


def test_gauss_exact_for_polynomials():
    nlat = 24
    x, w = gauss_legendre(nlat)
    for p in range(0, 2 * nlat):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.sum(w * x ** p) - exact) < 1e-14


def _normalised_lpmv(m, n, x):
    # scipy's P_n^m carries the Condon-Shortley phase (-1)^m; the oracle's does not.
    lognorm = 0.5 * (np.log((2 * n + 1) / 2.0) + gammaln(n - m + 1) - gammaln(n + m + 1))
    return (-1.0) ** m * np.exp(lognorm) * lpmv(m, n, x)


def test_legendre_matches_scipy():
    mu, _ = gauss_legendre(64)
    P = legendre_table(40, mu)
    for m in range(0, 41, 3):
        for n in range(m, 41, 2):
            ref = _normalised_lpmv(m, n, mu)
            assert np.max(np.abs(P[m, n] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_legendre_closed_forms():
    mu = np.linspace(-0.99, 0.99, 11)
    P = legendre_table(2, mu)
    assert np.allclose(P[0, 0], 1 / np.sqrt(2), atol=1e-16)
    assert np.allclose(P[0, 1], np.sqrt(1.5) * mu, atol=1e-15)
    assert np.allclose(P[1, 1], np.sqrt(3.0) / 2.0 * np.sqrt(1 - mu ** 2), atol=1e-15)
    assert np.allclose(P[0, 2], np.sqrt(2.5) * (3 * mu ** 2 - 1) / 2, atol=1e-15)


@pytest.mark.parametrize("M,nlat", [(31, 48), (255, 384)])
def test_legendre_orthonormal_by_quadrature(M, nlat):
    mu, w = gauss_legendre(nlat)
    P = legendre_table(M, mu)
    worst = 0.0
    for m in range(0, M + 1, max(1, M // 16)):
        B = P[m, m:]                                 # [n, j]
        G = (B * w) @ B.T
        worst = max(worst, np.max(np.abs(G - np.eye(G.shape[0]))))
    assert worst < 1e-13


def test_dlegendre_matches_finite_differences():
    mu = np.linspace(-0.9, 0.9, 37)
    h = 1e-5
    L = 20
    Pext = legendre_table(L + 1, mu)
    H = dlegendre_table(L, mu, Pext)
    Pp = legendre_table(L, mu + h)
    Pm = legendre_table(L, mu - h)
    for m in range(L + 1):
        for n in range(m, L + 1):
            fd = (1 - mu ** 2) * (Pp[m, n] - Pm[m, n]) / (2 * h)
            assert np.max(np.abs(H[m, n] - fd)) < 2e-7 * max(1.0, n * n)


def test_naive_dft_matches_numpy_fft():
    s = Sphere(31, 48, 96)
    rng = np.random.default_rng(1)
    g = rng.standard_normal((48, 96))
    F = s.grid_to_fourier(g)
    ref = np.fft.rfft(g, axis=1)[:, :32] / 96
    assert np.max(np.abs(F - ref)) < 1e-14
    # inverse: Hermitian synthesis
    spec = np.zeros((48, 49), dtype=complex)
    spec[:, :32] = F
    ref_g = np.fft.irfft(spec, n=96, axis=1) * 96
    assert np.max(np.abs(s.fourier_to_grid(F) - ref_g)) < 1e-13


def _random_dense(s, rng):
    f = (rng.standard_normal((s.M + 1, s.M + 1)) + 1j * rng.standard_normal((s.M + 1, s.M + 1))) * s.mask
    return s.real_m0(f)


@pytest.mark.parametrize("M,nlat,nlon", [(31, 48, 96), (63, 96, 192), (127, 192, 384)])
def test_sht_roundtrip(M, nlat, nlon):
    s = Sphere(M, nlat, nlon)
    f = _random_dense(s, np.random.default_rng(M))
    f2 = s.grid_to_sh(s.sh_to_grid(f))
    assert np.max(np.abs(f2 - f)) / np.max(np.abs(f)) < 1e-12


def test_vector_transforms_laplacian_eigenrelation():
    """div of the irrotational flow of chi is lap chi, curl of the rotational flow of psi is lap psi."""
    s = Sphere(31, 48, 96)
    rng = np.random.default_rng(3)
    chi = _random_dense(s, rng)
    psi = _random_dense(s, rng)
    chi[0, 0] = psi[0, 0] = 0.0
    z = np.zeros_like(chi)
    U, V = s.uv_to_grid(z, chi)
    div, curl = s.div_curl_from_grid(U, V)
    ref = -s.nn1 / s.a ** 2 * chi
    assert np.max(np.abs(div - ref)) / np.max(np.abs(ref)) < 1e-13
    assert np.max(np.abs(curl)) / np.max(np.abs(ref)) < 1e-13
    U, V = s.uv_to_grid(psi, z)
    div, curl = s.div_curl_from_grid(U, V)
    ref = -s.nn1 / s.a ** 2 * psi
    assert np.max(np.abs(curl - ref)) / np.max(np.abs(ref)) < 1e-13
    assert np.max(np.abs(div)) / np.max(np.abs(ref)) < 1e-13


def test_solid_body_streamfunction_gives_cosine_wind():
    """psi = -a u0 mu  (a single P_1^0 mode) is the solid-body flow u = u0 cos(lat), v = 0."""
    s = Sphere(31, 48, 96)
    u0 = 20.0
    psi = np.zeros((32, 32), dtype=complex)
    psi[0, 1] = -s.a * u0 / np.sqrt(1.5)               # P_1^0 = sqrt(3/2) mu
    U, V = s.uv_to_grid(psi, np.zeros_like(psi))
    coslat2 = (1 - s.mu ** 2)[:, None]
    assert np.max(np.abs(U - u0 * coslat2)) < 1e-12 * u0
    assert np.max(np.abs(V)) < 1e-12 * u0
