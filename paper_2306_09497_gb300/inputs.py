"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module draws random numbers and lays them out; it holds none of the
shallow-water method's arithmetic (no transforms, no operators, no stepping).
Both sides receive exactly the arrays produced here and build everything else
(balanced height, time stepping) with their own code.

Recipe (stand-in for the paper's test cases of §5, whose jet initial condition
is only cited, not defined):

* vorticity: complex Gaussian spherical-harmonic coefficients for
  1 <= n <= M, 0 <= m <= n (real for m = 0), with per-coefficient variance
  proportional to n(n+1) n^-3 / (2n+1), so that the kinetic-energy spectrum
  (§5.1, KE spectrum formula) falls off as n^-3; rescaled so that the global
  root-mean-square wind is ``rms_wind`` (20 m/s).
* height noise: band-limited white noise in the geopotential, rms ``g * 10 m``.
* divergence: zero.

Coefficients use the library's storage: m-major triangular (for each m the
entries n = m..M are contiguous), complex128, orthonormal associated Legendre
functions (integral over mu in [-1, 1] of P^2 is 1) and real fields expanded
as  f = sum_n f_{0n} P_n^0 + 2 Re sum_{m>=1} sum_n f_{mn} P_n^m e^{i m lambda}.
With that convention the area mean of f^2 is
(1/2) * sum_{m,n} c_m |f_{mn}|^2 with c_0 = 1, c_m = 2 (m >= 1), which is the
only identity used below to set amplitudes.
"""
from __future__ import annotations

import numpy as np

EARTH_RADIUS = 6371.22e3      # m            (§4.1, value of a)
EARTH_OMEGA = 7.292e-5        # 1/s          (§4.1, value of Omega)
GRAVITY = 9.80616             # m/s^2        (§5.1)
PHI_BAR = 1.0e5               # m^2/s^2      (§4.1, mean geopotential)


def ncoef(M: int) -> int:
    """Number of complex coefficients of a triangular truncation T_M (m >= 0)."""
    return (M + 1) * (M + 2) // 2


def mn_arrays(M: int):
    """(m, n) of every packed coefficient, in storage order."""
    m = np.concatenate([np.full(M + 1 - mm, mm) for mm in range(M + 1)])
    n = np.concatenate([np.arange(mm, M + 1) for mm in range(M + 1)])
    return m, n


def _mean_square(coef: np.ndarray, m: np.ndarray) -> float:
    c = np.where(m == 0, 1.0, 2.0)
    return 0.5 * float(np.sum(c * np.abs(coef) ** 2))


def _complex_normal(rng: np.random.Generator, m: np.ndarray) -> np.ndarray:
    z = rng.standard_normal(m.size) + 1j * rng.standard_normal(m.size)
    z[m == 0] = np.sqrt(2.0) * z[m == 0].real    # real coefficients for m = 0
    return z


def vorticity_coeffs(M: int, seed: int, rms_wind: float = 20.0,
                     a: float = EARTH_RADIUS) -> np.ndarray:
    """Random vorticity with an n^-3 kinetic-energy spectrum and rms wind ``rms_wind``.

    For a non-divergent flow the area-mean of |V|^2 equals the area mean of
    psi * (-lap psi) = sum c_m a^2/(n(n+1)) |xi_mn|^2 / 2.
    """
    rng = np.random.default_rng(seed)
    m, n = mn_arrays(M)
    nn = np.maximum(n, 1).astype(np.float64)
    var = nn * (nn + 1.0) * nn ** -3.0 / (2.0 * nn + 1.0)
    xi = _complex_normal(rng, m) * np.sqrt(var)
    xi[n == 0] = 0.0
    c = np.where(m == 0, 1.0, 2.0)
    ke2 = 0.5 * np.sum(c * a * a / (nn * (nn + 1.0)) * np.abs(xi) ** 2)  # mean |V|^2
    return xi * (rms_wind / np.sqrt(ke2))


def height_noise_coeffs(M: int, seed: int, rms_height: float = 10.0,
                        g: float = GRAVITY) -> np.ndarray:
    """Band-limited white noise in the geopotential, rms ``g * rms_height`` m^2/s^2."""
    rng = np.random.default_rng(seed + 7919)
    m, n = mn_arrays(M)
    z = _complex_normal(rng, m)
    z[n == 0] = 0.0
    return z * (g * rms_height / np.sqrt(_mean_square(z, m)))


def initial_fields(M: int, seed: int):
    """Raw random inputs of one forecast: (vorticity, height-noise) coefficients.

    The balanced geopotential is computed from the vorticity by each side's
    own nonlinear-balance routine; the noise is then added to it.
    """
    return vorticity_coeffs(M, seed), height_noise_coeffs(M, seed)


def random_state(M: int, nstate: int, seed: int, scale=(1.0e3, 1.0e-5, 1.0e-6)) -> np.ndarray:
    """Generic random band-limited states [nstate][3][NC] (Phi', xi, delta).

    Coefficients decay like n^-2 so the fields are smooth; amplitudes follow
    ``scale`` (geopotential m^2/s^2, vorticity 1/s, divergence 1/s).  Used for
    transform and operator parity checks where no physical balance is needed.
    """
    rng = np.random.default_rng(seed)
    m, n = mn_arrays(M)
    decay = 1.0 / (1.0 + n.astype(np.float64)) ** 2
    out = np.empty((nstate, 3, m.size), dtype=np.complex128)
    for s in range(nstate):
        for f in range(3):
            z = _complex_normal(rng, m) * decay
            z[n == 0] = 0.0 if f > 0 else z[n == 0]
            out[s, f] = z * (scale[f] / np.sqrt(_mean_square(z, m)))
    return out


def random_coeffs(M: int, nbatch: int, seed: int) -> np.ndarray:
    """Random band-limited scalar coefficient sets [nbatch][NC] with unit-order values."""
    rng = np.random.default_rng(seed)
    m, _ = mn_arrays(M)
    out = np.empty((nbatch, m.size), dtype=np.complex128)
    for b in range(nbatch):
        out[b] = _complex_normal(rng, m)
    return out


def random_grid(nlat: int, nlon: int, nbatch: int, seed: int) -> np.ndarray:
    """Random grid fields [nbatch][nlat][nlon] (not band-limited)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nbatch, nlat, nlon))


# ---------------------------------------------------------------------------------------------
# Gaussian-bumps test case of §5.1 (analytic; no random numbers)
BUMPS_HBAR = 29400.0                       # m, mean height: Phi_bar = g * 29400
BUMPS_AMPLITUDE = 6000.0                   # m, bump amplitude A (read as a height, times g)
BUMPS_CENTRES = ((np.pi / 5.0, np.pi / 3.0), (6.0 * np.pi / 5.0, np.pi / 5.0), (8.0 * np.pi / 5.0, -np.pi / 4.0))
BUMPS_WIDTHS = (20.0, 80.0, 360.0)


def gaussian_bumps_phi(lat: np.ndarray, lon: np.ndarray, g: float = GRAVITY) -> np.ndarray:
    """Geopotential perturbation of the three Gaussian bumps at the given latitudes (radians,
    any order) and longitudes: Phi' = g A sum_i exp(-a_i d_i^2), d_i the great-circle angle to
    bump centre i (§5.1); returns [len(lat)][len(lon)].  The velocity is zero."""
    la = np.asarray(lat, dtype=np.float64)[:, None]
    lo = np.asarray(lon, dtype=np.float64)[None, :]
    out = np.zeros((la.shape[0], lo.shape[1]))
    for (lc, tc), ai in zip(BUMPS_CENTRES, BUMPS_WIDTHS):
        c = np.sin(la) * np.sin(tc) + np.cos(la) * np.cos(tc) * np.cos(lo - lc)
        d = np.arccos(np.clip(c, -1.0, 1.0))
        out += np.exp(-ai * d * d)
    return g * BUMPS_AMPLITUDE * out


def single_bump_phi(lat: np.ndarray, lon: np.ndarray, height: float = 120.0, width: float = 80.0,
                    centre=(np.pi / 5.0, np.pi / 3.0), g: float = GRAVITY) -> np.ndarray:
    """A localised Gaussian height bump, g * height * exp(-width d^2), d the great-circle angle to
    the centre (longitude, latitude), at the given latitudes and longitudes (radians); the form of
    the §5.1 bumps, with a 120 m default height.  Returns [len(lat)][len(lon)]."""
    la = np.asarray(lat, dtype=np.float64)[:, None]
    lo = np.asarray(lon, dtype=np.float64)[None, :]
    lc, tc = centre
    c = np.sin(la) * np.sin(tc) + np.cos(la) * np.cos(tc) * np.cos(lo - lc)
    d = np.arccos(np.clip(c, -1.0, 1.0))
    return g * height * np.exp(-width * d * d)
