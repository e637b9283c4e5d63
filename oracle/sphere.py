"""Spherical-harmonic machinery of §2.2, written as plain sums (oracle; test use only).

Conventions (the paper fixes none of them; any consistent choice gives the
same grid fields):

* mu = sin(latitude); Gauss-Legendre nodes ordered north to south (mu descending).
* longitudes lambda_k = 2 pi k / nlon, k = 0..nlon-1.
* P[m, n, j] = normalised associated Legendre function with
  integral_{-1}^{1} P_n^m(mu)^2 dmu = 1, no Condon-Shortley phase.
* H[m, n, j] = (1 - mu^2) dP_n^m/dmu.
* a real field is f = sum_n f_{0n} P_n^0 + 2 Re sum_{m>=1} sum_n f_{mn} P_n^m e^{i m lambda}
  (the m < 0 coefficients are the complex conjugates, §2.2 Eq. 2).
* spectral arrays inside the oracle are dense complex [m, n] with zeros for n < m.

Every transform is a direct quadrature sum or a naive DFT written as a matrix
product; no FFT and no even/odd folding.
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(nlat: int):
    """Gauss-Legendre nodes mu_j (descending) and weights w_j on [-1, 1].

    Newton iteration for the roots of the Legendre polynomial P_nlat written
    in colatitude t (mu = cos t), from the initial guess t = pi (j - 1/4)/(nlat + 1/2);
    P_nlat and P_{nlat-1} come from the three-term recurrence, and
    dP_nlat/dt = nlat (mu P_nlat - P_{nlat-1}) / sin t.  Weights
    w_j = 2 / ((1 - mu_j^2) P'_nlat(mu_j)^2) = 2 sin^2 t / (nlat (mu P_nlat - P_{nlat-1}))^2.
    Pinned against numpy.polynomial.legendre.leggauss and exact quadrature of monomials.
    """
    j = np.arange(1, nlat + 1, dtype=np.float64)
    t = np.pi * (j - 0.25) / (nlat + 0.5)

    def pn(x):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for k in range(1, nlat):
            p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        return p1, p0                      # P_nlat, P_{nlat-1}

    for _ in range(100):
        x = np.cos(t)
        p1, p0 = pn(x)
        dpdt = nlat * (x * p1 - p0) / np.sin(t)
        dt = p1 / dpdt
        t = t - dt
        if np.max(np.abs(dt)) < 1e-17:
            break
    x = np.cos(t)
    p1, p0 = pn(x)
    w = 2.0 * np.sin(t) ** 2 / (nlat * (x * p1 - p0)) ** 2
    return x, w


def eps(m, n):
    """epsilon_n^m = sqrt((n^2 - m^2) / (4 n^2 - 1)); zero for n <= m.

    Coefficient of the recurrence  mu P_n^m = eps_{n+1}^m P_{n+1}^m + eps_n^m P_{n-1}^m.
    """
    m = np.asarray(m, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    num = np.maximum(n * n - m * m, 0.0)
    return np.sqrt(num / np.maximum(4.0 * n * n - 1.0, 1.0))


def legendre_table(L: int, mu: np.ndarray) -> np.ndarray:
    """P[m, n, j] for 0 <= m <= n <= L at the nodes mu (dense, zero for n < m).

    Sectoral start P_0^0 = 1/sqrt(2), P_m^m = sqrt((2m+1)/(2m)) sqrt(1-mu^2) P_{m-1}^{m-1},
    P_{m+1}^m = sqrt(2m+3) mu P_m^m, then the three-term recurrence in n.
    Pinned against scipy.special.lpmv (rescaled) and Gauss-quadrature
    orthonormality.  Values that underflow double precision near the poles
    are exponentially small (below 1e-300) and are left to underflow.
    """
    nlat = mu.size
    P = np.zeros((L + 1, L + 1, nlat))
    s = np.sqrt(1.0 - mu * mu)
    pmm = np.full(nlat, 1.0 / np.sqrt(2.0))
    for m in range(L + 1):
        if m > 0:
            pmm = np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm
        P[m, m] = pmm
        if m + 1 <= L:
            P[m, m + 1] = np.sqrt(2.0 * m + 3.0) * mu * pmm
        for n in range(m + 2, L + 1):
            P[m, n] = (mu * P[m, n - 1] - eps(m, n - 1) * P[m, n - 2]) / eps(m, n)
    return P


def dlegendre_table(L: int, mu: np.ndarray, P_ext: np.ndarray) -> np.ndarray:
    """H[m, n, j] = (1 - mu^2) dP_n^m/dmu for n <= L, from a P table extended to L+1.

    Uses the derivative identity
    (1 - mu^2) dP_n^m/dmu = -n eps_{n+1}^m P_{n+1}^m + (n+1) eps_n^m P_{n-1}^m.
    Pinned against centred finite differences of P.
    """
    assert P_ext.shape[0] >= L + 2
    H = np.zeros((L + 1, L + 1, mu.size))
    for m in range(L + 1):
        for n in range(m, L + 1):
            h = -n * eps(m, n + 1) * P_ext[m, n + 1]
            if n - 1 >= m:
                h = h + (n + 1) * eps(m, n) * P_ext[m, n - 1]
            H[m, n] = h
    return H


class Sphere:
    """Gaussian grid + tables for truncation T_M on an nlat x nlon grid (§2.2)."""

    def __init__(self, M: int, nlat: int, nlon: int, a: float = 6371.22e3):
        assert nlon > 2 * (M + 1) and nlat >= M + 2
        self.M, self.nlat, self.nlon, self.a = M, nlat, nlon, a
        self.mu, self.w = gauss_legendre(nlat)
        self.coslat2 = 1.0 - self.mu ** 2                   # cos^2(latitude)
        self.lon = 2.0 * np.pi * np.arange(nlon) / nlon
        Pext = legendre_table(M + 1, self.mu)
        self.P = Pext[: M + 1, : M + 1]                     # [m, n, j], n <= M
        self.H = dlegendre_table(M, self.mu, Pext)          # [m, n, j], n <= M
        mm = np.arange(M + 1)
        self.m = mm[:, None] * np.ones((1, M + 1))
        self.n = np.ones((M + 1, 1)) * mm[None, :]
        self.mask = (self.n >= self.m)
        self.nn1 = self.n * (self.n + 1.0)                  # n(n+1)
        # naive DFT tables (matrices), m = 0..M
        ml = np.outer(mm, self.lon)
        c = np.where(mm == 0, 1.0, 2.0)[:, None]
        self.inv_cos = c * np.cos(ml)                       # [m, k]
        self.inv_sin = c * np.sin(ml)
        self.fwd = (np.cos(ml) - 1j * np.sin(ml)).T / nlon  # [k, m]

    # ---------------- longitude DFT -----------------
    def fourier_to_grid(self, F: np.ndarray) -> np.ndarray:
        """g[j, k] = Re F_0 + 2 Re sum_{m>=1} F_m e^{i m lambda_k}   (F[j, m])."""
        return F.real @ self.inv_cos - F.imag @ self.inv_sin

    def grid_to_fourier(self, g: np.ndarray) -> np.ndarray:
        """F[j, m] = (1/nlon) sum_k g[j, k] e^{-i m lambda_k}, m = 0..M."""
        return g @ self.fwd

    # ---------------- scalar transforms -----------------
    def sh_to_fourier(self, f: np.ndarray, table=None) -> np.ndarray:
        """F[j, m] = sum_n f[m, n] P_n^m(mu_j)  (inverse Legendre, direct sum)."""
        T = self.P if table is None else table
        return np.einsum("mnj,mn->jm", T, f)

    def sh_to_grid(self, f: np.ndarray) -> np.ndarray:
        """Inverse spherical-harmonic transform of dense coefficients f[m, n]."""
        return self.fourier_to_grid(self.sh_to_fourier(f))

    def fourier_to_sh(self, F: np.ndarray, table=None) -> np.ndarray:
        """f[m, n] = sum_j w_j P_n^m(mu_j) F[j, m]  (forward Legendre, Gauss quadrature)."""
        T = self.P if table is None else table
        return np.einsum("mnj,j,jm->mn", T, self.w, F) * self.mask

    def grid_to_sh(self, g: np.ndarray) -> np.ndarray:
        """Forward spherical-harmonic transform of a grid field g[j, k]."""
        return self.fourier_to_sh(self.grid_to_fourier(g))

    # ---------------- spectral Laplacian -----------------
    def lap(self, f):
        """nabla^2 Y_mn = -n(n+1)/a^2 Y_mn (§2.2)."""
        return -self.nn1 / self.a ** 2 * f

    def inv_lap(self, f):
        """Inverse Laplacian; the n = 0 (global mean) coefficient is set to zero."""
        out = np.zeros_like(f)
        nz = self.nn1 > 0
        out[nz] = -f[nz] * self.a ** 2 / self.nn1[nz]
        return out * self.mask

    # ---------------- vector transforms -----------------
    def uv_to_grid(self, psi: np.ndarray, chi: np.ndarray):
        """(U, V) = (u cos(lat), v cos(lat)) of the flow with streamfunction psi, velocity potential chi.

        u = (1/(a cos)) dchi/dlambda - (1/a) dpsi/dlat,  v = (1/(a cos)) dpsi/dlambda + (1/a) dchi/dlat,
        so  U = (1/a)[dchi/dlambda - (1-mu^2) dpsi/dmu],  V = (1/a)[dpsi/dlambda + (1-mu^2) dchi/dmu].
        Evaluated with the H = (1-mu^2) dP/dmu table (direct sums).
        """
        im = 1j * self.m
        Uf = (np.einsum("mnj,mn->jm", self.P, im * chi) - np.einsum("mnj,mn->jm", self.H, psi)) / self.a
        Vf = (np.einsum("mnj,mn->jm", self.P, im * psi) + np.einsum("mnj,mn->jm", self.H, chi)) / self.a
        return self.fourier_to_grid(Uf), self.fourier_to_grid(Vf)

    def div_curl_from_grid(self, A: np.ndarray, B: np.ndarray):
        """Spectral divergence and vertical curl of the vector with A = a_lon cos, B = a_lat cos.

        div a  = (1/(a(1-mu^2))) [dA/dlambda + (1-mu^2) dB/dmu]
        curl a = (1/(a(1-mu^2))) [dB/dlambda - (1-mu^2) dA/dmu]
        projected on P_n^m e^{i m lambda} with the mu-derivative moved onto
        P by integration by parts (B and A vanish at the poles):
        div_mn  = (1/a) sum_j w_j [i m A_m P_n^m - B_m H_n^m] / (1 - mu_j^2)
        curl_mn = (1/a) sum_j w_j [i m B_m P_n^m + A_m H_n^m] / (1 - mu_j^2)
        """
        Af = self.grid_to_fourier(A) / self.coslat2[:, None]
        Bf = self.grid_to_fourier(B) / self.coslat2[:, None]
        im = 1j * self.m
        PA = np.einsum("mnj,j,jm->mn", self.P, self.w, Af)
        PB = np.einsum("mnj,j,jm->mn", self.P, self.w, Bf)
        HA = np.einsum("mnj,j,jm->mn", self.H, self.w, Af)
        HB = np.einsum("mnj,j,jm->mn", self.H, self.w, Bf)
        div = (im * PA - HB) / self.a
        curl = (im * PB + HA) / self.a
        return div * self.mask, curl * self.mask

    # ---------------- packing -----------------
    def pack(self, f: np.ndarray) -> np.ndarray:
        """Dense [m, n] -> m-major triangular vector (storage layout of the library)."""
        return np.concatenate([f[m, m:] for m in range(self.M + 1)])

    def unpack(self, v: np.ndarray) -> np.ndarray:
        """m-major triangular vector -> dense [m, n] (zeros for n < m)."""
        M = self.M
        f = np.zeros((M + 1, M + 1), dtype=np.complex128)
        o = 0
        for m in range(M + 1):
            f[m, m:] = v[o: o + M + 1 - m]
            o += M + 1 - m
        return f

    def real_m0(self, f):
        """Drop the imaginary part of the m = 0 row (real fields)."""
        g = f.copy()
        g[0] = g[0].real
        return g
