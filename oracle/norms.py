"""Error norms of §5 (oracle; test use only)."""
from __future__ import annotations

import numpy as np


def spectral_max(psi_dense: np.ndarray, R: int) -> float:
    """||psi||_{inf,R}: max |psi_mn| over 0 <= m <= R, m <= n <= R (Eq. 21)."""
    return float(np.max(np.abs(psi_dense[: R + 1, : R + 1])))


def spectral_error(psi, ref, R: int) -> float:
    """E_{psi,R} = ||psi - ref||_{inf,R} / ||ref||_{inf,R} (Eq. 21)."""
    return spectral_max(psi - ref, R) / spectral_max(ref, R)


def l2_error(g, gref) -> float:
    """Relative L2 error on the grid: sqrt(mean (g-gref)^2) / sqrt(mean gref^2) (§5, unweighted)."""
    return float(np.sqrt(np.mean((g - gref) ** 2)) / np.sqrt(np.mean(gref ** 2)))


def _cm(psi_dense):
    """Weights c_m (1 for m = 0, 2 for m >= 1) of the m >= 0 storage, as a column."""
    c = np.full((psi_dense.shape[0], 1), 2.0)
    c[0] = 1.0
    return c


def _real_m0(x):
    x = np.array(x, dtype=np.complex128)
    x[0] = x[0].real
    return x


def parseval_l2_error(psi, ref) -> float:
    """Area-weighted relative L2 error over the sphere from spectral coefficients.

    With the orthonormal basis the area mean of f^2 is (1/2) sum_m c_m |f_mn|^2 (c_0 = 1,
    c_m = 2 for the conjugate pair), so the ratio of the two sums is the ratio of the
    area-weighted mean squares of the grid fields (§5 L2 error, reading A8: weighted by
    area instead of an unweighted grid mean).  The imaginary part of m = 0 is ignored.
    Pinned against Gauss quadrature of the inverse-transformed fields.
    """
    d = _real_m0(psi) - _real_m0(ref)
    r = _real_m0(ref)
    c = _cm(psi)
    return float(np.sqrt(np.sum(c * np.abs(d) ** 2) / np.sum(c * np.abs(r) ** 2)))


def ke_spectrum(xi, delta, a: float) -> np.ndarray:
    """Kinetic-energy spectrum of §5.1, E(n) = a^2 / (4 n (n+1)) sum_{m=-n}^{n} (|xi_mn|^2 + |delta_mn|^2).

    Dense [m, n] arrays (m >= 0); the m < 0 coefficients are the complex conjugates, so the
    sum over m = -n..n is sum_{m>=0} c_m |.|^2.  Returns E[0..M] with E[0] = 0.  Pinned by
    the solid-body closed form E(1) = u0^2 / 3 and by sum_n E(n) = area mean of |V|^2 / 2
    (oversampled quadrature of the grid wind).
    """
    x, d = _real_m0(xi), _real_m0(delta)
    c = _cm(xi)
    s = np.sum(c * (np.abs(x) ** 2 + np.abs(d) ** 2), axis=0)
    M = xi.shape[1] - 1
    n = np.arange(M + 1, dtype=np.float64)
    E = np.zeros(M + 1)
    E[1:] = a * a / (4.0 * n[1:] * (n[1:] + 1.0)) * s[1:]
    return E
