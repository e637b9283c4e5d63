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
