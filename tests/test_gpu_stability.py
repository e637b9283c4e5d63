"""Stability-region kernel (§4 figures) against the oracle's region generator, through the C ABI."""
import numpy as np
import pytest

from oracle import stability as st

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

XI_T = 2.5e-4j
RE, IM = (-2.5, 0.5, 41), (-2.0, 2.0, 31)
NAMES = {0: "alone", 1: "parareal", 2: "mgrit", 3: "mgrit_printed"}
CASES = [
    # coarse scheme, method, xi_L, n, k, nu
    (0, 0, 0.0, 1, 0, 0),                  # serial IMEX
    (1, 0, 1e4 * XI_T, 1, 0, 0),           # serial SL-SI-SETTLS
    (1, 0, 2.5e4 * XI_T, 1, 0, 0),
    (0, 1, 0.0, 100, 5, 0),                # Parareal, IMEX coarse (paper: n = 100, cf = 2)
    (1, 1, 1e4 * XI_T, 100, 1, 0),         # Parareal, SL coarse
    (0, 1, 5e3 * XI_T, 100, 10, 0),
    (0, 2, 1e4 * XI_T, 100, 5, 2),         # two-level MGRIT, F(CF)^2 (path-count limit)
    (1, 2, 0.0, 100, 5, 1),
    (0, 3, 1e4 * XI_T, 100, 5, 3),         # Eq. 20 as printed
]


@pytest.mark.parametrize("coarse,method,xiL,n,k,nu", CASES)
def test_stability_region_matches_oracle(coarse, method, xiL, n, k, nu):
    from paper_2306_09497_gb300 import swe
    out = torch.empty((IM[2], RE[2]), dtype=torch.float64, device="cuda")
    swe.stability_region(out, coarse, method, xiL, RE, IM, n=n, k=k, cf=2, Nc=1, nu=nu, n_kappa=21)
    got = out.cpu().numpy()
    ref = st.region("imex" if coarse == 0 else "sl", NAMES[method], xiL, RE, IM, n=n, k=k, cf=2, Nc=1, nu=nu,
                    n_kappa=21)
    # relative to max(1, |A|): both sides sum the same closed forms in FP64 (the stability
    # boundary |A| = 1 is decided alike wherever the two differ by less than this)
    rel = np.abs(got - ref) / np.maximum(1.0, ref)
    assert np.max(rel) < 1e-9, np.max(rel)
    assert np.array_equal(got <= 1.0, ref <= 1.0) or np.sum((got <= 1.0) != (ref <= 1.0)) <= 2


def test_stability_region_rejects_bad_descriptors():
    from paper_2306_09497_gb300 import swe
    out = torch.empty((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(swe.SWEError):
        swe.stability_region(out, 0, 3, 0.0, (0, 1, 4), (0, 1, 4), n=10, k=40, nu=1)   # printed limit beyond n
    with pytest.raises(swe.SWEError):
        swe.stability_region(out, 5, 0, 0.0, (0, 1, 4), (0, 1, 4))
