"""Pins of the oracle's stability-region generator (§4 figures): identities that the
stability functions must satisfy at every grid point."""
import numpy as np
import pytest

from oracle import stability as st

XI_T = 2.5e-4j
GRID = dict(re=(-2.0, 0.5, 11), im=(-2.0, 2.0, 9))


@pytest.mark.parametrize("coarse", ["imex", "sl"])
@pytest.mark.parametrize("xiL", [0.0, 1e4 * XI_T])
def test_parareal_at_k_equal_n_is_the_fine_scheme(coarse, xiL):
    """Binomial theorem: sum_{i<=n} C(n,i) (F - R)^i R^{n-i} = F^n, whatever the coarse factor."""
    n, cf = 12, 2
    a = st.region(coarse, "parareal", xiL, n=n, k=n, cf=cf, n_kappa=5, **GRID)
    re0, re1, nre = GRID["re"]
    im0, im1, nim = GRID["im"]
    for iy in range(nim):
        for ix in range(nre):
            xiN = complex(re0 + ix * (re1 - re0) / (nre - 1), im0 + iy * (im1 - im0) / (nim - 1))
            F = st.A_imex(xiL / cf, xiN / cf) ** cf
            f = abs(F ** n)
            # rounding bound of the binomial sum: its terms add up to at most (|R| + |F - R|)^n
            if coarse == "imex":
                Rs = [st.A_imex(xiL, xiN)]
            else:
                Rs = [r for q in range(5) for r in st.sl_roots(xiL, xiN, 2.0 * np.pi * q / 4)]
            bound = max((abs(R) + abs(F - R)) ** n for R in Rs)
            assert abs(a[iy, ix] - f) <= 1e-13 * max(1.0, bound), (ix, iy, a[iy, ix], f, bound)


@pytest.mark.parametrize("coarse", ["imex", "sl"])
def test_mgrit_nu0_region_equals_parareal(coarse):
    a = st.region(coarse, "mgrit", 1e4 * XI_T, n=20, k=5, nu=0, n_kappa=5, **GRID)
    b = st.region(coarse, "parareal", 1e4 * XI_T, n=20, k=5, n_kappa=5, **GRID)
    assert np.max(np.abs(a - b) / np.maximum(1.0, b)) < 1e-12


def test_imex_region_independent_of_imaginary_xiL():
    """|(4 + xi_L)/(4 - xi_L)| = 1 on the imaginary axis, so the serial IMEX region does not
    depend on xi_L there (§4.1.1)."""
    a = st.region("imex", "alone", 0.0, n=1, **GRID)
    b = st.region("imex", "alone", 2.5e4 * XI_T, n=1, **GRID)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(a)


def test_parareal_k0_is_the_coarse_scheme_over_n_slices():
    a = st.region("sl", "parareal", 5e3 * XI_T, n=10, k=0, n_kappa=7, **GRID)
    b = st.region("sl", "alone", 5e3 * XI_T, n=10, n_kappa=7, **GRID)
    assert np.max(np.abs(a - b) / np.maximum(1.0, b)) < 1e-12


def test_sl_region_from_roots_decides_growth_of_the_recurrence():
    """Where every root of Eq. 13 (all kappa s) has modulus below one, iterating the two-step
    scheme (Eq. 7) on the scalar mode decays; where the largest exceeds one, it grows for some
    kappa s."""
    xiL = 1e4 * XI_T
    re, im = (-0.4, 0.2, 7), (-0.4, 0.4, 9)
    a = st.region("sl", "alone", xiL, n=1, n_kappa=21, re=re, im=im)
    assert np.any(a < 0.98) and np.any(a > 1.02)
    for iy in range(im[2]):
        for ix in range(re[2]):
            if 0.98 <= a[iy, ix] <= 1.02:
                continue
            xiN = complex(re[0] + ix * (re[1] - re[0]) / (re[2] - 1), im[0] + iy * (im[1] - im[0]) / (im[2] - 1))
            peak = 0.0
            for ks in np.linspace(0.0, 2.0 * np.pi, 21):
                u = [1.0 + 0j, 1.0 + 0j]
                for _ in range(600):
                    u.append(st.sl_step(u[-1], u[-2], xiL, xiN, ks))
                peak = max(peak, abs(u[-1]))
            assert (peak < 1e-2) if a[iy, ix] < 0.98 else (peak > 1.0), (xiN, a[iy, ix], peak)
