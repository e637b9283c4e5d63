"""Scalar linear test ODE of §4 (Eqs. 10-20): schemes and closed forms (oracle; test use only).

u' = lambda_L u + lambda_N u, xi_L = lambda_L dt, xi_N = lambda_N dt.
"""
from __future__ import annotations

from math import comb

import numpy as np


# ---------------- IMEX (§4.1.1) ----------------
def imex_step(u, xiL, xiN):
    """One IMEX Strang step of Eqs. 3-5 on the scalar ODE (Heun reading of Eq. 5)."""
    cn = lambda x: x * (1.0 + xiL / 4.0) / (1.0 - xiL / 4.0)   # u* - (xiL/4) u* = u + (xiL/4) u
    us = cn(u)
    ub = xiN * us
    ubb = xiN * (us + ub)
    uss = us + 0.5 * (ub + ubb)
    return cn(uss)


def A_imex_implicit(xiL):
    """A_IMEX-I = (4 + xi_L) / (4 - xi_L)  (§4.1.1)."""
    return (4.0 + xiL) / (4.0 - xiL)


def A_imex_explicit_printed(xiN):
    """A_IMEX-E as printed in §4.1.1: xi_N (2 + xi_N) / 2 (the increment of the RK2 stage)."""
    return xiN * (2.0 + xiN) / 2.0


def A_imex(xiL, xiN):
    """IMEX amplification under the Heun reading: A_I^2 (1 + xi_N (2 + xi_N)/2)."""
    return A_imex_implicit(xiL) ** 2 * (1.0 + A_imex_explicit_printed(xiN))


# ---------------- SL-SI-SETTLS (§4.1.2) ----------------
def sl_step(u_n, u_nm1, xiL, xiN, kappa_s):
    """Scalar SL-SI-SETTLS (Eq. 7) for the mode e^{i kappa x}: the departure-point
    value of a mode equals its arrival value times e^{-i kappa s}."""
    e = np.exp(-1j * kappa_s)
    rhs = e * ((1.0 + xiL / 2.0) * u_n + 0.5 * xiN * (2.0 * u_n - u_nm1)) + 0.5 * xiN * u_n
    return rhs / (1.0 - xiL / 2.0)


def sl_roots(xiL, xiN, kappa_s):
    """Roots of Eq. 13: A^2 (1 - xiL/2) - A (e (1 + xiL/2 + xiN) + xiN/2) + (xiN/2) e = 0."""
    e = np.exp(-1j * kappa_s)
    return np.roots([1.0 - xiL / 2.0, -(e * (1.0 + xiL / 2.0 + xiN) + xiN / 2.0), 0.5 * xiN * e])


# ---------------- Parareal (§4.2) ----------------
def A_parareal(n, k, R, S):
    """Eq. 17 with R = A_c^{N_c}, S = A_f^{N_f} - A_c^{N_c}."""
    return sum(comb(n, i) * S ** i * R ** (n - i) for i in range(0, k + 1))


# ---------------- MGRIT two-level (§4.3) ----------------
def A_mgrit_printed(n, k, nu, F, G):
    """Eq. 20 as printed: sum over i <= floor(k/(nu+1)) of
    C(n - i nu, i) (F^nu (F - G))^i G^(n - i(nu+1)), with F = A_f^{N_f}, G = A_c^{N_c}."""
    S = F ** nu * (F - G)
    return sum(comb(n - i * nu, i) * S ** i * G ** (n - i * (nu + 1))
               for i in range(0, k // (nu + 1) + 1))


def A_mgrit_pathcount(n, k, nu, F, G):
    """Path count of the recurrence u^k_n = G u^k_{n-1} + S u^{k-1}_{n-nu-1} (Eq. 19)
    with u^0_n = G^n u_0, u^k_0 = u_0 and zero for negative indices: each S-step
    costs one iteration, so i runs to min(k, floor(n/(nu+1)))."""
    S = F ** nu * (F - G)
    return sum(comb(n - i * nu, i) * S ** i * G ** (n - i * (nu + 1))
               for i in range(0, min(k, n // (nu + 1)) + 1))


def recurrence_eq19(n, k, nu, F, G):
    """Brute-force evaluation of the recurrence of Eq. 19 (boundary as in A_mgrit_pathcount)."""
    S = F ** nu * (F - G)
    u = np.zeros((k + 1, n + 1), dtype=complex)
    u[:, 0] = 1.0
    for j in range(1, n + 1):
        u[0, j] = G * u[0, j - 1]
    for kk in range(1, k + 1):
        for j in range(1, n + 1):
            u[kk, j] = G * u[kk, j - 1] + (S * u[kk - 1, j - nu - 1] if j - nu - 1 >= 0 else 0.0)
    return u[k, n]


# ---------------- stability regions on a grid of xi_N (§4.1-4.3 figures) ----------------
def region(coarse, method, xiL, re, im, n=100, k=0, cf=2, Nc=1, nu=0, n_kappa=21):
    """|A| on the grid xi_N = re[0] + i dre ... (re = (re0, re1, nre), im likewise), [nim][nre].

    coarse: "imex" or "sl"; method: "alone" (|A_c^{n N_c}|), "parareal" (Eq. 17),
    "mgrit" (Eq. 20 with the path-count limit, reading A14) or "mgrit_printed" (Eq. 20 as
    printed).  xi is relative to the coarse step Delta t_c; the fine scheme is IMEX with
    Delta t_c / cf and N_f = cf N_c steps per slice.  For SL-SI-SETTLS every root of Eq. 13 at
    every kappa s = 2 pi q / (n_kappa - 1) is used as the coarse factor and the largest |A| is
    kept (the region is the intersection over roots and kappa s).
    """
    re0, re1, nre = re
    im0, im1, nim = im
    dre = (re1 - re0) / (nre - 1) if nre > 1 else 0.0
    dim = (im1 - im0) / (nim - 1) if nim > 1 else 0.0
    out = np.zeros((nim, nre))
    for iy in range(nim):
        for ix in range(nre):
            xiN = complex(re0 + ix * dre, im0 + iy * dim)
            Af = A_imex(xiL / cf, xiN / cf)
            if coarse == "imex":
                coarse_factors = [A_imex(xiL, xiN)]
            else:
                coarse_factors = []
                for q in range(n_kappa):
                    ks = 2.0 * np.pi * q / (n_kappa - 1) if n_kappa > 1 else 0.0
                    coarse_factors.extend(sl_roots(xiL, xiN, ks))
            best = 0.0
            for Ac in coarse_factors:
                R = Ac ** Nc
                F = Af ** (cf * Nc)
                if method == "alone":
                    a = R ** n
                elif method == "parareal":
                    a = A_parareal(n, min(k, n), R, F - R)
                elif method == "mgrit":
                    a = A_mgrit_pathcount(n, k, nu, F, R)
                else:
                    a = A_mgrit_printed(n, k, nu, F, R)
                best = max(best, abs(a))
            out[iy, ix] = best
    return out
