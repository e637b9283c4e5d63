"""Shallow-water operators and time steppers (oracle; test use only).

State U = (Phi', xi, delta): geopotential perturbation, vorticity, divergence
(§2.1, Eq. 1), each a dense complex array [m, n].  The mean geopotential
Phi_bar is held separately.

Readings of the paper used here (where it is silent or garbled):

* Coriolis parameter on the sphere f = 2 Omega mu (the paper spells out only
  the f-plane value 2 Omega, §4.1).
* The explicit RK2 stage of Eq. 5 is read as Heun's method,
  U** = U* + (Ubar + Ubarbar)/2 (as printed, U** is the increment only).
* Nonlinear geopotential tendency -V.grad(Phi) - Phi' delta (N_A + N_R of
  Eq. 1) is evaluated in the analytically identical flux form -div(Phi' V).
* The implicit Crank-Nicolson problem of Eq. 4 keeps all of L = L_G + L_C
  implicit (Coriolis included), solved exactly per zonal wavenumber m.
* SL-SI-SETTLS (Eqs. 6-7) interpolates the three components of
  [U + (dt/2) L U + (dt/2)(2 N_R - N_R^{n-1})] to the departure points, two
  SETTLS iterations from x_d = x_a, trajectories in 3-D Cartesian
  coordinates, bicubic Lagrange interpolation with two halo rows across each
  pole; the first step of a chain, and every step of the one-step variant,
  replaces the t_{n-1} data by the t_n data (§3.2.4).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.linalg import solve_banded

from .sphere import Sphere, eps


@dataclass
class Physics:
    a: float = 6371.22e3      # m, §4.1
    omega: float = 7.292e-5   # 1/s, §4.1
    g: float = 9.80616        # m/s^2, §5.1
    phibar: float = 1.0e5     # m^2/s^2, §4.1


class SWE:
    """Operators of Eq. 1 on a given Sphere (dense spectral arrays).

    nphi_form selects the geopotential tendency of N: "flux" evaluates -div(Phi' V) (the
    default, mass-conserving form), "advective" evaluates Eq. 1 as written,
    -V.grad(Phi') - Phi' delta, with grad Phi' synthesised from its spectral derivatives.
    """

    def __init__(self, sph: Sphere, phys: Physics = Physics(), nphi_form: str = "flux"):
        assert nphi_form in ("flux", "advective")
        self.s, self.p = sph, phys
        self.nphi_form = nphi_form
        M = sph.M
        m, n = sph.m, sph.n
        e_n = eps(m, n)              # eps_n^m
        e_n1 = eps(m, n + 1)         # eps_{n+1}^m
        nz = n > 0
        # coefficient of the (n-1) neighbour, the (n+1) neighbour and the
        # diagonal i m term in the spectral form of L_C (see coriolis_spectral)
        self.cp = np.where(nz, (n + 1.0) / np.maximum(n, 1.0) * e_n, 0.0)
        self.cq = np.where(nz, n / (n + 1.0) * e_n1, 0.0)
        self.cr = np.where(nz, m / np.maximum(n * (n + 1.0), 1.0), 0.0)
        self.e_n, self.e_n1 = e_n, e_n1
        self.M = M
        self._band_cache = {}

    # ------------------------------------------------------------------
    # helpers on dense [m, n] arrays
    @staticmethod
    def _down(x):
        """x_{n-1} placed at index n (zero where n-1 is outside)."""
        y = np.zeros_like(x)
        y[:, 1:] = x[:, :-1]
        return y

    @staticmethod
    def _up(x):
        """x_{n+1} placed at index n (zero beyond the truncation)."""
        y = np.zeros_like(x)
        y[:, :-1] = x[:, 1:]
        return y

    def mu_times(self, x):
        """Spectral coefficients of mu * x:  eps_n^m x_{n-1} + eps_{n+1}^m x_{n+1} (truncated)."""
        return (self.e_n * self._down(x) + self.e_n1 * self._up(x)) * self.s.mask

    # ------------------------------------------------------------------
    # linear operator L = L_G + L_C of Eq. 1
    def coriolis_grid(self, U):
        """L_C U = (0, -div(f V), curl(f V)) with f = 2 Omega mu, products on the grid."""
        s = self.s
        _, xi, de = U
        Ug, Vg = s.uv_to_grid(s.inv_lap(xi), s.inv_lap(de))
        f = 2.0 * self.p.omega * s.mu[:, None]
        div, curl = s.div_curl_from_grid(f * Ug, f * Vg)
        return np.zeros_like(xi), -div, curl

    def coriolis_spectral(self, U):
        """L_C U in spectral space, exact for the truncated product.

        Product rule: -div(f V) = -f delta - (2 Omega / a) V_cos and
        curl(f V) = f xi - (2 Omega / a) U_cos (U_cos = u cos, V_cos = v cos);
        with mu-multiplication and the (1-mu^2) d/dmu recurrence this gives
        (L_C U)_xi,n    = -2 Omega [cp_n delta_{n-1} + cq_n delta_{n+1} - i cr_n xi_n]
        (L_C U)_delta,n =  2 Omega [cp_n xi_{n-1}    + cq_n xi_{n+1}    + i cr_n delta_n]
        cp_n = (n+1)/n eps_n^m, cq_n = n/(n+1) eps_{n+1}^m, cr_n = m/(n(n+1)).
        Pinned against coriolis_grid.
        """
        _, xi, de = U
        # xi_00 and delta_00 vanish for every flow (zero-mean vorticity and
        # divergence); they are ignored here, as the grid form ignores them.
        xi = xi.copy()
        de = de.copy()
        xi[0, 0] = 0.0
        de[0, 0] = 0.0
        w2 = 2.0 * self.p.omega
        Lxi = -w2 * (self.cp * self._down(de) + self.cq * self._up(de) - 1j * self.cr * xi)
        Lde = w2 * (self.cp * self._down(xi) + self.cq * self._up(xi) + 1j * self.cr * de)
        mk = self.s.mask
        return np.zeros_like(xi), Lxi * mk, Lde * mk

    def linear(self, U):
        """L U = L_G U + L_C U, L_G U = (-Phi_bar delta, 0, -lap Phi') (Eq. 1)."""
        Phi, xi, de = U
        _, cx, cd = self.coriolis_spectral(U)
        s = self.s
        return (-self.p.phibar * de, cx, -s.lap(Phi) + cd)

    def _band_matrices(self, alpha):
        """Banded (I - alpha L_m) for every m, unknowns ordered (Phi_n, xi_n, delta_n), n = m..M."""
        key = float(alpha)
        if key in self._band_cache:
            return self._band_cache[key]
        s, p = self.s, self.p
        M = self.M
        out = []
        for m in range(M + 1):
            K = M + 1 - m
            A = np.eye(3 * K, dtype=np.complex128)
            for k in range(K):
                n = m + k
                iP, iX, iD = 3 * k, 3 * k + 1, 3 * k + 2
                # row Phi:  -Phi_bar delta
                A[iP, iD] -= alpha * (-p.phibar)
                # row xi
                A[iX, iX] -= alpha * (2.0 * p.omega * 1j * self.cr[m, n])
                if k - 1 >= 0:
                    A[iX, 3 * (k - 1) + 2] -= alpha * (-2.0 * p.omega * self.cp[m, n])
                if k + 1 < K:
                    A[iX, 3 * (k + 1) + 2] -= alpha * (-2.0 * p.omega * self.cq[m, n])
                # row delta
                A[iD, iP] -= alpha * (n * (n + 1.0) / p.a ** 2)
                A[iD, iD] -= alpha * (2.0 * p.omega * 1j * self.cr[m, n])
                if k - 1 >= 0:
                    A[iD, 3 * (k - 1) + 1] -= alpha * (2.0 * p.omega * self.cp[m, n])
                if k + 1 < K:
                    A[iD, 3 * (k + 1) + 1] -= alpha * (2.0 * p.omega * self.cq[m, n])
            l = u = 4
            ab = np.zeros((l + u + 1, 3 * K), dtype=np.complex128)
            for j in range(3 * K):
                for i in range(max(0, j - u), min(3 * K, j + l + 1)):
                    ab[u + i - j, j] = A[i, j]
            out.append(ab)
        self._band_cache[key] = out
        return out

    def implicit_solve(self, R, alpha):
        """Solve (I - alpha L) X = R exactly, one banded system per m.

        The global means of vorticity and divergence (coefficient (0, 0) of xi and
        delta) vanish for every velocity field on the sphere, so they are not
        unknowns: a right-hand side built by interpolation (Eq. 7) can carry a small
        spurious mean, which is projected out here.
        """
        R = tuple(x.copy() for x in R)
        R[1][0, 0] = 0.0
        R[2][0, 0] = 0.0
        bands = self._band_matrices(alpha)
        M = self.M
        X = [np.zeros_like(R[0]) for _ in range(3)]
        for m in range(M + 1):
            rhs = np.stack([R[0][m, m:], R[1][m, m:], R[2][m, m:]], axis=1).reshape(-1)
            x = solve_banded((4, 4), bands[m], rhs)
            x = x.reshape(-1, 3)
            for f in range(3):
                X[f][m, m:] = x[:, f]
        return tuple(X)

    def cn_step(self, U, alpha):
        """Crank-Nicolson: U* - alpha L U* = U + alpha L U  (Eq. 4 with alpha = dt/4)."""
        LU = self.linear(U)
        R = tuple(U[f] + alpha * LU[f] for f in range(3))
        return self.implicit_solve(R, alpha)

    # ------------------------------------------------------------------
    # viscosity, App. A: backward Euler of d psi/dt = -nu (n(n+1)/a^2)^{q/2} psi
    def viscosity(self, U, dt, nu, q):
        if nu == 0.0:
            return U
        fac = 1.0 / (1.0 + dt * nu * (self.s.nn1 / self.p.a ** 2) ** (q // 2))
        return tuple(x * fac for x in U)

    # ------------------------------------------------------------------
    # nonlinear terms N = N_A + N_R (Eq. 1), pseudospectral
    def nonlinear(self, U):
        s = self.s
        Phi, xi, de = U
        Ug, Vg = s.uv_to_grid(s.inv_lap(xi), s.inv_lap(de))
        Pg = s.sh_to_grid(Phi)
        Xg = s.sh_to_grid(xi)
        divX, curlX = s.div_curl_from_grid(Xg * Ug, Xg * Vg)
        ke = (Ug * Ug + Vg * Vg) / (2.0 * s.coslat2[:, None])
        KE = s.grid_to_sh(ke)
        if self.nphi_form == "flux":
            divP, _ = s.div_curl_from_grid(Pg * Ug, Pg * Vg)
            NPhi = -divP
        else:
            NPhi = self.nphi_advective(U, Ug, Vg, Pg)
        return (NPhi, -divX, curlX - s.lap(KE))

    def nphi_advective(self, U, Ug=None, Vg=None, Pg=None):
        """Geopotential tendency in the advective form of Eq. 1, -V.grad(Phi') - Phi' delta.

        With U = u cos(lat), V = v cos(lat):
        V.grad(Phi') = [U dPhi'/dlambda + V (1 - mu^2) dPhi'/dmu] / (a (1 - mu^2)),
        the derivatives synthesised exactly from the spectral coefficients (i m P and the
        H = (1 - mu^2) dP/dmu table), the products and the forward projection on the grid.
        """
        s = self.s
        Phi, xi, de = U
        if Ug is None:
            Ug, Vg = s.uv_to_grid(s.inv_lap(xi), s.inv_lap(de))
            Pg = s.sh_to_grid(Phi)
        Plam = s.fourier_to_grid(np.einsum("mnj,mn->jm", s.P, 1j * s.m * Phi))
        Pmu = s.fourier_to_grid(np.einsum("mnj,mn->jm", s.H, Phi))
        Dg = s.sh_to_grid(de)
        adv = (Ug * Plam + Vg * Pmu) / (self.p.a * s.coslat2[:, None])
        return s.real_m0(s.grid_to_sh(-adv - Pg * Dg))

    def nonlinear_R_grid(self, U):
        """N_R of Eq. 1 on the grid: -Phi' delta (geopotential component only)."""
        s = self.s
        return -s.sh_to_grid(U[0]) * s.sh_to_grid(U[2])

    # ------------------------------------------------------------------
    def imex_step(self, U, dt, nu=0.0, q=2):
        """One IMEX Strang step, Eqs. 3-5, then backward-Euler viscosity (§2.3)."""
        alpha = dt / 4.0
        Us = self.cn_step(U, alpha)
        N1 = self.nonlinear(Us)
        Ub = tuple(dt * x for x in N1)
        N2 = self.nonlinear(tuple(Us[f] + Ub[f] for f in range(3)))
        Ubb = tuple(dt * x for x in N2)
        Uss = tuple(Us[f] + 0.5 * (Ub[f] + Ubb[f]) for f in range(3))
        U1 = self.cn_step(Uss, alpha)
        return self.viscosity(U1, dt, nu, q)

    # ------------------------------------------------------------------
    def balanced_geopotential(self, xi):
        """Phi' with d(delta)/dt = 0 for the non-divergent flow with vorticity xi.

        From the divergence row of Eq. 1 with delta = 0:
        lap Phi' = [L_C U]_delta + [N_A U]_delta, i.e.
        Phi'_mn = -(a^2/(n(n+1))) ([L_C U]_delta + [N U]_delta)_mn,  Phi'_00 = 0.
        """
        z = np.zeros_like(xi)
        U = (z, xi, z)
        _, _, cd = self.coriolis_spectral(U)
        _, _, nd = self.nonlinear(U)
        return self.s.inv_lap(cd + nd)

    # ------------------------------------------------------------------
    # semi-Lagrangian pieces (Eqs. 6-7)
    def _cart_velocity(self, U):
        """Cartesian velocity (m/s) on the grid from the spectral state."""
        s = self.s
        Ug, Vg = s.uv_to_grid(s.inv_lap(U[1]), s.inv_lap(U[2]))
        cosl = np.sqrt(s.coslat2)[:, None]
        u, v = Ug / cosl, Vg / cosl
        lam = s.lon[None, :]
        sinl = s.mu[:, None]
        vx = -u * np.sin(lam) - v * sinl * np.cos(lam)
        vy = u * np.cos(lam) - v * sinl * np.sin(lam)
        vz = v * cosl * np.ones_like(lam)
        return vx, vy, vz

    def _interp(self, fields, lat_d, lon_d):
        """Bicubic Lagrange interpolation at (lat_d, lon_d) with 2 halo rows across each pole."""
        s = self.s
        nlat, nlon = s.nlat, s.nlon
        th = np.arcsin(s.mu)
        thx = np.concatenate([[np.pi - th[1], np.pi - th[0]], th,
                              [-np.pi - th[-1], -np.pi - th[-2]]])
        rows = np.concatenate([[1, 0], np.arange(nlat), [nlat - 1, nlat - 2]])
        shift = np.concatenate([[nlon // 2, nlon // 2], np.zeros(nlat, int), [nlon // 2, nlon // 2]])
        # bracket: thx[i] >= lat_d > thx[i+1] (thx descending)
        i = np.searchsorted(-thx, -lat_d, side="right") - 1
        i = np.clip(i, 1, nlat + 1)
        y = np.stack([thx[i - 1], thx[i], thx[i + 1], thx[i + 2]], axis=-1)
        wl = np.ones_like(y)
        for k in range(4):
            for l2 in range(4):
                if l2 != k:
                    wl[..., k] *= (lat_d - y[..., l2]) / (y[..., k] - y[..., l2])
        dl = 2.0 * np.pi / nlon
        x = np.mod(lon_d, 2.0 * np.pi) / dl
        i0 = np.floor(x).astype(int)
        t = x - i0
        wx = np.stack([-t * (t - 1) * (t - 2) / 6.0, (t + 1) * (t - 1) * (t - 2) / 2.0,
                       -(t + 1) * t * (t - 2) / 2.0, (t + 1) * t * (t - 1) / 6.0], axis=-1)
        outs = []
        for F in fields:
            acc = np.zeros(lat_d.shape)
            for r in range(4):
                er = i - 1 + r
                row = rows[er]
                sh = shift[er]
                for c in range(4):
                    col = np.mod(i0 - 1 + c + sh, nlon)
                    acc += wl[..., r] * wx[..., c] * F[row, col]
            outs.append(acc)
        return outs

    def departure_points(self, vel_n, vel_nm1, dt, iters=2):
        """SETTLS trajectories, Eq. 6, in 3-D Cartesian form projected on the sphere."""
        s = self.s
        lat = np.arcsin(s.mu)[:, None] * np.ones((1, s.nlon))
        lon = s.lon[None, :] * np.ones((s.nlat, 1))
        xa = np.stack([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)])
        va = np.stack(vel_n)
        xd = xa.copy()
        latd, lond = lat.copy(), lon.copy()
        for _ in range(iters):
            vn = np.stack(self._interp(vel_n, latd, lond))
            vm = np.stack(self._interp(vel_nm1, latd, lond))
            mid = 2.0 * vn - vm + va
            xd = xa - (dt / (2.0 * self.p.a)) * mid
            xd = xd / np.sqrt(np.sum(xd * xd, axis=0))
            latd = np.arcsin(np.clip(xd[2], -1.0, 1.0))
            lond = np.mod(np.arctan2(xd[1], xd[0]), 2.0 * np.pi)
        return latd, lond

    def sl_si_settls_step(self, U, U_prev, dt, nu=0.0, q=2):
        """One SL-SI-SETTLS step, Eq. 7; ``U_prev`` None selects the one-step variant.

        (I - dt/2 L) U^{n+1} = [U^n + dt/2 L U^n + dt/2 (2 N_R^n - N_R^{n-1})]_* + dt/2 N_R^n
        followed by backward-Euler viscosity.
        """
        s = self.s
        if U_prev is None:
            U_prev = U
        vel_n = self._cart_velocity(U)
        vel_m = self._cart_velocity(U_prev)
        latd, lond = self.departure_points(vel_n, vel_m, dt)
        LU = self.linear(U)
        nr_n = self.nonlinear_R_grid(U)
        nr_m = self.nonlinear_R_grid(U_prev)
        X = [s.sh_to_grid(U[f] + 0.5 * dt * LU[f]) for f in range(3)]
        X[0] = X[0] + 0.5 * dt * (2.0 * nr_n - nr_m)
        Xd = self._interp(X, latd, lond)
        Xd[0] = Xd[0] + 0.5 * dt * nr_n
        R = tuple(s.real_m0(s.grid_to_sh(Xd[f])) for f in range(3))
        U1 = self.implicit_solve(R, 0.5 * dt)
        return self.viscosity(U1, dt, nu, q)


# ----------------------------------------------------------------------
# convenience: packed <-> dense state conversion
def to_dense(sph: Sphere, Upacked):
    return tuple(sph.unpack(Upacked[f]) for f in range(3))


def to_packed(sph: Sphere, U):
    return np.stack([sph.pack(U[f]) for f in range(3)])
