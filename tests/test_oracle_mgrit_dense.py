"""Pin of the oracle's multilevel MGRIT (§3.2) by explicit space-time linear algebra.

For a linear one-step propagator the level-l problem of MGRIT is the block
lower-bidiagonal system A_l u = g_l (§3.2.1): u_0 = g_0 and
u_j - Phi_l u_{j-1} = g_j for j = 1..N_l.  Here every step of the full
approximation scheme (§3.2.2) is written as a dense matrix operation on that
system, independently of the oracle's time-stepping loops:

1. F(CF)^nu relaxation: F-relaxation solves the F-point rows exactly,
   A_FF u_F = g_F - A_FC u_C; C-relaxation solves the C-point rows,
   A_CC u_C = g_C - A_CF u_F.
2. Restriction at C-points: v = R u_C (R = injection in time, truncation in
   space), coarse right-hand side g_c = R (g - A_l u)_C + A_{l+1} v.
3. Coarse-grid equation A_{l+1} u_c = g_c: a dense solve on the coarsest
   level, a recursive cycle otherwise.
4. Error approximation e = u_c - v.
5. Correction u_C += P e (P = zero padding in space), then F-relaxation.

The recursion is F-cycle followed by one V-cycle per level (§3.2.3, with the
reading F(l) = relax; restrict; F(l+1); V(l+1); correct).  The initial guess
is the serial coarsest-level solution injected upwards with F-relaxation.
The propagators are random complex matrices (different per level, and of
smaller dimension on spatially coarsened levels) so that a transposed
operand, a dropped residual term or a missing post V-cycle changes the
iterates.
"""
import numpy as np
import pytest

from oracle import pint


class DenseMGRIT:
    def __init__(self, Phis, N0, cf, nu, Rs, Ps):
        self.L = len(Phis)
        self.Phi, self.cf, self.nu = Phis, cf, nu
        self.N = [N0 // cf ** l for l in range(self.L)]
        self.d = [P.shape[0] for P in Phis]
        self.R, self.P = Rs, Ps        # R[l]: d_{l+1} x d_l, P[l]: d_l x d_{l+1}
        self.A = [self._system(l) for l in range(self.L)]

    def _system(self, l):
        N, d = self.N[l], self.d[l]
        A = np.eye((N + 1) * d, dtype=complex)
        for j in range(1, N + 1):
            A[j * d:(j + 1) * d, (j - 1) * d:j * d] = -self.Phi[l]
        return A

    def _idx(self, l, points):
        d = self.d[l]
        return np.concatenate([np.arange(p * d, (p + 1) * d) for p in points])

    def _sets(self, l):
        pts = np.arange(self.N[l] + 1)
        C = pts[pts % self.cf == 0]
        F = pts[pts % self.cf != 0]
        return self._idx(l, F), self._idx(l, C)

    def f_relax(self, l, u, g):
        F, C = self._sets(l)
        A = self.A[l]
        u = u.copy()
        u[F] = np.linalg.solve(A[np.ix_(F, F)], g[F] - A[np.ix_(F, C)] @ u[C])
        return u

    def c_relax(self, l, u, g):
        F, C = self._sets(l)
        A = self.A[l]
        u = u.copy()
        u[C] = np.linalg.solve(A[np.ix_(C, C)], g[C] - A[np.ix_(C, F)] @ u[F])
        return u

    def relax(self, l, u, g):
        u = self.f_relax(l, u, g)
        for _ in range(self.nu):
            u = self.c_relax(l, u, g)
            u = self.f_relax(l, u, g)
        return u

    def _restrict_vec(self, l, x):
        """Injection at C-points plus spatial restriction: level-l vector -> level-(l+1) vector."""
        d = self.d[l]
        C = np.arange(0, self.N[l] + 1, self.cf)
        return np.concatenate([self.R[l] @ x[c * d:(c + 1) * d] for c in C])

    def _prolong_add(self, l, u, e):
        d, dc = self.d[l], self.d[l + 1]
        u = u.copy()
        for i, c in enumerate(range(0, self.N[l] + 1, self.cf)):
            u[c * d:(c + 1) * d] += self.P[l] @ e[i * dc:(i + 1) * dc]
        return u

    def two_grid(self, l, u, g, coarse):
        """Steps 1-5 of §3.2.2 between levels l and l+1; coarse(l+1, u_c, g_c) solves step 3."""
        u = self.relax(l, u, g)
        v = self._restrict_vec(l, u)
        r = g - self.A[l] @ u
        gc = self._restrict_vec(l, r) + self.A[l + 1] @ v
        uc = coarse(l + 1, v.copy(), gc)
        u = self._prolong_add(l, u, uc - v)
        return self.f_relax(l, u, g)

    def solve(self, l, u, g):
        return np.linalg.solve(self.A[l], g)

    def v_cycle(self, l, u, g):
        if l == self.L - 1:
            return self.solve(l, u, g)
        return self.two_grid(l, u, g, self.v_cycle)

    def f_cycle(self, l, u, g):
        if l == self.L - 1:
            return self.solve(l, u, g)

        def coarse(lc, uc, gc):
            if lc == self.L - 1:
                return self.solve(lc, uc, gc)
            uc = self.f_cycle(lc, uc, gc)
            return self.v_cycle(lc, uc, gc)
        return self.two_grid(l, u, g, coarse)

    def initial(self, u0):
        L = self.L
        x = [u0]
        for l in range(L - 1):
            x.append(self.R[l] @ x[-1])
        gs = []
        for l in range(L):
            g = np.zeros((self.N[l] + 1) * self.d[l], dtype=complex)
            g[:self.d[l]] = x[l]
            gs.append(g)
        u = np.linalg.solve(self.A[L - 1], gs[L - 1])
        for l in range(L - 2, -1, -1):
            d, dc = self.d[l], self.d[l + 1]
            ul = np.zeros((self.N[l] + 1) * d, dtype=complex)
            ul[:d] = x[l]
            for i, c in enumerate(range(self.cf, self.N[l] + 1, self.cf), start=1):
                ul[c * d:(c + 1) * d] = self.P[l] @ u[i * dc:(i + 1) * dc]
            u = self.f_relax(l, ul, gs[l])
        return u, gs[0]

    def run(self, u0, iters, cycle="F"):
        u, g = self.initial(u0)
        out = [u]
        for _ in range(iters):
            u = self.f_cycle(0, u, g) if cycle == "F" else self.v_cycle(0, u, g)
            out.append(u)
        return out

    def cpoints(self, u):
        d = self.d[0]
        return [u[c * d:(c + 1) * d] for c in range(0, self.N[0] + 1, self.cf)]


def _random_prop(rng, d, scale):
    """A non-normal propagator of spectral size about one: a damped random unitary
    matrix plus ``scale`` times a random complex matrix."""
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)))
    return 0.97 * Q + scale * (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / d


def _case(L, dims, seed, N0, cf):
    """Level-l+1 propagator = the restricted cf-th power of level l's plus a random
    perturbation: a coarse propagator that approximates the fine one, as in MGRIT."""
    rng = np.random.default_rng(seed)
    Rs = [np.eye(dims[l + 1], dims[l]) for l in range(L - 1)]     # truncation
    Ps = [np.eye(dims[l], dims[l + 1]) for l in range(L - 1)]     # zero padding
    Phis = [_random_prop(rng, dims[0], 0.1)]
    for l in range(L - 1):
        Pc = Rs[l] @ np.linalg.matrix_power(Phis[l], cf) @ Ps[l]
        d = dims[l + 1]
        Phis.append(Pc + 0.05 * (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / d)
    u0 = rng.standard_normal(dims[0]) + 1j * rng.standard_normal(dims[0])
    return Phis, Rs, Ps, u0


def _oracle(Phis, Rs, Ps, N0, cf, nu):
    steps = [(lambda P: (lambda x, prev: P @ x))(P) for P in Phis]
    Rf = [(lambda R: (lambda x: R @ x))(R) for R in Rs] + [lambda x: x]
    Pf = [(lambda P: (lambda x: P @ x))(P) for P in Ps] + [lambda x: x]
    return pint.MGRIT(steps, N0=N0, cf=cf, nu=nu, restrict_space=Rf, prolong_space=Pf)


CASES = [
    # (levels, state dimension per level, N0, cf, nu)
    (2, [3, 3], 12, 3, 0),
    (2, [3, 3], 16, 2, 1),
    (3, [3, 3, 3], 32, 2, 0),
    (3, [3, 3, 3], 36, 3, 1),
    (3, [4, 3, 2], 32, 2, 0),    # spatial coarsening on both coarse levels
    (4, [3, 3, 3, 3], 32, 2, 0),
]


@pytest.mark.parametrize("L,dims,N0,cf,nu", CASES)
def test_oracle_mgrit_equals_dense_fas(L, dims, N0, cf, nu):
    Phis, Rs, Ps, u0 = _case(L, dims, 11 + L + N0 + nu, N0, cf)
    dense = DenseMGRIT(Phis, N0, cf, nu, Rs, Ps)
    ref = dense.run(u0, 4)
    got = _oracle(Phis, Rs, Ps, N0, cf, nu).run(u0, 4)
    for k in range(5):
        rc = dense.cpoints(ref[k])
        scale = max(np.max(np.abs(x)) for x in rc)
        for i, x in enumerate(got[k]):
            assert np.max(np.abs(x - rc[i])) <= 1e-12 * scale, (k, i)


@pytest.mark.parametrize("L,dims,N0,cf,nu", [c for c in CASES if len(set(c[1])) == 1])
def test_dense_fas_reaches_serial_fine_solution(L, dims, N0, cf, nu):
    """Finite termination (§3.2.3): the iterates become A_0^{-1} g_0, the serial fine
    solution, after N_0 / ((nu+1) cf) iterations at most.  (Only without spatial
    coarsening: a truncated coarse level cannot represent the whole residual.)"""
    Phis, Rs, Ps, u0 = _case(L, dims, 11 + L + N0 + nu, N0, cf)
    dense = DenseMGRIT(Phis, N0, cf, nu, Rs, Ps)
    kmax = N0 // ((nu + 1) * cf)
    it = dense.run(u0, kmax)
    exact = np.linalg.solve(dense.A[0], it[0] * 0 + np.concatenate([u0, np.zeros(N0 * dims[0])]))
    assert np.max(np.abs(it[-1] - exact)) <= 1e-10 * np.max(np.abs(exact))
    assert np.max(np.abs(it[0] - exact)) > 1e-3 * np.max(np.abs(exact))   # the guess really differs


def test_post_v_cycle_matters():
    """The 3-level F-cycle with and without the post V-cycle give different iterates
    (so the comparison above can tell them apart)."""
    Phis, Rs, Ps, u0 = _case(3, [3, 3, 3], 99, 32, 2)
    dense = DenseMGRIT(Phis, 32, 2, 0, Rs, Ps)
    u, g = dense.initial(u0)
    full = dense.f_cycle(0, u, g)

    def no_post(lc, uc, gc):
        if lc == dense.L - 1:
            return dense.solve(lc, uc, gc)
        return dense.f_cycle(lc, uc, gc)
    partial = dense.two_grid(0, u, g, no_post)
    assert np.max(np.abs(full - partial)) > 1e-6 * np.max(np.abs(full))
