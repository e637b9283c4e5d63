"""Serial fine reference, Parareal and MGRIT (oracle; test use only).

Propagators are plain Python callables on whatever state type the caller
uses (SWE state tuples, complex scalars, ...); states are combined through
the ``axpy`` helpers below so the same loops serve the scalar test ODE.
"""
from __future__ import annotations

from typing import Callable, List, Optional


def _add(a, b):
    if isinstance(a, tuple):
        return tuple(x + y for x, y in zip(a, b))
    return a + b


def _sub(a, b):
    if isinstance(a, tuple):
        return tuple(x - y for x, y in zip(a, b))
    return a - b


def serial(U0, step: Callable, nsteps: int):
    """Serial application of a one-step propagator nsteps times (fine reference, §3.1)."""
    U = U0
    for _ in range(nsteps):
        U = step(U)
    return U


def parareal(U0, fine: Callable, coarse: Callable, N: int, K: int):
    """Parareal, §3.1 Eq. 9.

    Iteration 0 is the serial coarse sweep U^0_{n+1} = G(U^0_n); then
    U^{k+1}_{n+1} = G(U^{k+1}_n) + F(U^k_n) - G(U^k_n).  ``fine``/``coarse``
    propagate one time slice [T_n, T_{n+1}].  Returns the list of iterates
    [U^0, ..., U^K], each a list of the N+1 slice-boundary states.
    """
    U = [U0]
    Gold = []
    for n in range(N):
        g = coarse(U[n])
        Gold.append(g)
        U.append(g)
    hist = [list(U)]
    for _ in range(K):
        F = [fine(U[n]) for n in range(N)]
        Unew = [U0]
        for n in range(N):
            g = coarse(Unew[n])
            Unew.append(_add(g, _sub(F[n], Gold[n])))
            Gold[n] = g
        U = Unew
        hist.append(list(U))
    return hist


class MGRIT:
    """Multilevel MGRIT with FAS (§3.2), F(CF)^nu relaxation, F-cycle + one V-cycle.

    Level l has N_l = N_0 / cf^l steps; ``steps[l](u, u_prev)`` advances one
    step of level l (``u_prev`` is the state one step earlier on that level,
    None when unavailable; one-step schemes ignore it).  ``two_step[l]``
    marks levels whose stepper uses the previous state during the serial
    coarsest-level solve (the two-step SL-SI-SETTLS variant of §3.2.4);
    relaxations always run the one-step form, because their steps start
    from a C-point without an earlier state.

    Readings (the paper defers to the XBraid documentation, which is not
    available): the initial guess is the serial coarsest-level propagation
    injected upwards with F-relaxation on every finer level; one iteration
    is one F-cycle: F(l) = relax(l); restrict; [solve | F(l+1); V(l+1)];
    correct(l) with F-relaxation; V(l) = relax(l); restrict; [solve | V(l+1)];
    correct(l).  Restriction is injection at C-points (§3.2.2 step 2).
    """

    def __init__(self, steps: List[Callable], N0: int, cf: int, nu: int,
                 two_step: Optional[List[bool]] = None,
                 restrict_space: Optional[List[Callable]] = None,
                 prolong_space: Optional[List[Callable]] = None):
        self.L = len(steps)
        self.steps, self.cf, self.nu = steps, cf, nu
        self.N = [N0 // cf ** l for l in range(self.L)]
        assert all(self.N[l] * cf ** l == N0 for l in range(self.L))
        self.two_step = two_step or [False] * self.L
        ident = lambda x: x
        # spatial transfer from level l to l+1 (index l) and back
        self.Rs = restrict_space or [ident] * self.L
        self.Ps = prolong_space or [ident] * self.L
        self.u: List[list] = [None] * self.L
        self.g: List[list] = [None] * self.L
        self.v: List[list] = [None] * self.L      # restricted values (for the correction)

    # -- elementary pieces -------------------------------------------
    def _phi(self, l, x):
        return self.steps[l](x, None)

    def _plus_g(self, l, j, x):
        g = self.g[l][j] if self.g[l] is not None else None
        return x if g is None else _add(x, g)

    def f_relax(self, l):
        cf, u = self.cf, self.u[l]
        for i in range(self.N[l] // cf):
            for j in range(cf * i + 1, cf * i + cf):
                u[j] = self._plus_g(l, j, self._phi(l, u[j - 1]))

    def c_relax(self, l):
        cf, u = self.cf, self.u[l]
        for i in range(1, self.N[l] // cf + 1):
            j = cf * i
            u[j] = self._plus_g(l, j, self._phi(l, u[j - 1]))

    def relax(self, l):
        self.f_relax(l)
        for _ in range(self.nu):
            self.c_relax(l)
            self.f_relax(l)

    def restrict(self, l):
        """FAS restriction: v_i = R u_{cf i};  g_{l+1,i} = R r_{cf i} + v_i - Phi_{l+1}(v_{i-1})."""
        cf, u, R = self.cf, self.u[l], self.Rs[l]
        Nc = self.N[l + 1]
        v = [R(u[cf * i]) for i in range(Nc + 1)]
        g = [None] * (Nc + 1)
        g[0] = v[0]
        for i in range(1, Nc + 1):
            j = cf * i
            # residual of A_l u = g_l at the C-point: g_j - (u_j - Phi_l(u_{j-1}))
            r = _sub(self._phi(l, u[j - 1]), u[j])
            if self.g[l] is not None and self.g[l][j] is not None:
                r = _add(r, self.g[l][j])
            g[i] = _add(R(r), _sub(v[i], self._phi(l + 1, v[i - 1])))
        self.v[l + 1] = v
        self.g[l + 1] = g
        self.u[l + 1] = list(v)

    def correct(self, l):
        """u_{cf i} += P(v_i^{new} - v_i^{restricted}), then F-relaxation (§3.2.2 step 5)."""
        cf, P = self.cf, self.Ps[l]
        for i in range(1, self.N[l + 1] + 1):
            e = _sub(self.u[l + 1][i], self.v[l + 1][i])
            self.u[l][cf * i] = _add(self.u[l][cf * i], P(e))
        self.f_relax(l)

    def solve_coarsest(self, l):
        u = self.u[l]
        g = self.g[l]
        u[0] = g[0] if g is not None else u[0]
        for i in range(1, self.N[l] + 1):
            prev = u[i - 2] if (self.two_step[l] and i >= 2) else None
            x = self.steps[l](u[i - 1], prev)
            u[i] = self._plus_g(l, i, x)

    def v_cycle(self, l):
        if l == self.L - 1:
            self.solve_coarsest(l)
            return
        self.relax(l)
        self.restrict(l)
        self.v_cycle(l + 1)
        self.correct(l)

    def f_cycle(self, l):
        if l == self.L - 1:
            self.solve_coarsest(l)
            return
        self.relax(l)
        self.restrict(l)
        if l + 1 == self.L - 1:
            self.solve_coarsest(l + 1)
        else:
            self.f_cycle(l + 1)
            self.v_cycle(l + 1)
        self.correct(l)

    # -- driver ---------------------------------------------------------
    def initial_guess(self, U0):
        """Serial coarsest-level propagation, injected to finer levels + F-relaxation."""
        Lc = self.L - 1
        # restrict the initial condition spatially down to the coarsest level
        x = U0
        xs = [U0]
        for l in range(Lc):
            x = self.Rs[l](x)
            xs.append(x)
        self.g = [None] * self.L
        self.u[Lc] = [xs[Lc]] + [None] * self.N[Lc]
        self.solve_coarsest(Lc)
        for l in range(Lc - 1, -1, -1):
            u = [None] * (self.N[l] + 1)
            u[0] = xs[l]
            for i in range(1, self.N[l + 1] + 1):
                u[self.cf * i] = self.Ps[l](self.u[l + 1][i])
            self.u[l] = u
            self.f_relax(l)
        # coarse RHS arrays are rebuilt by each restriction
        self.g = [None] * self.L

    def c_points(self):
        return [self.u[0][self.cf * i] for i in range(self.N[1] + 1)]

    def run(self, U0, iters: int):
        """Return C-point values of level 0 after the initial guess and each iteration."""
        self.initial_guess(U0)
        hist = [self.c_points()]
        for _ in range(iters):
            self.f_cycle(0)
            hist.append(self.c_points())
        return hist
