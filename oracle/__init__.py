"""Serial FP64 CPU oracle for the Parareal/MGRIT shallow-water method (arXiv 2306.09497).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (the CUDA library and its Python binding) never calls
it, and it shares no code with the product: every routine here is written
from the paper's equations in the plainest form (direct quadrature Legendre
sums, a naive DFT by matrix product, dense/banded linear solves, serial
Parareal and MGRIT loops).

Modules
-------
sphere     Gauss-Legendre grid, normalised associated Legendre functions,
           naive DFT, scalar and vector spherical-harmonic transforms (§2.2).
swe        operators L_G, L_C, N_A, N_R, viscosity (Eq. 1, App. A), the
           Crank-Nicolson solve (Eq. 4), IMEX (Eqs. 3-5), SL-SI-SETTLS (Eqs. 6-7),
           nonlinear balance used by the input recipe.
pint       serial fine reference, Parareal (Eq. 9), MGRIT FAS cycles (§3.2).
stability  scalar linear test ODE (Eqs. 10-20): schemes and closed forms.
norms      error norms of §5 (Eq. 21 and the physical L2 norm).

Parity status of every function is stated in its docstring; functions with
no independent pin say "parity unpinned".
"""
