"""Pins of the oracle's Parareal / MGRIT on the SWE (§3): finite termination and equivalence."""
import numpy as np
import pytest

from oracle import pint
from oracle.sphere import Sphere
from oracle.swe import SWE, to_dense
from paper_2306_09497_gb300 import inputs


@pytest.fixture(scope="module")
def setup():
    s = Sphere(15, 24, 48)
    sw = SWE(s)
    xi, noise = inputs.initial_fields(s.M, 1)
    xi = s.unpack(xi)
    U0 = (sw.balanced_geopotential(xi) + s.unpack(noise), xi, np.zeros_like(xi))
    fine = lambda U: pint.serial(U, lambda X: sw.imex_step(X, 600.0), 3)
    coarse = lambda U: sw.imex_step(U, 1800.0, nu=1e5, q=2)
    return s, sw, U0, fine, coarse


def _rel(a, b):
    scale = max(np.max(np.abs(b[f])) for f in range(3))
    return max(np.max(np.abs(a[f] - b[f])) / max(np.max(np.abs(b[f])), 1e-30 * scale) for f in range(3))


def test_parareal_reaches_serial_fine_after_N_iterations(setup):
    s, sw, U0, fine, coarse = setup
    N = 4
    hist = pint.parareal(U0, fine, coarse, N, N)
    ref = [U0]
    for n in range(N):
        ref.append(fine(ref[-1]))
    for k in range(N + 1):
        for n in range(k + 1):
            assert _rel(hist[k][n], ref[n]) < 1e-13
    assert _rel(hist[0][N], ref[N]) > 1e-6          # the coarse guess really differs


def test_two_level_mgrit_nu0_equals_parareal_swe(setup):
    s, sw, U0, fine, coarse = setup
    N, cf = 4, 3
    f_step = lambda U, p: sw.imex_step(U, 600.0)
    g_step = lambda U, p: coarse(U)
    m = pint.MGRIT([f_step, g_step], N0=N * cf, cf=cf, nu=0)
    hm = m.run(U0, 2)
    hp = pint.parareal(U0, fine, coarse, N, 2)
    for k in range(3):
        for n in range(N + 1):
            assert _rel(hm[k][n], hp[k][n]) < 1e-12
