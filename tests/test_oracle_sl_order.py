"""Temporal-order pin of the oracle's two-step SL-SI-SETTLS (§2.3.2, Eqs. 6-7).

SL-SI-SETTLS is a second-order scheme: the SETTLS trajectory uses the
extrapolated midpoint velocity 2V^n - V^{n-1} (Eq. 6) and the nonlinear
remainder is the average of its extrapolation 2N_R^n - N_R^{n-1} at the
departure point and N_R^n at the arrival point (Eq. 7).  On a smooth,
divergent, unbalanced T21 state (gravity waves plus advection, with a large
Phi' so that N_R = -Phi' delta matters) the error against a run with a 4x
smaller step than the finest one must fall by about 4 each time the step is
halved.  Swapping the extrapolation to 2N_R^{n-1} - N_R^n, interpolating the
trajectory velocity at one time level only, or exchanging the two time
levels of the velocity each makes the scheme first order (ratios of about 2),
so each of those mistakes fails this test.  The one-step variant used inside
PinT (t_{n-1} data replaced by t_n data, §3.2.4) is first order.

Interpolation error does not spoil the order: at Courant numbers below one
the cubic Lagrange error per step is proportional to the displacement, so its
accumulated value over a fixed horizon hardly depends on the step.
"""
import numpy as np
import pytest

from oracle.sphere import Sphere
from oracle.swe import SWE, to_dense
from paper_2306_09497_gb300 import inputs

T = 4 * 3600.0
STEPS = (24, 48, 96)
REF_STEPS = 384


@pytest.fixture(scope="module")
def t21():
    s = Sphere(21, 32, 64)
    sw = SWE(s)
    U = inputs.random_state(21, 1, seed=5, scale=(2.0e4, 2.0e-5, 5.0e-6))[0]
    _, n = inputs.mn_arrays(21)
    U[:, n > 8] = 0.0                      # smooth: degrees up to 8
    return s, sw, to_dense(s, U)


def _run(sw, U0, nsteps, two_step=True):
    dt = T / nsteps
    U, Up = U0, None
    for _ in range(nsteps):
        U, Up = sw.sl_si_settls_step(U, Up if two_step else None, dt), U
    return U


def _err(a, b):
    return max(np.linalg.norm(a[f] - b[f]) / np.linalg.norm(b[f]) for f in range(3))


@pytest.fixture(scope="module")
def reference(t21):
    s, sw, U0 = t21
    return _run(sw, U0, REF_STEPS)


def test_two_step_sl_si_settls_is_second_order(t21, reference):
    s, sw, U0 = t21
    e = [_err(_run(sw, U0, n), reference) for n in STEPS]
    ratios = [e[i] / e[i + 1] for i in range(len(e) - 1)]
    for r in ratios:
        assert 3.5 < r < 4.6, (e, ratios)


def test_one_step_variant_is_first_order(t21, reference):
    s, sw, U0 = t21
    e = [_err(_run(sw, U0, n, two_step=False), reference) for n in STEPS[:2]]
    assert 1.6 < e[0] / e[1] < 2.6, e
