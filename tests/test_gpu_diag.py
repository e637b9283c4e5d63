"""Parity of the §5 diagnostics (Eq. 21 error norms, area-weighted L2, KE spectrum) with the
oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import norms
from paper_2306_09497_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()


def _unpack(M, v):
    """Packed m-major triangular coefficients -> dense [m, n] (storage layout only)."""
    m, n = inputs.mn_arrays(M)
    d = np.zeros((M + 1, M + 1), dtype=np.complex128)
    d[m, n] = v
    return d


@pytest.mark.parametrize("M,nlat,nlon,S,R", [(31, 48, 96, 5, 16), (63, 96, 192, 3, 63), (255, 384, 768, 7, 32),
                                             (127, 192, 384, 300, 0)])
def test_error_norms_match_oracle(M, nlat, nlon, S, R):
    from paper_2306_09497_gb300 import swe
    plan = swe.Plan(M, nlat, nlon)
    ref = inputs.random_state(M, S, seed=21)
    rng = np.random.default_rng(5)
    U = ref + 1e-4 * inputs.random_state(M, S, seed=22) * rng.uniform(0.1, 2.0, size=(S, 3, 1))
    got = plan.error_norms(_dev(U), _dev(ref), S, R)
    for k in range(S):
        for f in range(3):
            a, b = _unpack(M, U[k, f]), _unpack(M, ref[k, f])
            if np.max(np.abs(b[: R + 1, : R + 1])) > 0:
                e = norms.spectral_error(a, b, R)
                assert abs(got[k, f, 0] - e) <= 1e-13 * e
            l2 = norms.parseval_l2_error(a, b)
            assert abs(got[k, f, 1] - l2) <= 1e-13 * l2
    plan.close()


def test_error_norms_of_equal_states_are_zero():
    from paper_2306_09497_gb300 import swe
    plan = swe.Plan(31, 48, 96)
    U = _dev(inputs.random_state(31, 2, seed=3))
    got = plan.error_norms(U, U, 2, 31)
    assert np.all(got == 0.0)
    with pytest.raises(swe.SWEError):
        plan.error_norms(U, U, 2, 32)          # R_norm > M
    plan.close()


@pytest.mark.parametrize("M,nlat,nlon,S", [(31, 48, 96, 4), (255, 384, 768, 9), (511, 768, 1536, 2)])
def test_ke_spectrum_matches_oracle(M, nlat, nlon, S):
    from paper_2306_09497_gb300 import swe
    plan = swe.Plan(M, nlat, nlon, prec=swe.SWE_SPLIT_BF16X3 if M > 300 else swe.SWE_FP64)
    U = inputs.random_state(M, S, seed=30, scale=(1.0e3, 1.0e-5, 3.0e-6))
    E = torch.empty((S, M + 1), dtype=torch.float64, device="cuda")
    plan.ke_spectrum(_dev(U), S, E)
    got = E.cpu().numpy()
    for k in range(S):
        ref = norms.ke_spectrum(_unpack(M, U[k, 1]), _unpack(M, U[k, 2]), plan.a)
        assert np.max(np.abs(got[k] - ref)) <= 1e-13 * np.max(ref)
    plan.close()
