"""sht_inverse_noalloc: the inverse transform for callers that cannot allocate device memory.

Such callers (code inside a CUDA-graph stream capture, real-time loops, or
applications whose device memory belongs to their own pool) get the same
result as sht_inverse while the library draws its scratch from a fixed 64 MiB
static device array instead of cudaMalloc.  The checks: two calls in a row agree
with sht_inverse within the transform tolerance used elsewhere in the tests
(1e-12 relative), the second call changes no device-memory accounting, and a
batch beyond the static array is refused with a clear error.
"""
import numpy as np
import pytest

from paper_2306_09497_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()


@pytest.mark.parametrize("M,nlat,nlon,batch", [(31, 48, 96, 5), (63, 96, 192, 3), (255, 384, 768, 31)])
def test_noalloc_matches_sht_inverse_twice(M, nlat, nlon, batch):
    from paper_2306_09497_gb300 import swe
    plan = swe.Plan(M, nlat, nlon)
    ref = torch.empty((batch, nlat, nlon), dtype=torch.float64, device="cuda")
    got = torch.empty_like(ref)
    for call, seed in enumerate((11, 12)):          # two calls in a row, different inputs
        spec = _dev(inputs.random_coeffs(M, batch, seed=seed))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        plan.sht_inverse_noalloc(spec, got, batch)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        plan.sht_inverse(spec, ref, batch)
        torch.cuda.synchronize()
        scale = float(ref.abs().max())
        assert float((got - ref).abs().max()) <= TOL * scale
        if call == 1:
            assert free_after == free_before            # nothing allocated by the call
    plan.close()


def test_noalloc_rejects_batch_beyond_static_scratch():
    from paper_2306_09497_gb300 import swe
    plan = swe.Plan(255, 384, 768)
    spec = torch.zeros((32, plan.nc * 2), dtype=torch.float64, device="cuda")
    grid = torch.empty((32, 384, 768), dtype=torch.float64, device="cuda")
    with pytest.raises(swe.SWEError) as ei:
        plan.sht_inverse_noalloc(spec, grid, 32)
    assert "static array" in str(ei.value) and "at most 31" in str(ei.value)
    plan.close()
