"""sht_inverse_noalloc: the inverse transform for callers that cannot allocate device memory.

Such callers (real-time loops that forbid allocator calls, or applications
whose device memory belongs to their own pool) get the same
result as sht_inverse while the library draws its scratch from a fixed 64 MiB
static device array instead of cudaMalloc.  The checks, on FP64 and on
split-precision plans: two calls in a row agree with sht_inverse within the
transform tolerance used elsewhere in the tests (1e-12 relative on FP64 plans; on
split plans both entry points run the same FP32/tensor-core kernels, so the same
bound holds), the second call changes no device-memory accounting, and a batch
beyond the static array is refused with a clear error that names the largest
batch the array takes.
"""
import numpy as np
import pytest

from paper_2306_09497_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()


@pytest.mark.parametrize("M,nlat,nlon,batch,prec", [
    (31, 48, 96, 5, "fp64"), (63, 96, 192, 3, "fp64"), (255, 384, 768, 31, "fp64"),
    # split-precision plans: a narrow batch (FP32 SIMT contraction) and batches above 8
    # fields, where the tcgen05 inverse reads its TMA-fed operand from the static array
    (63, 96, 192, 3, "split"), (127, 192, 384, 40, "split"), (255, 384, 768, 40, "split")])
def test_noalloc_matches_sht_inverse_twice(M, nlat, nlon, batch, prec):
    from paper_2306_09497_gb300 import swe
    plan = swe.Plan(M, nlat, nlon, prec=swe.SWE_FP64 if prec == "fp64" else swe.SWE_SPLIT_BF16X3)
    # the same kernels run in both calls, so the split plans are held to the same bound
    ref = torch.empty((batch, nlat, nlon), dtype=torch.float64 if prec == "fp64" else torch.float32,
                      device="cuda")
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
    # the largest batch the message names is accepted
    plan.sht_inverse_noalloc(spec, grid, 31)
    torch.cuda.synchronize()
    plan.close()
