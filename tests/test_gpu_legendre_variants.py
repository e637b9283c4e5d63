"""The two tensor-core Legendre kernel variants (persistent: one CTA per SM over all work items
with double-buffered TMEM accumulators; per tile: one CTA per item) issue the same MMAs in the
same order for every (column tile, m, N tile) item, so their results must agree bit for bit.
Each is also checked against the FP64 oracle through the scalar transforms (bounds of the
split path: inverse 1e-6 of the largest grid value, forward 5e-6 of the largest coefficient),
at widths that give one and many column tiles, and through one nonlinear evaluation in the
benchmark's T255 configuration.  The autotuner's record names the variant it kept.
"""
import numpy as np
import pytest

from oracle.sphere import Sphere
from paper_2306_09497_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy()).cuda()


@pytest.mark.parametrize("M,nlat,nlon,B", [(63, 96, 192, 20), (127, 192, 384, 96), (255, 384, 768, 20),
                                           (255, 384, 768, 200)])
def test_variants_identical_and_match_oracle(M, nlat, nlon, B):
    from paper_2306_09497_gb300 import swe
    plan = swe.Plan(M, nlat, nlon, prec=swe.SWE_SPLIT_BF16X3)
    s = Sphere(M, nlat, nlon)
    coef = _dev(inputs.random_coeffs(M, B, seed=31))
    g = inputs.random_grid(nlat, nlon, B, seed=32).astype(np.float32)
    grid_in = torch.from_numpy(g).cuda()
    outs = {}
    for mode in (swe.SWE_LEGENDRE_PERSISTENT, swe.SWE_LEGENDRE_PER_TILE):
        plan.set_legendre_mode(mode)
        grid = torch.empty((B, nlat, nlon), dtype=torch.float32, device="cuda")
        spec = torch.empty((B, plan.nc * 2), dtype=torch.float64, device="cuda")
        plan.sht_inverse(coef, grid, B)
        plan.sht_forward(grid_in, spec, B)
        assert plan.check() == swe.SWE_OK
        outs[mode] = (grid.cpu().numpy(), spec.cpu().numpy())
    gp, sp = outs[swe.SWE_LEGENDRE_PERSISTENT]
    gt, st = outs[swe.SWE_LEGENDRE_PER_TILE]
    assert np.array_equal(gp, gt)
    assert np.array_equal(sp, st)
    c = coef.cpu().numpy().view(np.complex128).reshape(B, -1)
    got = sp.view(np.complex128).reshape(B, -1)
    for b in (0, B - 1):
        ref = s.sh_to_grid(s.unpack(c[b]))
        assert np.max(np.abs(gp[b].astype(np.float64) - ref)) < 1e-6 * np.max(np.abs(ref))
        refs = s.pack(s.grid_to_sh(g[b].astype(np.float64)))
        assert np.max(np.abs(got[b] - refs)) < 5e-6 * np.max(np.abs(refs))
    plan.close()


def test_variants_identical_nonlinear_t255_and_tuning_record():
    from paper_2306_09497_gb300 import swe
    M, nlat, nlon, S = 255, 384, 768, 32
    plan = swe.Plan(M, nlat, nlon, prec=swe.SWE_SPLIT_BF16X3)
    U = _dev(inputs.random_state(M, S, 33))
    res = []
    for mode in (swe.SWE_LEGENDRE_PERSISTENT, swe.SWE_LEGENDRE_PER_TILE, swe.SWE_LEGENDRE_AUTO):
        plan.set_legendre_mode(mode)
        N = torch.empty((S, 3, plan.nc * 2), dtype=torch.float64, device="cuda")
        plan.nonlinear(U, N, S)
        assert plan.check() == swe.SWE_OK
        res.append(N.cpu().numpy())
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])
    text = plan.tuning()
    # the automatic mode timed both variants for the 4S inverse and 5S forward columns
    assert "inverse ncol %d" % (2 * 4 * S) in text and "forward ncol %d" % (2 * 5 * S) in text, text
    plan.close()
