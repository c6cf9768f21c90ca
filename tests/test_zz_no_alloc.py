"""The allocation-free residual entry point (trs_residual_norm_noalloc).

It serves callers that may not allocate device memory while they run; its
reduction scratch is a static array inside the library.  Checked here
against the existing entry points on two calls in a row: the residual
against r = b - A x from trs_bsr_spmv, and the norm against the true
residual that trs_fgmres_solve reports (same kernel, same grid).  This file
is collected last so that a failure here comes after every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def trs():
    from paper_1812_03952_gb300 import build as B
    B.build()
    from paper_1812_03952_gb300 import trs as T
    T.load()
    return T


# 80x80x50 has 320,000 cell rows, more than the 1,216 blocks of 256 threads
# cover in one pass, so there the blocks stride over the rows more than once.
@pytest.mark.parametrize("shape,b", [((13, 11, 7), 4), ((9, 8, 5), 5), ((40, 30, 20), 4), ((80, 80, 50), 4)])
def test_noalloc_residual_matches_existing_entry_points(trs, synth, shape, b):
    sysm = synth.small_system(*shape, b=b, seed=61, n_pairs=2)
    ds = trs.DeviceSystem(sysm)
    A = ds.assemble()
    M = trs.CPR(A, precision="fp64")
    x, res = trs.fgmres_solve(A, M, ds.rhs, rtol=1e-8)
    assert res.status == trs.TRS_OK
    bnorm = float(torch.linalg.norm(ds.rhs))
    xs = [x, x + 1e-3 * torch.randn_like(x)]
    for xi in xs:                       # two calls in a row share the static scratch
        r = torch.full_like(ds.rhs, float("nan"))
        nrm = trs.residual_norm_noalloc(A, xi, ds.rhs, r)
        ref = ds.rhs.clone()
        A.spmv(xi, ref, alpha=-1.0, beta=1.0)
        scale = float(torch.linalg.norm(ds.rhs)) + float(torch.linalg.norm(xi))
        assert float(torch.max(torch.abs(r - ref))) <= 1e-12 * scale
        np.testing.assert_allclose(nrm, float(torch.linalg.norm(ref)), rtol=1e-12)
    # the same kernel and grid as the solver's own true-residual check
    r = torch.empty_like(ds.rhs)
    nrm = trs.residual_norm_noalloc(A, x, ds.rhs, r)
    np.testing.assert_allclose(nrm / bnorm, res.stats["true_relres"], rtol=1e-12)
