"""The bounded waits of the staged Gram-Schmidt kernels.

Their basis tiles arrive by bulk copies completed on mbarriers.  Here every
stage is made to expect 16 bytes more than its copies deliver (through
trs_test_stall_staged_copies), so no wait can succeed: each gives up after
its poll limit, the block's sums become NaN and the solve must end with
TRS_ERR_NAN rather than hang.  Afterwards, with normal operation restored, the
same solve on the same handles must give the same x bit for bit: the context
and the library state are intact.  Nothing faults: the copies all land, only
the barrier's byte count is never reached.
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


def test_stall_hook_validates_its_argument(trs):
    for bad in (-16, 8, 65552):
        with pytest.raises(trs.TrsError) as e:
            trs.test_stall_staged_copies(bad)
        assert e.value.code == trs.TRS_ERR_INVALID
    trs.test_stall_staged_copies(0)


def test_stalled_stages_end_the_solve_with_nan_status(trs, synth):
    sysm = synth.small_system(24, 20, 10, 4, seed=71, n_pairs=1)   # N even: the staged kernels run
    ds = trs.DeviceSystem(sysm)
    A = ds.assemble()
    M = trs.CPR(A)
    x0, r0 = trs.fgmres_solve(A, M, ds.rhs, rtol=1e-8)
    assert r0.status == trs.TRS_OK
    x0 = x0.cpu().numpy().copy()
    trs.test_stall_staged_copies(16)
    try:
        with pytest.raises(trs.TrsError) as e:
            trs.fgmres_solve(A, M, ds.rhs, rtol=1e-8)
        assert e.value.code == trs.TRS_ERR_NAN
    finally:
        trs.test_stall_staged_copies(0)
    torch.cuda.synchronize()
    x1, r1 = trs.fgmres_solve(A, M, ds.rhs, rtol=1e-8)
    assert r1.status == trs.TRS_OK and r1.stats["iters"] == r0.stats["iters"]
    np.testing.assert_array_equal(x1.cpu().numpy(), x0)
