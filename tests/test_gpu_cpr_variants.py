"""CPR stage orderings (FPF, FP, PF) and decoupling methods (ABF, NONE, FRS,
FRS+ABF) of the CUDA path against the oracle (Sec. "Preconditioners",
Sec. "Decoupling Methods").

The decoupled blocks, D^-1, the pressure operators of every level, the
aggregates and the colours are compared bit for bit (same operations in
the same order on both sides); one preconditioner application is compared
at 1e-11 relative (same operations, different summation order); the solves
meet the true FP64 residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from test_gpu_parity import CASES, _case_id, _gpu_system, _rel, _sys  # noqa: E402

DECOUPLINGS = ["abf", "none", "frs", "frs+abf"]
STAGES = ["fpf", "fp", "pf"]
VCASES = [CASES[0], CASES[3], CASES[4], CASES[5]]


@pytest.fixture(scope="module")
def trs():
    from paper_1812_03952_gb300 import build as B
    B.build()
    from paper_1812_03952_gb300 import trs as T
    T.load()
    return T


@pytest.mark.parametrize("decoupling", DECOUPLINGS)
@pytest.mark.parametrize("case", VCASES, ids=_case_id)
def test_decoupling_setup_bit_exact(trs, oracle, synth, case, decoupling):
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    Mo = oracle.CPR(Ao, coarse_max=40, decoupling=decoupling)
    amg = Mo.amg
    for precision in ("fp64", "fp32"):
        M = trs.CPR(ds.A, coarse_max=40, decoupling=decoupling, precision=precision)
        info = M.info()
        assert info["level_rows"] == amg.sizes()
        for l in range(amg.n_levels):
            rp, col, val = M.level(l)
            rpo, colo, valo = amg.level(l)
            np.testing.assert_array_equal(rp, rpo)
            np.testing.assert_array_equal(col, colo)
            np.testing.assert_array_equal(val, valo)
            np.testing.assert_array_equal(M.aggregates(l), amg.agg(l))
        np.testing.assert_array_equal(M.colours(), Mo.colours())
        if precision == "fp64":
            vt, dinv = M.decoupled(Ao.nnzb)
            vto, dinvo = Mo.decoupled()
            np.testing.assert_array_equal(dinv, dinvo)
            np.testing.assert_array_equal(vt, vto)


@pytest.mark.parametrize("decoupling", DECOUPLINGS)
@pytest.mark.parametrize("stages", STAGES)
@pytest.mark.parametrize("case", VCASES, ids=_case_id)
def test_cpr_apply_variants(trs, oracle, synth, case, stages, decoupling):
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    kw = dict(coarse_max=40, stages=stages, decoupling=decoupling)
    M = trs.CPR(ds.A, **kw)
    Mo = oracle.CPR(Ao, **kw)
    v = np.random.default_rng(12).standard_normal(Ao.n * Ao.b)
    z = M.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert _rel(z, Mo.apply(v)) <= 1e-11


@pytest.mark.parametrize("method", ["fgmres", "bicgstab"])
@pytest.mark.parametrize("decoupling", ["abf", "none", "frs"])
@pytest.mark.parametrize("stages", STAGES)
def test_solve_with_variants(trs, oracle, synth, stages, decoupling, method):
    s = _sys(synth, 20, 18, 10, 4, seed=9, n_pairs=2, sigma=2.0, shale_frac=0.1)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    kw = dict(stages=stages, decoupling=decoupling)
    ref_iters = {
        "fgmres": lambda: oracle.fgmres(Ao, oracle.CPR(Ao, **kw), s.rhs, rtol=1e-8).iters,
        "bicgstab": lambda: oracle.bicgstab(Ao, oracle.CPR(Ao, **kw), s.rhs, rtol=1e-8).iters,
    }[method]()
    for precision in ("fp64", "fp32"):
        M = trs.CPR(ds.A, precision=precision, **kw)
        x, res = trs.krylov_solve(method, ds.A, M, ds.rhs, rtol=1e-8)
        assert res.status == trs.TRS_OK
        tr = np.linalg.norm(s.rhs - oracle.spmv(Ao, x.cpu().numpy())) / np.linalg.norm(s.rhs)
        assert tr <= 1.01e-8
        if precision == "fp64":
            assert abs(res.stats["iters"] - ref_iters) <= max(2, ref_iters // 10)


def test_invalid_variant_options(trs, synth):
    s = _sys(synth, 4, 4, 2, 4, seed=3)
    ds = _gpu_system(trs, s)
    for bad in (dict(stages=3), dict(stages=-1), dict(decoupling=4)):
        with pytest.raises(trs.TrsError) as ei:
            trs.CPR(ds.A, **bad)
        assert ei.value.code == trs.TRS_ERR_INVALID
