"""Block ILU(1) as the F stage of CPR (Sec. "Preconditioners": block ILU(k),
level 1 recommended) on the CUDA path against the oracle.

The distance-2 colours are compared bit for bit; one preconditioner
application is compared at 1e-11 relative in FP64 (same operations on the
same level-1 pattern, different summation order in the sweeps' gathers);
the solves meet the true FP64 residual and need no more iterations than
with ILU(0).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from test_gpu_parity import CASES, _case_id, _gpu_system, _rel, _sys  # noqa: E402

ICASES = CASES   # b = 1 ... 5, wells, shale, ragged tails


@pytest.fixture(scope="module")
def trs():
    from paper_1812_03952_gb300 import build as B
    B.build()
    from paper_1812_03952_gb300 import trs as T
    T.load()
    return T


def _grid(s):
    return (s.nx, s.ny, s.nz)


@pytest.mark.parametrize("case", ICASES, ids=_case_id)
def test_ilu1_setup_and_apply_match_oracle(trs, oracle, synth, case):
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    v = np.random.default_rng(31).standard_normal(Ao.n * Ao.b)
    zo = {}
    for stages in ("fpf", "pf"):
        Mo = oracle.CPR(Ao, coarse_max=40, stages=stages, ilu_fill=1, grid=_grid(s))
        M = trs.CPR(ds.A, coarse_max=40, stages=stages, ilu_fill=1, precision="fp64")
        np.testing.assert_array_equal(M.colours(), Mo.colours())
        assert M.info()["n_colours"] == Mo.info()[1]
        z = M.apply(torch.from_numpy(v).cuda()).cpu().numpy()
        zo[stages] = Mo.apply(v)
        assert _rel(z, zo[stages]) <= 1e-11
    # FP32 preconditioner: the same operator to single-precision accuracy
    M32 = trs.CPR(ds.A, coarse_max=40, ilu_fill=1, precision="fp32")
    z32 = M32.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert _rel(z32, zo["fpf"]) <= 1e-4


@pytest.mark.parametrize("method", ["fgmres", "bicgstab"])
def test_ilu1_solves(trs, oracle, synth, method):
    s = _sys(synth, 20, 18, 10, 4, seed=9, n_pairs=2, sigma=2.0, shale_frac=0.1)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    solve = {"fgmres": oracle.fgmres, "bicgstab": oracle.bicgstab}[method]
    ref = solve(Ao, oracle.CPR(Ao, ilu_fill=1, grid=_grid(s)), s.rhs, rtol=1e-8)
    its0 = None
    for fill in (0, 1):
        for precision in ("fp64", "fp32"):
            M = trs.CPR(ds.A, precision=precision, ilu_fill=fill)
            x, res = trs.krylov_solve(method, ds.A, M, ds.rhs, rtol=1e-8)
            assert res.status == trs.TRS_OK
            tr = np.linalg.norm(s.rhs - oracle.spmv(Ao, x.cpu().numpy())) / np.linalg.norm(s.rhs)
            assert tr <= 1.01e-8
            if precision == "fp64" and fill == 0:
                its0 = res.stats["iters"]
            if precision == "fp64" and fill == 1:
                assert abs(res.stats["iters"] - ref.iters) <= max(2, ref.iters // 10)
                assert res.stats["iters"] <= its0


def test_ilu1_update_refreshes_factors(trs, oracle, synth):
    """After new values (same pattern), the refreshed ILU(1) factors give the
    oracle's application for the new matrix."""
    s = _sys(synth, 12, 9, 6, 4, seed=33, n_pairs=2)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A, precision="fp64", ilu_fill=1)
    s.acc *= 1.3
    ds2 = _gpu_system(trs, s)
    M.update(ds2.A, reuse_amg=False)
    Mo = oracle.CPR(oracle.assemble(s), ilu_fill=1, grid=_grid(s))
    v = np.random.default_rng(34).standard_normal(ds.A.n * ds.A.b)
    z = M.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert _rel(z, Mo.apply(v)) <= 1e-11


def test_ilu1_rejections(trs, oracle, synth):
    s = _sys(synth, 7, 6, 4, 3, seed=35, n_pairs=1)
    Ao = oracle.assemble(s)
    general = trs.Matrix.from_bsr(Ao.rp, Ao.col, Ao.val, s.b, None)
    with pytest.raises(trs.TrsError) as ei:
        trs.CPR(general, ilu_fill=1)
    assert ei.value.code == trs.TRS_ERR_UNSUPPORTED
    # a flattened grid is not a distance-2 order of the 3-D pattern
    flat = trs.Matrix.from_bsr(Ao.rp, Ao.col, Ao.val, s.b, (s.nx * s.ny * s.nz, 1, 1))
    with pytest.raises(trs.TrsError) as ei:
        trs.CPR(flat, ilu_fill=1)
    assert ei.value.code == trs.TRS_ERR_UNSUPPORTED
    with pytest.raises(oracle.OracleError):
        oracle.CPR(Ao, ilu_fill=1, grid=(s.nx * s.ny * s.nz, 1, 1))
    ds = _gpu_system(trs, s)
    with pytest.raises(trs.TrsError) as ei:
        trs.CPR(ds.A, ilu_fill=2)
    assert ei.value.code == trs.TRS_ERR_INVALID


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 1), (1, 1, 7), (3, 1, 2), (2, 2, 2), (4, 3, 2)])
def test_ilu1_degenerate_grids(trs, oracle, synth, dims):
    """Grids with fewer than 7 colours present, with and without wells, against a dense solve."""
    s = synth.small_system(*dims, b=3, seed=42, n_pairs=1 if dims == (4, 3, 2) else 0)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A, ilu_fill=1, precision="fp64")
    np.testing.assert_array_equal(M.colours(), oracle.colour_geo(Ao, _grid(s))[0])
    x, res = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-12)
    assert res.status == trs.TRS_OK
    assert _rel(x.cpu().numpy(), np.linalg.solve(Ao.to_dense(), s.rhs)) <= 1e-10


def test_ilu1_adjoint(trs, oracle, synth):
    """The adjoint solve with block ILU(1) in the CPR built on A^T."""
    s = _sys(synth, 10, 8, 6, 4, seed=31, n_pairs=2)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A, ilu_fill=1)
    x, _ = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-11)
    g = oracle.well_cell_indicator(s)
    AT = ds.A.transpose()
    MT = trs.CPR(AT, ilu_fill=1, decoupling="none")
    lam, dA, res = trs.solve_adjoint(ds.A, AT, MT, torch.from_numpy(g).cuda(), x, want_dA=True, rtol=1e-11)
    assert res.status == trs.TRS_OK
    xo = oracle.fgmres(Ao, oracle.CPR(Ao), s.rhs, rtol=1e-11).x
    lamo, dAo, _ = oracle.adjoint(Ao, g, xo, rtol=1e-11)
    assert _rel(lam.cpu().numpy(), lamo) <= 1e-8
    assert _rel(dA.cpu().numpy().reshape(dAo.shape), dAo) <= 1e-8
