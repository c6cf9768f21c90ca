"""Checks at the full benchmark size: 128x128x64 cells, b = 4, 8 wells
(4.19M unknowns), in the configuration the benchmark times (FP32 CPR inside
FP64 Krylov, rtol 1e-6, default CPR options).

The oracle still finishes the pieces that decide integers at this size
(assembly 0.2 s, CPR setup 2 s, one application 1 s), so those are compared
whole: assembled values, decoupled blocks and D^-1, every aggregate, every
colour, bit for bit.  The solves are checked by a property that holds at any
size: the true FP64 residual of the returned x, recomputed by the oracle on
the host, meets rtol.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def trs():
    from paper_1812_03952_gb300 import build as B
    B.build()
    from paper_1812_03952_gb300 import trs as T
    T.load()
    return T


@pytest.fixture(scope="module")
def full(trs, oracle, synth):
    sysm = synth.config(1)
    ds = trs.DeviceSystem(sysm)
    A = ds.assemble()
    Ao = oracle.assemble(sysm)
    return sysm, ds, A, Ao


def _relres(oracle, Ao, rhs, x):
    return np.linalg.norm(rhs - oracle.spmv(Ao, x)) / np.linalg.norm(rhs)


def test_full_size_assembly_and_setup_bit_exact(trs, oracle, full):
    sysm, ds, A, Ao = full
    rp, col = A.pattern()
    np.testing.assert_array_equal(rp, Ao.rp)
    np.testing.assert_array_equal(col, Ao.col)
    np.testing.assert_array_equal(A.values(), Ao.val)
    Mo = oracle.CPR(Ao)
    for precision in ("fp64", "fp32"):
        M = trs.CPR(A, precision=precision)
        info = M.info()
        assert info["level_rows"] == Mo.amg.sizes()
        for l in range(Mo.amg.n_levels - 1):
            np.testing.assert_array_equal(M.aggregates(l), Mo.amg.agg(l))
        np.testing.assert_array_equal(M.colours(), Mo.colours())
        if precision == "fp64":
            vt, dinv = M.decoupled(Ao.nnzb)
            vto, dinvo = Mo.decoupled()
            np.testing.assert_array_equal(dinv, dinvo)
            np.testing.assert_array_equal(vt, vto)
            # one CPR application on a seeded vector, against the oracle's
            v = np.random.default_rng(7).standard_normal(Ao.n * Ao.b)
            z = M.apply(torch.from_numpy(v).cuda()).cpu().numpy()
            zo = Mo.apply(v)
            assert np.linalg.norm(z - zo) / np.linalg.norm(zo) <= 1e-11


@pytest.mark.parametrize("method", ["fgmres", "bicgstab"])
def test_full_size_solve_meets_tolerance(trs, oracle, full, method):
    sysm, ds, A, Ao = full
    M = trs.CPR(A, precision="fp32")
    x = torch.empty_like(ds.rhs)
    # the benchmark's step: refresh the values, rebuild CPR, solve
    ds.assemble()
    M.update(A, reuse_amg=False)
    x, res = trs.krylov_solve(method, A, M, ds.rhs, x, rtol=1e-6)
    assert res.status == trs.TRS_OK and res.stats["converged"]
    tr = _relres(oracle, Ao, sysm.rhs, x.cpu().numpy())
    assert tr <= 1.01e-6
    assert abs(tr - res.stats["true_relres"]) <= 1e-12


def test_full_size_ilu1(trs, oracle, full):
    """Block ILU(1) at the full size: the distance-2 colours bit for bit, one
    FP64 application against the oracle's, and the benchmark's FP32 solve to
    the true residual."""
    sysm, ds, A, Ao = full
    grid = (sysm.nx, sysm.ny, sysm.nz)
    Mo = oracle.CPR(Ao, ilu_fill=1, grid=grid)
    M = trs.CPR(A, precision="fp64", ilu_fill=1)
    np.testing.assert_array_equal(M.colours(), Mo.colours())
    v = np.random.default_rng(8).standard_normal(Ao.n * Ao.b)
    z = M.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    zo = Mo.apply(v)
    assert np.linalg.norm(z - zo) / np.linalg.norm(zo) <= 1e-11
    M32 = trs.CPR(A, precision="fp32", ilu_fill=1)
    x, res = trs.krylov_solve("fgmres", A, M32, ds.rhs, torch.empty_like(ds.rhs), rtol=1e-6)
    assert res.status == trs.TRS_OK
    assert _relres(oracle, Ao, sysm.rhs, x.cpu().numpy()) <= 1.01e-6


@pytest.mark.parametrize("decoupling", ["abf", "none", "frs", "frs+abf"])
def test_full_size_fp32_apply_matches_oracle(trs, oracle, full, decoupling):
    """The benchmark's FP32 CPR application (block ILU(0)) against the
    oracle's FP64 application, for every stage ordering, within the
    rounding count of test_gpu_fp32_apply."""
    from test_gpu_fp32_apply import fp32_apply_tolerance
    sysm, ds, A, Ao = full
    v = np.random.default_rng(9).standard_normal(Ao.n * Ao.b)
    vd = torch.from_numpy(v).cuda()
    for stages in ("fpf", "fp", "pf"):
        Mo = oracle.CPR(Ao, stages=stages, decoupling=decoupling)
        M = trs.CPR(A, precision="fp32", stages=stages, decoupling=decoupling)
        z = M.apply(vd).cpu().numpy()
        zo = Mo.apply(v)
        err = np.linalg.norm(z - zo) / np.linalg.norm(zo)
        tol = fp32_apply_tolerance(Ao, Mo, stages)
        print(f"full size FP32 apply {stages}/{decoupling}: rel err {err:.3e} (bound {tol:.3e})")
        assert 0.0 < err <= tol
        del M, Mo


def test_full_size_error_vs_oracle_solution(trs, oracle, full):
    """Solution error against the oracle's FP64 solution at the benchmark
    size.  Both FP64 paths run the same algorithm, so at rtol 1e-10 their
    solutions agree to 1e-8; the FP32-preconditioner solve at the
    benchmark's rtol 1e-6 is as accurate as the FP64-preconditioner solve
    at the same tolerance, within a factor 10."""
    sysm, ds, A, Ao = full
    ref = oracle.fgmres(Ao, oracle.CPR(Ao), sysm.rhs, rtol=1e-10)
    assert ref.converged
    xs = ref.x
    err = lambda x: np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs)
    M64 = trs.CPR(A, precision="fp64")
    x64, r64 = trs.fgmres_solve(A, M64, ds.rhs, rtol=1e-10)
    assert r64.status == trs.TRS_OK
    e64_tight = err(x64)
    assert e64_tight <= 1e-8
    x64, r64 = trs.fgmres_solve(A, M64, ds.rhs, rtol=1e-6)
    e64 = err(x64)
    del M64
    M32 = trs.CPR(A, precision="fp32")
    x32, r32 = trs.fgmres_solve(A, M32, ds.rhs, rtol=1e-6)
    assert r32.status == trs.TRS_OK
    e32 = err(x32)
    print(f"full size error vs the oracle's x (rtol 1e-10, {ref.iters} its): FP64 at 1e-10 {e64_tight:.3e}, "
          f"FP64 at 1e-6 {e64:.3e} ({r64.stats['iters']} its), FP32 CPR at 1e-6 {e32:.3e} "
          f"({r32.stats['iters']} its)")
    assert e32 <= 10.0 * e64


def test_full_size_physics_jacobian_sampled_rows(trs, oracle, synth, full):
    """The physics Jacobian at the benchmark size (the thermal model on the
    128x128x64 grid and wells, steam chambers around the injectors): the GPU
    values against the oracle's complex-step Jacobian on 2,000 seeded cell rows
    plus every well row, 1e-12 of each scalar row's largest entry, and the
    residual on the same rows; then the benchmark's physics step (block ILU(1),
    FGMRES(60)) meets rtol on the true residual."""
    from test_gpu_thermal import _compare
    sysm, ds, A, Ao = full
    state = synth.thermal_state(sysm, synth.SEED_BASE + 77)
    ts = trs.ThermalSystem(sysm, state, synth.SWT, synth.SLT)
    R = ts.assemble()
    th = oracle.Thermal(sysm, state, synth.SWT, synth.SLT)
    rows = np.sort(np.random.default_rng(3).choice(sysm.n_cells, 2000, replace=False))
    # the perforated cells too (their rows carry the well columns)
    rows = np.union1d(rows, np.unique(sysm.perf_cell))
    Jo = th.jacobian(rows=rows, pattern=Ao)
    Ro = th.residual(rows=rows)
    well_rows = np.arange(sysm.n_cells, sysm.n_rows)
    _compare(ts.A.values(), R.cpu().numpy(), Jo, Ro, rows=np.concatenate([rows, well_rows]))
    M = trs.CPR(ts.A, precision="fp32", ilu_fill=1)
    d, res = trs.fgmres_solve(ts.A, M, R, rtol=1e-6, restart=60)
    assert res.status == trs.TRS_OK and res.stats["true_relres"] <= 1e-6
