"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer and setup objects whose values decide integers are compared bit for
bit (assembly, decoupling, pressure matrices of every level, aggregates,
colours).  Floating-point results are compared within tolerances derived
from the arithmetic: a few ulp times the condition of the summation for
products, 1e-12 for one preconditioner application (same operations,
different summation order), and ||x - x_oracle|| / ||x_oracle|| <= 1e-8 for
solves where both sides reach ||r|| / ||b|| <= 1e-10.
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


def _sys(synth, nx, ny, nz, b, seed, **kw):
    return synth.small_system(nx, ny, nz, b, seed=seed, **kw)


CASES = [
    dict(nx=6, ny=5, nz=3, b=4, seed=3),
    dict(nx=6, ny=5, nz=3, b=1, seed=4, n_pairs=0),
    dict(nx=5, ny=4, nz=3, b=2, seed=5),
    dict(nx=7, ny=3, nz=4, b=3, seed=6),
    dict(nx=9, ny=7, nz=5, b=5, seed=7, n_pairs=2),
    dict(nx=33, ny=17, nz=9, b=4, seed=8, n_pairs=3, sigma=1.5, kvkh=0.1),   # ragged vs 256-row tiles
    dict(nx=20, ny=18, nz=10, b=4, seed=9, n_pairs=2, sigma=2.0, shale_frac=0.1),
]


def _case_id(c):
    return f"{c['nx']}x{c['ny']}x{c['nz']}_b{c['b']}"


def _gpu_system(trs, sysm):
    ds = trs.DeviceSystem(sysm)
    ds.assemble()
    return ds


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------ assembly
@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_assembly_bit_exact(trs, oracle, synth, case):
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    rp, col = ds.A.pattern()
    np.testing.assert_array_equal(rp, Ao.rp)
    np.testing.assert_array_equal(col, Ao.col)
    np.testing.assert_array_equal(ds.A.values(), Ao.val)


@pytest.mark.parametrize("grid", [True, False], ids=["structured", "general"])
@pytest.mark.parametrize("case", CASES[:5], ids=_case_id)
def test_spmv_parity(trs, oracle, synth, case, grid):
    s = _sys(synth, **case)
    Ao = oracle.assemble(s)
    A = trs.Matrix.from_bsr(Ao.rp, Ao.col, Ao.val, s.b, (s.nx, s.ny, s.nz) if grid else None)
    np.testing.assert_array_equal(A.values(), Ao.val)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(Ao.n * Ao.b)
    y0 = rng.standard_normal(Ao.n * Ao.b)
    xt = torch.from_numpy(x).cuda()
    for transpose in (False, True):
        yt = torch.from_numpy(y0.copy()).cuda()
        A.spmv(xt, yt, alpha=1.5, beta=-0.5, transpose=transpose)
        ref = oracle.spmv(Ao, x, alpha=1.5, beta=-0.5, y=y0, transpose=transpose)
        absA = oracle.BSR(Ao.n, Ao.b, Ao.rp, Ao.col, np.abs(Ao.val))
        bound = oracle.spmv(absA, np.abs(x), 1.5, 0.5, np.abs(y0), transpose=transpose)
        err = np.abs(yt.cpu().numpy() - ref)
        assert np.all(err <= 16 * 2.2e-16 * bound + 1e-300)


@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_transpose_matrix_exact(trs, oracle, synth, case):
    """A^T (cell slots from the opposite slot of the neighbour, well blocks
    from the tail) is A's blocks transposed, bit for bit; refreshed in place
    after A's values change, it is the new A's transpose."""
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    AT = ds.A.transpose()
    ATo = oracle.transpose(oracle.assemble(s))
    rp, col = AT.pattern()
    np.testing.assert_array_equal(rp, ATo.rp)
    np.testing.assert_array_equal(col, ATo.col)
    np.testing.assert_array_equal(AT.values(), ATo.val)
    s2 = _sys(synth, **dict(case, seed=case["seed"] + 50))
    ds2 = trs.DeviceSystem(s2)
    ds.A.assemble(ds2.k, ds2.M, ds2.acc, ds2.wi, ds2.lam, s2.kvkh, s2.c_t, False)
    ds.A.transpose(into=AT)
    np.testing.assert_array_equal(AT.values(), oracle.transpose(oracle.assemble(s2)).val)


def test_transpose_unstructured_exact(trs, oracle):
    """A matrix with no grid (a structurally symmetric random pattern, values
    unsymmetric): every block goes through the tail path."""
    rng = np.random.default_rng(12)
    n, b = 300, 3
    pairs = {(i, i) for i in range(n)}
    for i in range(n):
        for j in rng.choice(n, 3, replace=False):
            pairs |= {(i, int(j)), (int(j), i)}
    rows = [np.array(sorted(j for (r, j) in pairs if r == i)) for i in range(n)]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    val = rng.standard_normal((rp[-1], b, b))
    A = trs.Matrix.from_bsr(rp, col, val, b)
    AT = A.transpose()
    ATo = oracle.transpose(oracle.BSR(n, b, rp, col, val))
    trp, tcol = AT.pattern()
    np.testing.assert_array_equal(trp, ATo.rp)
    np.testing.assert_array_equal(tcol, ATo.col)
    np.testing.assert_array_equal(AT.values(), ATo.val)


# --------------------------------------------------------------------- setup
@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_setup_bit_exact(trs, oracle, synth, case):
    """Decoupled blocks, D^-1, every level's pressure operator, aggregates
    and colours are identical to the oracle's."""
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    kw = dict(coarse_max=40)
    M = trs.CPR(ds.A, **kw)
    Mo = oracle.CPR(Ao, **kw)
    vt, dinv = M.decoupled(Ao.nnzb)
    vto, dinvo = Mo.decoupled()
    np.testing.assert_array_equal(dinv, dinvo)
    np.testing.assert_array_equal(vt, vto)
    info = M.info()
    amg = Mo.amg
    assert info["n_levels"] == amg.n_levels
    assert info["level_rows"] == amg.sizes()
    for l in range(amg.n_levels):
        rp, col, val = M.level(l)
        rpo, colo, valo = amg.level(l)
        np.testing.assert_array_equal(rp, rpo)
        np.testing.assert_array_equal(col, colo)
        np.testing.assert_array_equal(val, valo)
        np.testing.assert_array_equal(M.aggregates(l), amg.agg(l))
        assert info["level_lambda"][l] == amg.lam(l)
    np.testing.assert_array_equal(M.colours(), Mo.colours())
    assert info["n_colours"] == Mo.info()[1]


# ------------------------------------------------------------ applications
@pytest.mark.parametrize("coarse_max", [40, 400], ids=["smem-coarsest", "multiblock-coarsest"])
@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_vcycle_and_cpr_apply_parity(trs, oracle, synth, case, coarse_max):
    """One V-cycle and one CPR application against the oracle; coarse_max 400
    leaves a coarsest level above 64 rows (multi-launch Gauss-Jordan inverse)."""
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A, coarse_max=coarse_max)
    Mo = oracle.CPR(Ao, coarse_max=coarse_max)
    rng = np.random.default_rng(2)
    r = rng.standard_normal(Ao.n)
    e = M.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    assert _rel(e, Mo.amg.vcycle(r)) <= 1e-11
    v = rng.standard_normal(Ao.n * Ao.b)
    z = M.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert _rel(z, Mo.apply(v)) <= 1e-11


@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_fgmres_fp64_matches_oracle(trs, oracle, synth, case):
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A, precision="fp64")
    x, res = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-10)
    ref = oracle.fgmres(Ao, oracle.CPR(Ao), s.rhs, rtol=1e-10)
    assert res.status == trs.TRS_OK and res.stats["converged"]
    assert res.stats["true_relres"] <= 1e-10 and ref.true_relres <= 1e-10
    xg = x.cpu().numpy()
    assert _rel(xg, ref.x) <= 1e-8
    # the true FP64 residual, recomputed on the host
    assert np.linalg.norm(s.rhs - oracle.spmv(Ao, xg)) / np.linalg.norm(s.rhs) <= 1.01e-10
    assert abs(res.stats["iters"] - ref.iters) <= max(2, ref.iters // 10)


@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_fgmres_fp32_preconditioner(trs, oracle, synth, case):
    """FP32 CPR inside FP64 FGMRES reaches a true FP64 residual of 1e-6
    (and 1e-10); the error against the FP64 oracle solution is bounded by
    cond(A) * rtol (checked here against 1e-6 * ||A^-1|| * ||A|| estimate)."""
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A, precision="fp32")
    ref = oracle.fgmres(Ao, oracle.CPR(Ao), s.rhs, rtol=1e-12)
    for rtol in (1e-6, 1e-10):
        x, res = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=rtol)
        xg = x.cpu().numpy()
        tr = np.linalg.norm(s.rhs - oracle.spmv(Ao, xg)) / np.linalg.norm(s.rhs)
        assert res.status == trs.TRS_OK and tr <= rtol * 1.01
        if Ao.n * Ao.b <= 3000:
            cond = np.linalg.cond(Ao.to_dense())
            assert _rel(xg, ref.x) <= cond * rtol * 1.01


def test_solve_host_buffers(trs, oracle, synth):
    s = _sys(synth, 9, 7, 5, 4, seed=21)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A)
    x, res = trs.fgmres_solve_host(ds.A, M, s.rhs, rtol=1e-10)
    xd, _ = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-10)
    np.testing.assert_array_equal(x, xd.cpu().numpy())
    # a second call reuses the handle's device copies; pinned CPU tensors work too
    hb = torch.from_numpy(s.rhs.copy()).pin_memory()
    hx = torch.full((ds.A.N,), float("nan"), dtype=torch.float64).pin_memory()
    x2, _ = trs.fgmres_solve_host(ds.A, M, hb, rtol=1e-10, x=hx)
    assert x2 is hx
    np.testing.assert_array_equal(hx.numpy(), x)


def test_assemble_host_buffers(trs, oracle, synth):
    """trs_bsr_assemble_host gives the bits of the device-input assembly."""
    s = _sys(synth, 9, 7, 5, 4, seed=22, n_pairs=2)
    ds = _gpu_system(trs, s)
    ref = ds.A.values()
    A2 = trs.Matrix.synthetic_pattern(s.nx, s.ny, s.nz, s.b, s.n_wells, s.perf_well, s.perf_cell)
    for _ in range(2):   # the second call reuses the staging area
        A2.assemble_host(s.k, s.M.reshape(-1), s.acc.reshape(-1), s.wi, s.lam.reshape(-1), s.kvkh, s.c_t)
        np.testing.assert_array_equal(A2.values(), ref)
    np.testing.assert_array_equal(A2.values(), oracle.assemble(s).val)


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_parity_and_chain(trs, oracle, synth, prec):
    s = _sys(synth, 10, 8, 6, 4, seed=31, n_pairs=2)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A, precision=prec)
    x, _ = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-10)
    g = oracle.well_cell_indicator(s)
    AT = ds.A.transpose()
    MT = trs.CPR(AT, precision=prec)
    lam, dA, res = trs.solve_adjoint(ds.A, AT, MT, torch.from_numpy(g).cuda(), x, want_dA=True, rtol=1e-10)
    assert res.status == trs.TRS_OK
    xo = oracle.fgmres(Ao, oracle.CPR(Ao), s.rhs, rtol=1e-10).x
    lamo, dAo, _ = oracle.adjoint(Ao, g, xo, rtol=1e-10)
    lg = lam.cpu().numpy()
    assert _rel(lg, lamo) <= 1e-8
    assert np.linalg.norm(oracle.spmv(Ao, lg, transpose=True) - g) / np.linalg.norm(g) <= 1.01e-10
    dA_g = dA.cpu().numpy().reshape(dAo.shape)
    assert _rel(dA_g, dAo) <= 1e-8
    dth = trs.chain_theta(ds.A, ds.k, ds.M, lam, x, s.kvkh, s.c_t).cpu().numpy()
    dtho = oracle.chain_theta(s, Ao, dAo)
    assert _rel(dth, dtho) <= 1e-8


# ------------------------------------------------------------ edge cases
def test_no_flux_is_one_iteration(trs, synth):
    s = _sys(synth, 5, 4, 3, 4, seed=41, n_pairs=0)
    s.k[:] = 0.0
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A)
    _, res = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-12)
    assert res.status == trs.TRS_OK and res.stats["iters"] == 1


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 1), (1, 1, 7), (3, 1, 2)])
def test_degenerate_grids(trs, oracle, synth, dims):
    s = synth.small_system(*dims, b=3, seed=42, n_pairs=0)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A)
    x, res = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-12)
    Ao = oracle.assemble(s)
    xr = np.linalg.solve(Ao.to_dense(), s.rhs)
    assert res.status == trs.TRS_OK
    assert _rel(x.cpu().numpy(), xr) <= 1e-10


def test_zero_rhs(trs, synth):
    s = _sys(synth, 4, 4, 2, 4, seed=43)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A)
    x, res = trs.fgmres_solve(ds.A, M, torch.zeros_like(ds.rhs), rtol=1e-8)
    assert res.status == trs.TRS_OK and float(x.abs().max()) == 0.0


def test_error_statuses(trs, synth):
    s = _sys(synth, 4, 4, 3, 4, seed=44)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A)
    # iteration limit: status reported, stats filled, last iterate kept
    x, res = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-14, maxit=1)
    assert res.status == trs.TRS_ERR_NOT_CONVERGED and res.stats["iters"] == 1
    assert 0 < res.stats["true_relres"] < 1
    # NaN in the right-hand side
    bad = ds.rhs.clone()
    bad[3] = float("nan")
    with pytest.raises(trs.TrsError) as ei:
        trs.fgmres_solve(ds.A, M, bad)
    assert ei.value.code == trs.TRS_ERR_NAN
    # a singular diagonal block
    rp, col = ds.A.pattern()
    vals = ds.A.values().copy()
    diag = np.where(np.repeat(np.arange(len(rp) - 1), np.diff(rp)) == col)[0][0]
    vals[diag] = 0.0
    B = trs.Matrix.from_bsr(rp, col, vals, s.b, (s.nx, s.ny, s.nz))
    with pytest.raises(trs.TrsError) as ei:
        trs.CPR(B)
    assert ei.value.code == trs.TRS_ERR_SINGULAR_BLOCK
    # malformed BSR: rejected on the host before any upload
    col2 = col.copy()
    col2[[0, 1]] = col2[[1, 0]]
    with pytest.raises(trs.TrsError) as ei:
        trs.Matrix.from_bsr(rp, col2, vals, s.b)
    assert ei.value.code == trs.TRS_ERR_INVALID


def test_determinism(trs, synth):
    s = _sys(synth, 12, 10, 6, 4, seed=45, n_pairs=2)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A, precision="fp32")
    x1, _ = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-9)
    x2, _ = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-9)
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("method", ["fgmres", "bicgstab"])
def test_phase_timing(trs, synth, method):
    """opts.time_phases fills the per-phase device times without changing the
    result: the phases sum to at most the solve time, one operator SpMV per
    FGMRES step (two per BiCGSTAB iteration), and the bits of x are those of
    an untimed solve."""
    s = _sys(synth, 12, 10, 6, 4, seed=47, n_pairs=2)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A, precision="fp32")
    x0, r0 = trs.krylov_solve(method, ds.A, M, ds.rhs, rtol=1e-9)
    assert r0.stats["ms_precond"] == 0.0 and r0.stats["spmv_launches"] == 0
    x1, r1 = trs.krylov_solve(method, ds.A, M, ds.rhs, rtol=1e-9, time_phases=True)
    assert torch.equal(x0, x1)
    st = r1.stats
    assert st["spmv_launches"] == st["iters"] * (1 if method == "fgmres" else 2)
    for k in ("ms_precond", "ms_spmv", "ms_orth"):
        assert st[k] > 0.0
    assert st["ms_precond"] + st["ms_spmv"] + st["ms_orth"] <= st["ms_solve"] * 1.001


def test_update_reuse_amg(trs, oracle, synth):
    """Newton-like sequence: diagonal blocks rescaled, AMG hierarchy kept."""
    s = _sys(synth, 12, 10, 6, 4, seed=46, n_pairs=2)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A, precision="fp32")
    scales = synth.diagonal_scalings(ds.A.n, 2, 7)
    for step in range(2):
        ds.assemble()
        ds.A.scale_diagonal(torch.from_numpy(scales[step]).cuda())
        M.update(ds.A, reuse_amg=True)
        x, res = trs.fgmres_solve(ds.A, M, ds.rhs, rtol=1e-8)
        assert res.status == trs.TRS_OK
        Ao = oracle.assemble(s)
        rows = Ao.row_of_block()
        diag = rows == Ao.col
        Ao.val[diag] *= scales[step][rows[diag]][:, None, None]
        np.testing.assert_array_equal(ds.A.values(), Ao.val)
        xg = x.cpu().numpy()
        assert np.linalg.norm(s.rhs - oracle.spmv(Ao, xg)) / np.linalg.norm(s.rhs) <= 1.01e-8
        # the aggregates are kept; the values of every level follow the new matrix: level 0 is
        # the new pressure matrix and level 1 its Galerkin product over the kept aggregates
        # (FP64 preconditioner, so the decoupled values are the oracle's bit for bit)
        M64 = trs.CPR(ds.A, precision="fp64") if step == 0 else M64
        if step > 0:
            M64.update(ds.A, reuse_amg=True)
            vt, _ = oracle.decouple(Ao)
            ap = oracle.pressure_matrix(Ao, vt)
            rp0, col0, val0 = M64.level(0)
            np.testing.assert_array_equal(val0, ap)
            agg0 = M64.aggregates(0)
            n1 = M64.info()["level_rows"][1]
            crp, ccol, cval = oracle.galerkin(Ao.n, rp0, col0, val0, agg0, n1)
            rp1, col1, val1 = M64.level(1)
            np.testing.assert_array_equal(rp1, crp)
            np.testing.assert_array_equal(col1, ccol)
            np.testing.assert_array_equal(val1, cval)


def test_stream_order_with_caller_kernels(trs, synth):
    """The library's kernels start with a programmatic-dependent-launch wait:
    a caller's kernel queued just before a call on the same stream (here a
    torch scaling of b and of x0) must be complete before the library reads
    its output, and a caller's kernel queued just after must see the result."""
    s = _sys(synth, 12, 10, 6, 4, seed=51, n_pairs=2)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A, precision="fp64")
    x_ref, _ = trs.fgmres_solve(ds.A, M, ds.rhs * 3.0, x=torch.zeros_like(ds.rhs), rtol=1e-10, use_x0=True)
    for _ in range(3):
        b = ds.rhs.clone()
        b.mul_(3.0)                                   # queued right before the solve
        x = torch.full_like(b, 7.0)
        x.mul_(0.0)                                   # x0 = 0, written by a caller kernel
        x, res = trs.fgmres_solve(ds.A, M, b, x=x, rtol=1e-10, use_x0=True)
        y = x * 2.0                                   # queued right after
        assert res.status == trs.TRS_OK
        assert torch.equal(x, x_ref)
        assert torch.equal(y, x_ref * 2.0)


@pytest.mark.parametrize("case", [CASES[0], CASES[4]], ids=_case_id)
def test_gridless_matrix_solve(trs, oracle, synth, case):
    """A matrix created without grid dimensions (a user's Jacobian in plain
    BSR): every row goes through the tail paths (decoupling, pressure
    operator, colouring and ILU(0) as long rows, SpMV).  CPR-FGMRES in FP64
    matches the oracle's solve of the same BSR; the FP32 form meets rtol on
    the host; both agree with the structured matrix's solves."""
    s = _sys(synth, **case)
    Ao = oracle.assemble(s)
    A = trs.Matrix.from_bsr(Ao.rp, Ao.col, Ao.val, s.b, None)
    rhs = torch.from_numpy(s.rhs).cuda()
    M = trs.CPR(A, precision="fp64")
    x, res = trs.fgmres_solve(A, M, rhs, rtol=1e-10)
    ref = oracle.fgmres(Ao, oracle.CPR(Ao), s.rhs, rtol=1e-10)
    assert res.status == trs.TRS_OK and ref.converged
    xg = x.cpu().numpy()
    assert _rel(xg, ref.x) <= 1e-8
    assert abs(res.stats["iters"] - ref.iters) <= max(2, ref.iters // 10)
    np.testing.assert_array_equal(M.colours(), oracle.CPR(Ao).colours())
    M32 = trs.CPR(A, precision="fp32")
    x32, res32 = trs.fgmres_solve(A, M32, rhs, rtol=1e-6)
    assert res32.status == trs.TRS_OK
    assert np.linalg.norm(s.rhs - oracle.spmv(Ao, x32.cpu().numpy())) / np.linalg.norm(s.rhs) <= 1e-6
    ds = _gpu_system(trs, s)
    xs, _ = trs.fgmres_solve(ds.A, trs.CPR(ds.A, precision="fp64"), ds.rhs, rtol=1e-10)
    assert _rel(xg, xs.cpu().numpy()) <= 1e-8
