"""Jacobian of the thermal model on the GPU (trs_thermal_assemble: dual-number
derivatives in CUDA) against the oracle's (oracle/trs_thermal.c: the same
residual, differentiated by complex step), and the solver on it.

Both sides differentiate the same residual exactly up to rounding, by
different methods and with different transcendental-function libraries, so
each Jacobian entry agrees within 1e-12 of its row's largest entry and each
residual equation within 1e-12 of that equation's largest value.  The
pattern is the synthetic assembly's.  Then CPR-FGMRES solves J du = -R, and
Newton's method with GPU Jacobians and GPU solves converges quadratically.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

CASES = [
    dict(nx=5, ny=4, nz=4, seed=11, n_pairs=1),
    dict(nx=9, ny=7, nz=6, seed=12, n_pairs=2, sigma=1.5, kvkh=0.1),
    dict(nx=33, ny=17, nz=9, seed=13, n_pairs=3, gravity=0.0),     # ragged against 128-row blocks
    dict(nx=12, ny=10, nz=8, seed=14, n_pairs=0),                  # no wells
    dict(nx=1, ny=1, nz=3, seed=15, n_pairs=0),
]


def _cid(c):
    return f"{c['nx']}x{c['ny']}x{c['nz']}_w{c.get('n_pairs', 1)}" + ("_nog" if c.get("gravity") == 0.0 else "")


@pytest.fixture(scope="module")
def trs():
    from paper_1812_03952_gb300 import build as B
    B.build()
    from paper_1812_03952_gb300 import trs as T
    T.load()
    return T


# (p kPa, T C) of compressed water where the Redlich-Kwong cubic has one real
# root below a positive local minimum (Newton's method from above the roots
# cycles there)
COMPRESSED = ((1915.35, 12.43), (3000.0, 64.0), (3000.0, 69.0), (3800.0, 88.0), (4700.0, 129.0),
              (5800.0, 148.0))


def _make(synth, case, mode="chamber"):
    c = dict(case)
    gravity = c.pop("gravity", 9.80665)
    seed = c.pop("seed")
    nx, ny, nz = c.pop("nx"), c.pop("ny"), c.pop("nz")
    s = synth.small_system(nx, ny, nz, 4, seed=seed, **c)
    t = synth.thermal_state(s, seed + 100, gravity=gravity)
    u = t.u.reshape(-1, 4)
    if mode == "all_gas":
        u[:s.n_cells, 1] = 0.52
        u[:s.n_cells, 2] = 0.21
        u[:s.n_cells, 3] = 195.0
        t.gas[:] = 1
    elif mode == "uniform":
        # every cell in the first cell's state: each horizontal face (each face
        # without gravity) has zero potential differences, so each side takes
        # itself as upstream
        u[:s.n_cells] = u[0]
        t.gas[:s.n_cells] = t.gas[0]
    elif mode == "compressed":
        pt = np.array(COMPRESSED)[np.arange(s.n_cells) % len(COMPRESSED)]
        u[:s.n_cells, 0] = pt[:, 0]
        u[:s.n_cells, 2] = 0.0
        u[:s.n_cells, 3] = pt[:, 1]
        t.gas[:s.n_cells] = 0
    return s, t


def _compare(J, R, Jo, Ro, rows=None):
    """J (GPU values, canonical order) against the oracle's Jo entry by entry,
    relative to the largest entry of each scalar row; R against Ro per
    equation, relative to that equation's largest value.  rows: compare only
    these block rows."""
    b = 4
    brow = Jo.row_of_block()
    sel = np.ones(len(brow), bool) if rows is None else np.isin(brow, rows)
    Jv, Jg, rr = Jo.val[sel], J[sel], brow[sel]
    scale = np.zeros((Jo.n, b))
    np.maximum.at(scale, rr, np.abs(Jv).max(axis=2))
    err = np.abs(Jg - Jv).max(axis=2) / np.maximum(scale[rr], 1e-300)
    if err.max() > 1e-12:
        k, e = np.unravel_index(np.argmax(err), err.shape)
        blk = np.flatnonzero(sel)[k]
        raise AssertionError(f"relative error {err.max():.3e} in block row {rr[k]}, column {Jo.col[blk]}, "
                             f"scalar row {e}: GPU {Jg[k][e].tolist()} oracle {Jv[k][e].tolist()}")
    keep = np.arange(Jo.n) if rows is None else np.asarray(rows)
    Rr, Ror = R.reshape(-1, b)[keep], Ro.reshape(-1, b)[keep]
    for e in range(b):
        mag = max(np.abs(Ror[:, e]).max(), 1e-300)
        assert np.abs(Rr[:, e] - Ror[:, e]).max() <= 1e-12 * mag, (e, float(np.abs(Rr[:, e] - Ror[:, e]).max() / mag))


@pytest.mark.parametrize("mode", ["chamber", "all_gas", "compressed", "uniform"])
@pytest.mark.parametrize("case", CASES, ids=_cid)
def test_thermal_jacobian_matches_oracle(trs, oracle, synth, case, mode):
    s, t = _make(synth, case, mode)
    th = oracle.Thermal(s, t, synth.SWT, synth.SLT)
    Jo, Ro = th.jacobian(), th.residual()
    ts = trs.ThermalSystem(s, t, synth.SWT, synth.SLT)
    for _ in range(2):   # the second call reuses the property scratch and overwrites every entry
        R = ts.assemble().cpu().numpy()
        rp, col = ts.A.pattern()
        np.testing.assert_array_equal(rp, Jo.rp)
        np.testing.assert_array_equal(col, Jo.col)
        _compare(ts.A.values(), R, Jo, Ro)


def test_thermal_solve_with_cpr(trs, oracle, synth):
    """CPR-FGMRES on J du = -R in both precisions: the true residual, checked
    on the host with the oracle's own Jacobian, meets rtol."""
    s, t = _make(synth, dict(nx=20, ny=16, nz=10, seed=21, n_pairs=2, sigma=1.5, kvkh=0.1))
    th = oracle.Thermal(s, t, synth.SWT, synth.SLT)
    Jo, Ro = th.jacobian(), th.residual()
    ts = trs.ThermalSystem(s, t, synth.SWT, synth.SLT)
    R = ts.assemble()
    for precision in ("fp64", "fp32"):
        M = trs.CPR(ts.A, precision=precision)
        du, res = trs.fgmres_solve(ts.A, M, -R, rtol=1e-8)
        assert res.status == trs.TRS_OK, res
        d = du.cpu().numpy()
        rel = np.linalg.norm(oracle.spmv(Jo, d) + Ro) / np.linalg.norm(Ro)
        assert rel <= 1.01e-8 * (1 + 1e-3), rel


def test_thermal_newton_on_gpu(trs, oracle, synth):
    """Newton's method with GPU Jacobians and GPU CPR-FGMRES solves (rtol
    1e-12) on R(u) - R(u*) = 0 from a perturbed start: the error falls
    quadratically to the solver's tolerance."""
    s, t = _make(synth, dict(nx=8, ny=6, nz=6, seed=31, n_pairs=1))
    ts = trs.ThermalSystem(s, t, synth.SWT, synth.SLT)
    ustar = ts.u.clone()
    R0 = ts.assemble(ustar).clone()
    rng = np.random.default_rng(5)
    n_c = s.n_cells
    du = np.zeros((s.n_rows, 4))
    du[:n_c, 0] = rng.normal(0.0, 0.05, n_c)
    du[:n_c, 1] = rng.normal(0.0, 5e-5, n_c)
    du[:n_c, 2] = np.where(t.gas == 1, rng.normal(0.0, 5e-5, n_c), 0.0)
    du[:n_c, 3] = rng.normal(0.0, 0.005, n_c)
    du[n_c:, 0] = rng.normal(0.0, 0.05, s.n_wells)
    u = ustar + torch.from_numpy(du.reshape(-1)).cuda()
    errs = []
    M = None
    for it in range(6):
        errs.append(float(torch.linalg.norm(u - ustar) / torch.linalg.norm(ustar)))
        if errs[-1] <= 1e-13:
            break
        R = ts.assemble(u) - R0
        if M is None:
            M = trs.CPR(ts.A, precision="fp64")
        else:
            M.update(ts.A, reuse_amg=False)
        step, res = trs.fgmres_solve(ts.A, M, -R, rtol=1e-13)
        assert res.status == trs.TRS_OK
        u = u + step
    e = np.array(errs)
    assert e[-1] <= 1e-12, e
    ks = [k for k in range(len(e) - 1) if e[k + 1] > 1e-12]
    assert ks and all(e[k + 1] <= 1e4 * e[k] ** 2 for k in ks), e


def test_thermal_rejections(trs, synth):
    s = synth.small_system(4, 3, 2, 3, seed=3, n_pairs=0)
    with pytest.raises(ValueError):
        trs.ThermalSystem(s, None, synth.SWT, synth.SLT)
    s4 = synth.small_system(4, 3, 2, 4, seed=3, n_pairs=0)
    t = synth.thermal_state(s4, 7)
    bad = synth.SWT[::-1].copy()
    ts = trs.ThermalSystem(s4, t, bad, synth.SLT)
    with pytest.raises(trs.TrsError) as ei:
        ts.assemble()
    assert ei.value.code == trs.TRS_ERR_INVALID
