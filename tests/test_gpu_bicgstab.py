"""Parity of the CUDA BiCGSTAB (through the C ABI) with the oracle's.

BiCGSTAB is the Krylov method of the paper's runs (Sec. "Numerical
Studies").  The k-th iterate of the FP64 path equals the oracle's k-th
iterate up to summation order, so early iterates are compared directly
(the recurrences amplify rounding only mildly over a few steps); converged
solutions are compared as the FGMRES ones are: both sides reach
||r|| / ||b|| <= 1e-10 and agree to 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from test_gpu_parity import CASES, _case_id, _gpu_system, _rel, _sys  # noqa: E402


@pytest.fixture(scope="module")
def trs():
    from paper_1812_03952_gb300 import build as B
    B.build()
    from paper_1812_03952_gb300 import trs as T
    T.load()
    return T


def _true_relres(oracle, Ao, rhs, x):
    return np.linalg.norm(rhs - oracle.spmv(Ao, x)) / np.linalg.norm(rhs)


@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_bicgstab_fp64_matches_oracle(trs, oracle, synth, case):
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A, precision="fp64")
    x, res = trs.bicgstab_solve(ds.A, M, ds.rhs, rtol=1e-10)
    ref = oracle.bicgstab(Ao, oracle.CPR(Ao), s.rhs, rtol=1e-10)
    assert res.status == trs.TRS_OK and res.stats["converged"]
    assert ref.converged and ref.true_relres <= 1e-10
    xg = x.cpu().numpy()
    assert res.stats["true_relres"] <= 1e-10
    assert _true_relres(oracle, Ao, s.rhs, xg) <= 1.01e-10
    assert _rel(xg, ref.x) <= 1e-8
    assert abs(res.stats["iters"] - ref.iters) <= max(2, ref.iters // 10)


@pytest.mark.parametrize("case", CASES[::2], ids=_case_id)
def test_bicgstab_early_iterates_match_oracle(trs, oracle, synth, case):
    """x_k after k = 1, 2, 3 iterations (no convergence): same recurrences."""
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A, precision="fp64")
    Mo = oracle.CPR(Ao)
    for k in (1, 2, 3):
        ref = oracle.bicgstab(Ao, Mo, s.rhs, rtol=1e-15, maxit=k)
        x, res = trs.bicgstab_solve(ds.A, M, ds.rhs, rtol=1e-15, maxit=k)
        if ref.converged:
            break
        assert res.status == trs.TRS_ERR_NOT_CONVERGED and res.stats["iters"] == k
        assert _rel(x.cpu().numpy(), ref.x) <= 1e-10
        np.testing.assert_allclose(res.stats["true_relres"], ref.true_relres, rtol=1e-6, atol=1e-13)


@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_bicgstab_fp32_preconditioner(trs, oracle, synth, case):
    s = _sys(synth, **case)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A, precision="fp32")
    for rtol in (1e-6, 1e-10):
        x, res = trs.bicgstab_solve(ds.A, M, ds.rhs, rtol=rtol)
        assert res.status == trs.TRS_OK
        assert _true_relres(oracle, Ao, s.rhs, x.cpu().numpy()) <= rtol * 1.01


def test_bicgstab_host_buffers(trs, synth):
    s = _sys(synth, 9, 7, 5, 4, seed=21)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A)
    x, res = trs.bicgstab_solve_host(ds.A, M, s.rhs, rtol=1e-10)
    xd, _ = trs.bicgstab_solve(ds.A, M, ds.rhs, rtol=1e-10)
    assert res.status == trs.TRS_OK
    np.testing.assert_array_equal(x, xd.cpu().numpy())


def test_bicgstab_adjoint(trs, oracle, synth):
    s = _sys(synth, 10, 8, 6, 4, seed=31, n_pairs=2)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A)
    x, _ = trs.bicgstab_solve(ds.A, M, ds.rhs, rtol=1e-11)
    g = oracle.well_cell_indicator(s)
    AT = ds.A.transpose()
    MT = trs.CPR(AT)
    lam, dA, res = trs.solve_adjoint(ds.A, AT, MT, torch.from_numpy(g).cuda(), x, want_dA=True,
                                     rtol=1e-11, method="bicgstab")
    assert res.status == trs.TRS_OK
    xo = oracle.fgmres(Ao, oracle.CPR(Ao), s.rhs, rtol=1e-11).x
    lamo, dAo, _ = oracle.adjoint(Ao, g, xo, rtol=1e-11)
    assert _rel(lam.cpu().numpy(), lamo) <= 1e-8
    assert _rel(dA.cpu().numpy().reshape(dAo.shape), dAo) <= 1e-8


def test_bicgstab_edge_cases(trs, oracle, synth):
    # no flux: M = A^-1, so the first half step already meets the tolerance
    s = _sys(synth, 5, 4, 3, 4, seed=41, n_pairs=0)
    s.k[:] = 0.0
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A)
    _, res = trs.bicgstab_solve(ds.A, M, ds.rhs, rtol=1e-12)
    assert res.status == trs.TRS_OK and res.stats["iters"] == 1
    # zero right-hand side
    x, res = trs.bicgstab_solve(ds.A, M, torch.zeros_like(ds.rhs), rtol=1e-8)
    assert res.status == trs.TRS_OK and res.stats["iters"] == 0 and float(x.abs().max()) == 0.0
    # degenerate grids, against a dense solve
    for dims in [(1, 1, 1), (2, 1, 1), (1, 1, 7), (3, 1, 2)]:
        s = synth.small_system(*dims, b=3, seed=42, n_pairs=0)
        ds = _gpu_system(trs, s)
        x, res = trs.bicgstab_solve(ds.A, trs.CPR(ds.A), ds.rhs, rtol=1e-12)
        Ao = oracle.assemble(s)
        assert res.status == trs.TRS_OK
        assert _rel(x.cpu().numpy(), np.linalg.solve(Ao.to_dense(), s.rhs)) <= 1e-10
    # iteration limit and NaN input
    s = _sys(synth, 4, 4, 3, 4, seed=44)
    ds = _gpu_system(trs, s)
    M = trs.CPR(ds.A)
    x, res = trs.bicgstab_solve(ds.A, M, ds.rhs, rtol=1e-15, maxit=1)
    assert res.status == trs.TRS_ERR_NOT_CONVERGED and res.stats["iters"] == 1
    bad = ds.rhs.clone()
    bad[5] = float("inf")
    with pytest.raises(trs.TrsError) as ei:
        trs.bicgstab_solve(ds.A, M, bad)
    assert ei.value.code == trs.TRS_ERR_NAN


def test_bicgstab_warm_start_and_determinism(trs, oracle, synth):
    s = _sys(synth, 12, 10, 6, 4, seed=45, n_pairs=2)
    ds = _gpu_system(trs, s)
    Ao = oracle.assemble(s)
    M = trs.CPR(ds.A, precision="fp32")
    x1, r1 = trs.bicgstab_solve(ds.A, M, ds.rhs, rtol=1e-9)
    x2, _ = trs.bicgstab_solve(ds.A, M, ds.rhs, rtol=1e-9)
    assert torch.equal(x1, x2)
    # from the converged x the solve ends at once; from a perturbed x it converges again
    x3, r3 = trs.bicgstab_solve(ds.A, M, ds.rhs, x=x1.clone(), rtol=1e-9, use_x0=True)
    assert r3.stats["iters"] == 0 and torch.equal(x3, x1)
    x4, r4 = trs.bicgstab_solve(ds.A, M, ds.rhs, x=x1 * 1.01, rtol=1e-9, use_x0=True)
    assert r4.status == trs.TRS_OK
    assert _true_relres(oracle, Ao, s.rhs, x4.cpu().numpy()) <= 1.01e-9
