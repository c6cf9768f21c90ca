"""Adjoint gradients of the autograd wrapper against central finite
differences along seeded directions, computed on the GPU with the
difference-solve form L(t+hd) - L(t-hd) = g^T A+^-1 ((A- - A+) x-), which
needs no 1e-14-accurate solves; and against the oracle's FP64 adjoint."""
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


def _fd_difference(trs, sysm, theta_m, theta_p, g, precision, rtol=1e-12):
    """L(theta_p) - L(theta_m) with the difference-solve form."""
    minus = trs.DeviceSystem(sysm)
    plus = trs.DeviceSystem(sysm)
    Am = minus.assemble(theta_m, perm_is_log=True)
    Ap = plus.assemble(theta_p, perm_is_log=True)
    xm, r1 = trs.fgmres_solve(Am, trs.CPR(Am, precision=precision), minus.rhs, rtol=rtol)
    rhs = Am.spmv(xm)
    Ap.spmv(xm, rhs, alpha=-1.0, beta=1.0)
    delta, r2 = trs.fgmres_solve(Ap, trs.CPR(Ap, precision=precision), rhs, rtol=rtol)
    assert r1.status == trs.TRS_OK and r2.status == trs.TRS_OK
    return float(torch.dot(g, delta))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,ndir", [((10, 8, 6), 8), ((64, 64, 32), 64)], ids=["small", "64x64x32"])
def test_autograd_gradient_vs_finite_differences(trs, oracle, synth, precision, shape, ndir):
    from paper_1812_03952_gb300 import autograd as AG
    if shape == (64, 64, 32):
        sysm = synth.config(3)
    else:
        sysm = synth.small_system(*shape, b=4, seed=51, n_pairs=2)
    theta = torch.from_numpy(np.log(sysm.k)).cuda().requires_grad_(True)
    rhs = torch.from_numpy(sysm.rhs).cuda().requires_grad_(True)
    # both the gradient and the differences are accurate to about cond(A) * rtol
    sctx = AG.SolveContext(sysm, precision=precision, rtol=1e-12)
    x = AG.solve(theta, rhs, sctx)
    g = torch.from_numpy(oracle.well_cell_indicator(sysm)).cuda()
    loss = torch.dot(g, x)
    loss.backward()
    assert sctx.last_forward.status == trs.TRS_OK and sctx.last_adjoint.status == trs.TRS_OK
    grad = theta.grad.detach()
    h = 1e-6
    dirs = synth.seeded_directions(sysm.n_cells, ndir, 4321)
    fd, an = [], []
    for d in dirs:
        dt = torch.from_numpy(d).cuda()
        th_p, th_m = theta.detach() + h * dt, theta.detach() - h * dt
        fd.append(_fd_difference(trs, sysm, th_m, th_p, g, precision) / (2 * h))
        # the perturbation actually applied (theta +- h d rounded to FP64)
        an.append(float(torch.dot(grad, th_p - th_m)) / (2 * h))
    fd, an = np.array(fd), np.array(an)
    # relative error of the vector of directional derivatives (a single
    # direction whose derivative nearly cancels would otherwise dominate)
    assert np.linalg.norm(fd - an) / np.linalg.norm(an) <= 1e-5
    assert np.max(np.abs(fd - an)) <= 1e-5 * np.max(np.abs(an))
    # dL/db = lambda: L is linear in b
    e = torch.randn_like(rhs)
    A = sctx.assemble(theta.detach())
    M = trs.CPR(A, precision="fp64")
    xe, _ = trs.fgmres_solve(A, M, e.detach(), rtol=1e-12)
    np.testing.assert_allclose(float(torch.dot(g, xe)), float(torch.dot(rhs.grad, e)), rtol=1e-8)


def test_gradient_matches_oracle_adjoint(trs, oracle, synth):
    from paper_1812_03952_gb300 import autograd as AG
    sysm = synth.small_system(12, 9, 5, 4, seed=52, n_pairs=2)
    theta = torch.from_numpy(np.log(sysm.k)).cuda().requires_grad_(True)
    rhs = torch.from_numpy(sysm.rhs).cuda()
    sctx = AG.SolveContext(sysm, precision="fp64", rtol=1e-10)
    x = AG.solve(theta, rhs, sctx)
    g = oracle.well_cell_indicator(sysm)
    torch.dot(torch.from_numpy(g).cuda(), x).backward()
    Ao = oracle.assemble(sysm)
    xo = oracle.fgmres(Ao, oracle.CPR(Ao), sysm.rhs, rtol=1e-10).x
    lam, dA, _ = oracle.adjoint(Ao, g, xo, rtol=1e-10)
    dth = oracle.chain_theta(sysm, Ao, dA)
    got = theta.grad.cpu().numpy()
    assert np.linalg.norm(got - dth) / np.linalg.norm(dth) <= 1e-8
