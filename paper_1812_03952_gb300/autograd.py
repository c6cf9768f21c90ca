"""PyTorch autograd wrapper of the solve x = A(theta)^-1 b.

Forward: assembly of A from theta = ln k on the GPU, CPR setup (or refresh),
FGMRES.  Backward (hand-written, no tape): A^T lambda = dL/dx with a CPR
built on A^T, then dL/db = lambda and dL/dtheta from the pattern-restricted
outer product -lambda_i x_j^T chained through the harmonic transmissibility.
"""
from __future__ import annotations

import torch

from . import trs


class SolveContext:
    """Holds a synthetic system on the GPU and the preconditioners reused
    across forward/backward calls."""

    def __init__(self, sysm, device="cuda", precision="fp64", rtol=1e-10, restart=30, maxit=1000,
                 adjoint_decoupling="none"):
        self.ds = trs.DeviceSystem(sysm, device)
        self.precision = precision
        # the CPR on A^T works best undecoupled: ABF of A^T turns the dominant pressure column of A
        # into a dominant row, which the pressure extraction then weights badly
        self.adjoint_decoupling = adjoint_decoupling
        self.rtol = rtol
        self.restart = restart
        self.maxit = maxit
        self.M = None
        self.AT = None
        self.MT = None
        self.last_forward = None
        self.last_adjoint = None

    def assemble(self, theta):
        return self.ds.assemble(theta.detach().contiguous(), perm_is_log=True)

    def forward_solve(self, theta, rhs):
        A = self.assemble(theta)
        if self.M is None:
            self.M = trs.CPR(A, precision=self.precision)
        else:
            self.M.update(A, reuse_amg=False)
        x, res = trs.fgmres_solve(A, self.M, rhs.detach().contiguous(), rtol=self.rtol,
                                  restart=self.restart, maxit=self.maxit)
        self.last_forward = res
        return x

    def adjoint(self, theta, x, g):
        A = self.assemble(theta)
        self.AT = A.transpose(into=self.AT)
        if self.MT is None:
            self.MT = trs.CPR(self.AT, precision=self.precision, decoupling=self.adjoint_decoupling)
        else:
            self.MT.update(self.AT, reuse_amg=False)
        lam, _, res = trs.solve_adjoint(A, self.AT, self.MT, g.contiguous(), x, rtol=self.rtol,
                                        restart=self.restart, maxit=self.maxit)
        self.last_adjoint = res
        s = self.ds.sysm
        dtheta = trs.chain_theta(A, theta.detach().contiguous(), self.ds.M, lam, x, s.kvkh, s.c_t,
                                 perm_is_log=True)
        return lam, dtheta


class TrsSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, rhs, sctx: SolveContext):
        x = sctx.forward_solve(theta, rhs)
        ctx.sctx = sctx
        ctx.save_for_backward(theta, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        theta, x = ctx.saved_tensors
        lam, dtheta = ctx.sctx.adjoint(theta, x, gx.to(torch.float64))
        return dtheta, lam, None


def solve(theta, rhs, sctx: SolveContext):
    """x = A(theta)^-1 rhs, differentiable in theta and rhs."""
    return TrsSolve.apply(theta, rhs, sctx)
