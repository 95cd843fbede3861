"""torch.autograd.Function for the Poisson control solve.

u = PoissonControlSolve.apply(yD, log_alpha, solver_factory) returns the
optimal control u = lambda / alpha of the discretised problem (eq. (mp2) and
u = alpha^{-1} lambda) for the desired state yD (nodal values, float64 CUDA
tensor) and log_alpha (0-d float64 tensor).  The backward pass is the adjoint
solve of the library (mg_adjoint: A is symmetric, so the adjoint system is
A z = (0, dL/du / alpha)), giving dL/dyD = M z_y and
dL/dlog(alpha) = alpha dL/dalpha with
dL/dalpha = -alpha^{-2} (dL/du . lambda + z_lambda^T M lambda).
This differentiates the exact discrete solution, not the iteration.
"""
from __future__ import annotations

import math

import torch

from . import aaomg


class PoissonControlSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, yD, log_alpha, levels: int, tol: float = 1e-10, smoother: str = "lsgs",
                precision: str = "fp32_refine"):
        alpha = math.exp(float(log_alpha))
        s = aaomg.Solver(levels, alpha, smoother=smoother, precision=precision, max_iter=200)
        f = s.rhs_from_yd(yD.contiguous())
        x = torch.zeros_like(f)
        s.solve(f, x, tol=tol)
        u = s.control(x)
        ctx.solver, ctx.alpha, ctx.tol = s, alpha, tol
        ctx.save_for_backward(x)
        return u

    @staticmethod
    def backward(ctx, ubar):
        (x,) = ctx.saved_tensors
        s = ctx.solver
        gyD, dalpha, _ = s.adjoint(x, ubar.contiguous().to(torch.float64), tol=ctx.tol)
        g_log_alpha = torch.tensor(ctx.alpha * dalpha, dtype=torch.float64, device=x.device)
        return gyD, g_log_alpha, None, None, None, None


def control(yD, log_alpha, levels: int, tol: float = 1e-10, smoother: str = "lsgs", precision: str = "fp32_refine"):
    """The optimal control u(yD, alpha), differentiable in yD and log_alpha."""
    return PoissonControlSolve.apply(yD, log_alpha, levels, tol, smoother, precision)
