"""torch.autograd.Functions for the Poisson control solve.

u = control(yD, log_alpha, levels) returns the optimal control u = lambda /
alpha of the discretised problem (eq. (mp2) and u = alpha^{-1} lambda) for the
desired state yD (nodal values, float64 CUDA tensor; a 2-D tensor of shape
(B, N) solves B instances at once) and log_alpha (0-d float64 tensor, shared by
the instances).  The backward pass is the adjoint solve of the library
(mg_adjoint, or mg_batch_adjoint for a batch: A is symmetric, so the adjoint
system is A z = (0, dL/du / alpha)), giving dL/dyD = M z_y and
dL/dlog(alpha) = alpha dL/dalpha with
dL/dalpha = -alpha^{-2} (dL/du . lambda + z_lambda^T M lambda),
summed over the instances of a batch.  This differentiates the exact discrete
solution, not the iteration.

The multigrid hierarchies (and for a batch its recorded graph) are kept in a
small cache keyed by (levels, alpha, smoother, precision, instances), so that
repeated forward/backward passes at the same alpha set up nothing.
"""
from __future__ import annotations

import collections
import math
import threading

import torch

from . import aaomg

_CACHE_SIZE = 4
_cache: "collections.OrderedDict[tuple, tuple]" = collections.OrderedDict()
_cache_lock = threading.Lock()


def _hierarchy(levels: int, alpha: float, smoother: str, precision: str, count: int):
    """(solvers, batch or None) for the key, set up on first use; the least
    recently used entry is closed when the cache is full."""
    key = (int(levels), float(alpha), smoother, precision, int(count))
    with _cache_lock:
        if key in _cache:
            _cache.move_to_end(key)
            return _cache[key]
        solvers = [aaomg.Solver(levels, alpha, smoother=smoother, precision=precision, max_iter=200)
                   for _ in range(count)]
        batch = aaomg.Batch(solvers) if count > 1 else None
        _cache[key] = (solvers, batch)
        while len(_cache) > _CACHE_SIZE:
            _, (old, ob) = _cache.popitem(last=False)
            if ob is not None:
                ob.close()
            for s in old:
                s.close()
        return solvers, batch


def clear_cache():
    """Close every cached hierarchy."""
    with _cache_lock:
        while _cache:
            _, (old, ob) = _cache.popitem()
            if ob is not None:
                ob.close()
            for s in old:
                s.close()


class PoissonControlSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, yD, log_alpha, levels: int, tol: float = 1e-10, smoother: str = "lsgs",
                precision: str = "fp32_refine"):
        alpha = math.exp(float(log_alpha))
        batched = yD.dim() == 2
        Y = yD.contiguous() if batched else yD.contiguous().unsqueeze(0)
        solvers, batch = _hierarchy(levels, alpha, smoother, precision, Y.shape[0])
        fs = [s.rhs_from_yd(Y[k]) for k, s in enumerate(solvers)]
        xs = [torch.zeros_like(f) for f in fs]
        if batch is None:
            solvers[0].solve(fs[0], xs[0], tol=tol)
        else:
            batch.solve(fs, xs, tol=tol)
        u = torch.stack([s.control(x) for s, x in zip(solvers, xs)])
        ctx.key = (levels, alpha, smoother, precision, Y.shape[0])
        ctx.alpha, ctx.tol, ctx.batched = alpha, tol, batched
        ctx.save_for_backward(torch.stack(xs))
        return u if batched else u[0]

    @staticmethod
    def backward(ctx, ubar):
        (X,) = ctx.saved_tensors
        solvers, batch = _hierarchy(*ctx.key)
        U = ubar.contiguous().to(torch.float64)
        if not ctx.batched:
            U = U.unsqueeze(0)
        if batch is None:
            gyD, dalpha, _ = solvers[0].adjoint(X[0].contiguous(), U[0].contiguous(), tol=ctx.tol)
            gs, das = [gyD], [dalpha]
        else:
            gs, das, _, _ = batch.adjoint([X[k].contiguous() for k in range(X.shape[0])],
                                          [U[k].contiguous() for k in range(U.shape[0])], tol=ctx.tol)
        g_log_alpha = torch.tensor(ctx.alpha * sum(das), dtype=torch.float64, device=X.device)
        G = torch.stack(gs)
        return (G if ctx.batched else G[0]), g_log_alpha, None, None, None, None


def control(yD, log_alpha, levels: int, tol: float = 1e-10, smoother: str = "lsgs", precision: str = "fp32_refine"):
    """The optimal control u(yD, alpha), differentiable in yD and log_alpha;
    yD of shape (N,) or (B, N) (B instances solved as one batch)."""
    return PoissonControlSolve.apply(yD, log_alpha, levels, tol, smoother, precision)
