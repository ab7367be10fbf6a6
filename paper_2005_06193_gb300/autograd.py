"""torch.autograd wrappers: gradients of a functional of the converged Newton solution.

``newton_solve(d, kappa, handle)`` returns u* with r(u*; d, kappa) = 0.  Its backward pass
is the implicit-function adjoint computed by the CUDA library (egfem_adjoint):

    J(u*)^T lambda = dj/du   (free rows; lambda = 0 on Dirichlet rows)
    dj/dd = lambda,          dj/dkappa_m = -sum_{i,k} lambda_i T_imk u*_k

(the forward and backward solves that optimal control repeats, Sec. 6).  ``load_cellwise``
maps a cellwise-constant source to the load vector (egfem_load_cellwise) and back
(egfem_load_cellwise_transpose).  Only argument marshalling happens here.
"""
from __future__ import annotations

import torch

from .egfem import BatchHandle


class _NewtonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, d, kappa, handle):
        # The handle holds one kappa state, which later forwards may change.  Record the field
        # this solve used (None: the handle's constant kappa) and set it again before the adjoint,
        # so the backward pass linearises at the coefficient that produced u*.
        k_used = None if kappa is None else kappa.detach().contiguous().clone()
        handle.set_kappa(k_used)
        u = torch.zeros_like(d)
        if isinstance(handle, BatchHandle):
            stats = handle.batch_newton_solve(u, d.detach().contiguous())
        else:
            stats = [handle.newton_solve(u, d.detach().contiguous())]
        ctx.handle = handle
        ctx.k_used = k_used
        ctx.stats = stats
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        h = ctx.handle
        h.set_kappa(ctx.k_used)
        lam = torch.zeros_like(u)
        gk = torch.zeros(h.sizes.n_wa, device=u.device, dtype=u.dtype) if ctx.k_used is not None else None
        h.adjoint(u, gu.contiguous(), lam, gk)
        return lam, gk, None


class _LoadCellwise(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f_cell, handle):
        d = torch.empty(handle.sizes.n_nodes, device=f_cell.device, dtype=f_cell.dtype)
        handle.load_cellwise(f_cell.detach().contiguous(), d)
        ctx.handle = handle
        ctx.n_cells = f_cell.numel()
        return d

    @staticmethod
    def backward(ctx, gd):
        g = torch.empty(ctx.n_cells, device=gd.device, dtype=gd.dtype)
        ctx.handle.load_cellwise_transpose(gd.contiguous(), g)
        return g, None


def newton_solve(d: torch.Tensor, kappa: torch.Tensor | None, handle) -> torch.Tensor:
    """u* solving the discrete problem for load d (and W-field kappa, or the handle's
    constant kappa when None); differentiable with respect to d and kappa."""
    return _NewtonSolve.apply(d, kappa, handle)


def load_cellwise(f_cell: torch.Tensor, handle) -> torch.Tensor:
    """Load vector of a cellwise-constant source (differentiable)."""
    return _LoadCellwise.apply(f_cell, handle)
