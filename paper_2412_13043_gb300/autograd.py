"""torch.autograd.Function around ffrg_rhs / ffrg_rhs_adjoint.

forward: tables (CUDA float64 tensor [n_tables, n_stack, n_pts]) -> the RHS at
scale k (one value per external point).  backward: the library's hand-written
adjoint kernel gives d(RHS)/d(tables)^T grad_out.  Marshalling only.
"""
from __future__ import annotations

import torch

from . import FP64, Context


class RhsFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tables: torch.Tensor, lib_ctx: Context, problem, k: float, precision: int = FP64):
        if not tables.is_cuda or tables.dtype != torch.float64:
            raise ValueError("tables must be a CUDA float64 tensor")
        t = tables.detach().contiguous()
        handle = lib_ctx.tables(problem, t)
        try:
            out = lib_ctx.rhs(problem, handle, k, precision=precision)
        finally:
            handle.free()
        ctx.lib_ctx = lib_ctx
        ctx.problem = problem
        ctx.k = k
        ctx.save_for_backward(t)
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (t,) = ctx.saved_tensors
        handle = ctx.lib_ctx.tables(ctx.problem, t)
        try:
            tbar = ctx.lib_ctx.rhs_adjoint(ctx.problem, handle, ctx.k, grad_out.contiguous().to(torch.float64))
        finally:
            handle.free()
        return tbar.view_as(t), None, None, None, None


def rhs(tables: torch.Tensor, lib_ctx: Context, problem, k: float, precision: int = FP64) -> torch.Tensor:
    """Differentiable RHS: gradients flow back to `tables` through the adjoint kernel."""
    return RhsFunction.apply(tables, lib_ctx, problem, k, precision)
