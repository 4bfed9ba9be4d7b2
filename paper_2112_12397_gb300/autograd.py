"""torch.autograd.Function around the forward and adjoint solves.

forward:  x = J^-1 b                      (fc_solve, FGMRES with M^-1)
backward: lambda = J^-T (dL/dx)           (fc_solve_adjoint, FGMRES with M^-T)
          dL/db = lambda

The adjoint solve builds its own Krylov basis: nothing of the forward basis is
stored between the two passes.
"""
from __future__ import annotations

import torch

from . import Context


class FracSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b: torch.Tensor, solver: Context, variant: str = "tup", tol: float = 1e-8,
                maxit: int = 500):
        x = torch.zeros_like(b)
        solver.solve(variant, b.detach().contiguous(), x, tol, maxit)
        ctx.solver, ctx.variant, ctx.tol, ctx.maxit = solver, variant, tol, maxit
        return x

    @staticmethod
    def backward(ctx, grad_x: torch.Tensor):
        lam = torch.zeros_like(grad_x)
        ctx.solver.solve_adjoint(ctx.variant, grad_x.detach().contiguous(), lam, ctx.tol, ctx.maxit)
        return lam, None, None, None, None


def frac_solve(b: torch.Tensor, solver: Context, variant: str = "tup", tol: float = 1e-8,
               maxit: int = 500) -> torch.Tensor:
    """Differentiable x = J^-1 b with the block-preconditioned FGMRES."""
    return FracSolve.apply(b, solver, variant, tol, maxit)
