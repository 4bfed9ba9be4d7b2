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


class ApertureSystem:
    """J(a) for fracture apertures a: the input generator assembles the
    blocks (and their aperture derivatives) for a given a; the library sets
    up the preconditioner and solves.  `options` are fc_options."""

    def __init__(self, cfg, options=None):
        self.cfg = cfg
        self.options = options
        self.ctx = None
        self.problem = None

    def assemble(self, a: torch.Tensor):
        import fracgen
        from . import context_for, device_dk
        P = fracgen.generate(self.cfg, aperture=a.detach().double().cpu().numpy())
        if self.ctx is not None:
            self.ctx.close()
        self.ctx = context_for(P, self.options)
        self.problem = P
        self.dk = device_dk(P)
        return P


class FracSolveAperture(torch.autograd.Function):
    """x = J(a)^-1 b; backward gives dL/db = lambda and
    dL/da_f = -lambda^T (dJ/da_f) x through T and Q2."""

    @staticmethod
    def forward(ctx, a: torch.Tensor, b: torch.Tensor, system: ApertureSystem, variant: str = "tup",
                tol: float = 1e-8, maxit: int = 500):
        system.assemble(a)
        x = torch.zeros_like(b)
        system.ctx.solve(variant, b.detach().contiguous(), x, tol, maxit)
        ctx.save_for_backward(x)
        ctx.system, ctx.variant, ctx.tol, ctx.maxit = system, variant, tol, maxit
        return x

    @staticmethod
    def backward(ctx, grad_x: torch.Tensor):
        (x,) = ctx.saved_tensors
        sysm = ctx.system
        lam = torch.zeros_like(grad_x)
        sysm.ctx.solve_adjoint(ctx.variant, grad_x.detach().contiguous(), lam, ctx.tol, ctx.maxit)
        grad_a = torch.zeros(sysm.problem.n_face, dtype=torch.float64, device=x.device)
        sysm.ctx.aperture_gradient(sysm.dk, x, lam, grad_a)
        return grad_a, lam, None, None, None, None


def frac_solve_aperture(a: torch.Tensor, b: torch.Tensor, system: ApertureSystem, variant: str = "tup",
                        tol: float = 1e-8, maxit: int = 500) -> torch.Tensor:
    """Differentiable x = J(a)^-1 b in both the apertures a and b."""
    return FracSolveAperture.apply(a, b, system, variant, tol, maxit)
