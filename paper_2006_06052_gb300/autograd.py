"""torch.autograd wrapper of the solve: x = K(vals)^-1 b.

Backward (reverse-mode through a linear solve): with g = dL/dx the
adjoint lam = K^-T g gives dL/db = lam and dL/dK_ij = -lam_i x_j^T on the
stored block pattern (sampled outer product).  Only x is saved from the
forward pass; the adjoint solve is recomputed in backward from x and the
hierarchy (no Krylov history is stored).  The preconditioner hierarchy is
treated as a constant: x = K^-1 b does not depend on it once the solve
has converged.
"""
from __future__ import annotations

import torch

from . import Hierarchy, sampled_outer, solve, solve_adjoint, update_values


class StokesSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals: torch.Tensor, b: torch.Tensor, H: Hierarchy):
        update_values(H, vals.detach().contiguous())
        x, info = solve(H, b.detach().contiguous())
        if not info.converged:
            raise RuntimeError("forward solve did not converge: %s" % info.as_dict())
        ctx.H = H
        ctx.save_for_backward(x)
        ctx.info = info.as_dict()
        return x

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        (x,) = ctx.saved_tensors
        lam, info = solve_adjoint(ctx.H, gx.detach().contiguous())
        if not info.converged:
            raise RuntimeError("adjoint solve did not converge: %s" % info.as_dict())
        grad_vals = sampled_outer(ctx.H, lam, x, -1.0) if ctx.needs_input_grad[0] else None
        grad_b = lam if ctx.needs_input_grad[1] else None
        return grad_vals, grad_b, None


def stokes_solve(vals: torch.Tensor, b: torch.Tensor, H: Hierarchy) -> torch.Tensor:
    """Differentiable x = K(vals)^-1 b with K's pattern and preconditioner from H."""
    return StokesSolve.apply(vals, b, H)
