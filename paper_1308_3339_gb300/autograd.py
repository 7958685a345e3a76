"""Differentiable solve u = A^{-1} f for torch.

FmmSolve.apply(f, P, opts) runs the FMM-preconditioned Krylov solve of the 5-point system
(fmmpc_solve).  Its backward is the adjoint solve A^{-T} g; the 5-point matrix with zero
Dirichlet values is symmetric, so that is the same preconditioned solve applied to the
incoming gradient.  Both passes run entirely in libfmmpc.
"""
from __future__ import annotations

import torch

__all__ = ["FmmSolve", "fmm_solve"]

_DEFAULTS = dict(method="fgmres", restart=30, maxit=200, rtol=1e-10, use_graphs=1)


class FmmSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, P, opts):
        o = dict(_DEFAULTS, **(opts or {}))
        u, info = P.solve(f.detach().contiguous(), **o)
        ctx.P, ctx.opts = P, o
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, grad_u):
        g, info = ctx.P.solve(grad_u.detach().contiguous(), **ctx.opts)
        return g, None, None


def fmm_solve(f: torch.Tensor, P, **opts) -> torch.Tensor:
    """u = A^{-1} f with gradients; f is a float64 CUDA tensor of n*n (or [R, n*n]) values."""
    return FmmSolve.apply(f, P, opts)
