"""Differentiable solve u = A^{-1} f and preconditioner apply z = P^{-1} r for torch.

FmmSolve.apply(f, P, opts) runs the FMM-preconditioned Krylov solve of the 5-point system
(fmmpc_solve).  Its backward is the adjoint solve A^{-T} g; the 5-point matrix with zero
Dirichlet values is symmetric, so that is the same preconditioned solve applied to the
incoming gradient.  Both passes run entirely in libfmmpc.  A solve of either pass that stops
at maxit above rtol (or meets a NaN) raises FmmpcError with its status and residual, so a
gradient is never returned from an unconverged adjoint solve.

FmmApply.apply(r, P) is the preconditioner itself, z = P^{-1} r (fmmpc_apply); its backward
is the FMM-transpose pass rb = P^{-T} zb (fmmpc_apply_transpose), the gradient with respect
to the source weights r.  P^{-1} is not symmetric (its boundary correction is a collocation
system), so the transpose is a pass of its own.
"""
from __future__ import annotations

import torch

from ._lib import FmmpcError

__all__ = ["FmmSolve", "fmm_solve", "FmmApply", "fmm_apply"]

_DEFAULTS = dict(method="fgmres", restart=30, maxit=200, rtol=1e-10, use_graphs=2)


def _checked_solve(P, rhs, opts, what):
    u, info = P.solve(rhs, raise_on_fail=False, **opts)
    if info["status"] != 0:
        raise FmmpcError(info["status"], f"{what} solve did not converge: {info['iters']} iterations, "
                                         f"relative residual {info['rel_res']:.3e} > rtol {opts['rtol']:.1e}")
    return u, info


class FmmSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, P, opts):
        o = dict(_DEFAULTS, **(opts or {}))
        o.pop("raise_on_fail", None)
        u, info = _checked_solve(P, f.detach().contiguous(), o, "forward")
        ctx.P, ctx.opts = P, o
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, grad_u):
        g, info = _checked_solve(ctx.P, grad_u.detach().contiguous(), ctx.opts, "adjoint")
        ctx.info_backward = info
        return g, None, None


def fmm_solve(f: torch.Tensor, P, **opts) -> torch.Tensor:
    """u = A^{-1} f with gradients; f is a float64 CUDA tensor of n*n (or [R, n*n]) values."""
    return FmmSolve.apply(f, P, opts)


class FmmApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r, P):
        ctx.P = P
        return P.apply(r.detach().contiguous())

    @staticmethod
    def backward(ctx, grad_z):
        return ctx.P.apply_transpose(grad_z.detach().contiguous()), None


def fmm_apply(r: torch.Tensor, P) -> torch.Tensor:
    """z = P^{-1} r with gradients through the FMM-transpose pass."""
    return FmmApply.apply(r, P)
