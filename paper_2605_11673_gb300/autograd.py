"""Differentiable assembly (adjoint form) and a Jacobi-preconditioned CG consumer.

``Assemble.apply(E, nu, X, asm)`` returns the CSR values of A = sum_tau P^T K^(tau) P + eps I
(Eq. 8) for the context's current active mask, as a function of per-tetrahedron Young's
modulus E, Poisson ratio nu and node positions X (CUDA float64 tensors).  Its backward is
the library's adjoint kernel (sta_adjoint): element matrices are recomputed, not stored.
Run the backward before the context's mask or parameters change.

``Solve.apply(val, f, asm, free, tol)`` solves A_ff u_f = f_f (pinned DOFs: u = 0) with
Jacobi-preconditioned conjugate gradients (the paper's solver, Sec. 4) in the library
(sta_solve).  Its backward is the adjoint solve A lam = dL/du and dL/dA_ij = -lam_i u_j on
free rows and columns (sta_outer_grad).  The solve is the consumer of the assembly, not part
of it.
"""
from __future__ import annotations

import torch

from . import Assembler, sta_adjoint, sta_outer_grad, sta_solve


class Assemble(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E, nu, X, asm: Assembler):
        asm.set_params(X=X.detach(), E=E.detach(), nu=nu.detach())
        asm.refold()
        ctx.asm = asm
        return asm.values().clone()

    @staticmethod
    def backward(ctx, grad_val):
        dE, dnu, dX = sta_adjoint(ctx.asm.h, grad_val.contiguous())
        return dE, dnu, dX, None


def pcg(asm: Assembler, val: torch.Tensor, b: torch.Tensor, free: torch.Tensor,
        tol: float = 1e-12, maxiter: int | None = None, x0: torch.Tensor | None = None):
    """Jacobi-preconditioned CG on the free DOFs: A_ff x_f = b_f, x = 0 on pinned DOFs
    (the library's sta_solve).  Stops when ||r|| <= tol ||b_f||, at maxiter, or once the
    residual stagnates.  Returns (x, iterations, relative residual)."""
    maxiter = maxiter or min(10 * int(free.sum().item()) + 100, 20000)
    return sta_solve(asm.h, b, free, val, tol, maxiter, x0)


class Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, val, f, asm: Assembler, free, tol: float = 1e-12):
        u, _, _ = pcg(asm, val.detach(), f.detach(), free, tol)
        ctx.save_for_backward(val, u)
        ctx.asm, ctx.free, ctx.tol = asm, free, tol
        return u

    @staticmethod
    def backward(ctx, grad_u):
        val, u = ctx.saved_tensors
        lam, _, _ = pcg(ctx.asm, val.detach(), grad_u, ctx.free, ctx.tol)
        grad_val = sta_outer_grad(ctx.asm.h, lam, u, ctx.free)
        grad_f = lam * ctx.free.to(lam.dtype)
        return grad_val, grad_f, None, None, None
