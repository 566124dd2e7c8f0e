"""Differentiable assembly (adjoint form) and a Jacobi-preconditioned CG consumer.

``Assemble.apply(E, nu, X, asm)`` returns the CSR values of A = sum_tau P^T K^(tau) P + eps I
(Eq. 8) for the context's current active mask, as a function of per-tetrahedron Young's
modulus E, Poisson ratio nu and node positions X (CUDA float64 tensors).  Its backward is
the library's adjoint kernel (sta_adjoint): element matrices are recomputed, not stored.
Run the backward before the context's mask or parameters change.

``Solve.apply(val, f, asm, free, tol)`` solves A_ff u_f = f_f (pinned DOFs: u = 0) with
Jacobi-preconditioned conjugate gradients (the paper's solver, Sec. 4), the operator applied
by the library's SpMV over the context's pattern.  Its backward is the adjoint solve
A lam = dL/du and dL/dA_ij = -lam_i u_j on free rows and columns.  The solve is the consumer
of the assembly, not part of it.
"""
from __future__ import annotations

import torch

from . import Assembler, sta_adjoint, sta_spmv


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


def row_index(asm: Assembler) -> torch.Tensor:
    rp, _, _ = asm.csr()
    return torch.repeat_interleave(torch.arange(asm.n_rows, device=rp.device),
                                   (rp[1:] - rp[:-1]).long())


def diagonal(asm: Assembler, val: torch.Tensor) -> torch.Tensor:
    rp, col, _ = asm.csr()
    rows = row_index(asm)
    d = torch.zeros(asm.n_rows, dtype=val.dtype, device=val.device)
    on = col.long() == rows
    d[rows[on]] = val[on]
    return d


def pcg(asm: Assembler, val: torch.Tensor, b: torch.Tensor, free: torch.Tensor,
        tol: float = 1e-12, maxiter: int | None = None, x0: torch.Tensor | None = None):
    """Jacobi-preconditioned CG on the free DOFs: A_ff x_f = b_f, x = 0 on pinned DOFs.
    Stops when ||r|| <= tol ||b_f||.  Returns (x, iterations, relative residual)."""
    fm = free.to(val.dtype)
    b = b * fm
    d = diagonal(asm, val)
    dinv = torch.where(free & (d != 0), 1.0 / torch.where(d != 0, d, torch.ones_like(d)),
                       torch.zeros_like(d))

    def A(x):
        return sta_spmv(asm.h, x * fm, val) * fm

    x = torch.zeros_like(b) if x0 is None else x0 * fm
    r = b - A(x)
    z = dinv * r
    p = z.clone()
    rz = torch.dot(r, z)
    bn = torch.linalg.norm(b)
    if bn == 0:
        return x, 0, 0.0
    maxiter = maxiter or min(10 * int(free.sum().item()) + 100, 20000)
    rel = float(torch.linalg.norm(r) / bn)
    best, best_it = rel, 0
    it = 0
    while it < maxiter and rel > tol:
        Ap = A(p)
        alpha = rz / torch.dot(p, Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        if it % 10 == 0 or it < 10:
            rel = float(torch.linalg.norm(r) / bn)
            if rel <= tol:
                break
            if rel < 0.5 * best:
                best, best_it = rel, it
            elif it - best_it > 1000:  # stagnated at the attainable accuracy
                break
        z = dinv * r
        rz_new = torch.dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    rel = float(torch.linalg.norm(b - A(x)) / bn)
    return x, it, rel


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
        _, col, _ = ctx.asm.csr()
        rows = row_index(ctx.asm)
        cols = col.long()
        both = ctx.free[rows] & ctx.free[cols]
        grad_val = torch.where(both, -lam[rows] * u[cols], torch.zeros_like(val))
        grad_f = lam * ctx.free.to(lam.dtype)
        return grad_val, grad_f, None, None, None
