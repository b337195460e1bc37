"""torch.autograd.Function for the SPD solve X = A^{-1} B with a hand-written
adjoint (the paper exposes potrs as a primitive that composes with the
framework's transformations, "Summary"; this is its reverse mode).

forward : X = A^{-1} B through the library (FP64 potrf + potrs, or the mixed
          tensor-core factor + FP64 refinement).  The factor is kept.
backward: Bbar = A^{-1} Xbar with the kept factor (FP64 potrs, or refinement
          against the kept mixed factor without refactoring), then
          Abar = -(Bbar X^T + X Bbar^T) / 2 in one fused kernel.

A is symmetric and only one triangle is read, so the gradient returned for A
is the symmetric one: a symmetric perturbation dA changes the loss by
<Abar, dA>.  Every step runs in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import jmg


def _as_colmajor_sym(A: torch.Tensor) -> torch.Tensor:
    # a symmetric matrix is its own transpose: a row-major tensor's .mT view is
    # the same matrix in column-major layout
    return A if A.stride(0) == 1 else A.mT


class SPDSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, prec="fp64", words=1, tol=1e-13):
        if A.dim() != 2 or A.shape[0] != A.shape[1]:
            raise ValueError("A must be square")
        vec = B.dim() == 1
        B2 = B.reshape(-1, 1) if vec else B
        Acm = _as_colmajor_sym(A)
        ctx.prec, ctx.words, ctx.tol, ctx.vec = prec, words, tol, vec
        if prec == "fp64":
            L = jmg.colmajor_copy(Acm)
            info = jmg.potrf_(L)
            if int(info.item()) != 0:
                raise jmg.JmgError(3, "SPDSolve: potrf info=%d" % int(info.item()))
            X = jmg.colmajor_copy(B2)
            jmg.potrs_(L, X)
            ctx.save_for_backward(L, X)
            ctx.work = None
        else:
            n, nrhs = B2.shape
            opts = jmg.default_options(prec=prec, words=words)
            work = jmg.workspace(jmg.OP_POSV, n, nrhs, opts, A.device)
            X, _ = jmg.posv(Acm, B2, prec=prec, words=words, tol=tol, work=work)
            ctx.save_for_backward(Acm, X)
            ctx.work = work
        return X.reshape(-1) if vec else X

    @staticmethod
    def backward(ctx, Xbar):
        F, X = ctx.saved_tensors
        Xb = jmg.colmajor_copy(Xbar.reshape(-1, 1) if ctx.vec else Xbar)
        if ctx.prec == "fp64":
            Bbar = jmg.potrs_(F, Xb)
        else:
            Bbar, _ = jmg.posv(F, Xb, prec=ctx.prec, words=ctx.words, tol=ctx.tol, work=ctx.work,
                               reuse_factor=True)
        Abar = jmg.sym_grad(Bbar, X) if ctx.needs_input_grad[0] else None
        gB = None
        if ctx.needs_input_grad[1]:
            gB = Bbar.reshape(-1) if ctx.vec else Bbar
        return Abar, gB, None, None, None


def solve(A: torch.Tensor, B: torch.Tensor, prec: str = "fp64", words: int = 1,
          tol: float = 1e-13) -> torch.Tensor:
    """Differentiable X = A^{-1} B for symmetric positive-definite A (CUDA, FP64)."""
    return SPDSolve.apply(A, B, prec, words, tol)
