"""Differentiable CTA solve: a torch.autograd.Function whose backward runs adjoint
solves on the GPU through the C ABI.

Forward: x = the CTA solution of A x = b (Alg. 1.1, H = A Aᵀ). From x0 = 0 CTA's
iterates stay in range(Aᵀ) (Thm. thmone (4)), so for a square nonsingular A it is
A^{-1} b and for a full-row-rank A (m < n) it is the minimum-norm solution A⁺ b.

Backward, for a loss L with g = dL/dx:
  * lambda = (A⁺)ᵀ g, the least-squares solution of Aᵀ lambda = g: a CTA solve with
    the plan of Aᵀ;
  * dL/db = lambda;
  * square A:           dL/dA = -lambda xᵀ;
  * full row rank m<n:  w = (A Aᵀ)^{-1} b is the least-squares solution of Aᵀ w = x
    (a second CTA solve with Aᵀ), and dL/dA = w (g - Aᵀ lambda)ᵀ - lambda xᵀ.
dL/dA is formed on A's stored pattern only (CSR: one value per nonzero) by the
library's pattern outer-product kernel; Aᵀ lambda comes from the library's product.
The paper has no counterpart: this makes its solver usable inside training loops.
"""
from __future__ import annotations

import torch

from . import CSR, PRECISION_FP64, Plan


class CTASolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, rowptr, colidx, shape, opts):
        A = CSR(rowptr, colidx, vals.detach().contiguous(), shape) if rowptr is not None \
            else vals.detach().contiguous()
        plan = Plan(A)
        x, _, info = plan.cta(b.detach().contiguous(), **opts)
        ctx.plan, ctx.opts, ctx.shape = plan, dict(opts), tuple(shape)
        ctx.csr = rowptr is not None
        ctx.nvals = vals.numel()
        ctx.info = info
        ctx.save_for_backward(b, x)
        return x

    @staticmethod
    def backward(ctx, g):
        b, x = ctx.saved_tensors
        m, n = ctx.shape
        plan = ctx.plan
        opts = dict(ctx.opts)
        # the adjoint systems are least-squares problems (Aᵀ lambda = g has no exact solution
        # unless g is in range(Aᵀ)): their stop is the normal-equation test, at the forward
        # tolerance unless a positive one was given
        if not opts.get("tol_normal", 0.0) or opts["tol_normal"] <= 0.0:
            opts["tol_normal"] = opts.get("tol", 1e-10)
        pt = plan.transpose()
        try:
            lam, _, _ = pt.cta(g.contiguous(), **opts)
            grad = torch.zeros(ctx.nvals, dtype=torch.float64, device=b.device)
            plan.outer(-1.0, lam, x, grad)                          # -lambda xᵀ
            if m < n:
                w, _, _ = pt.cta(x.contiguous(), **opts)           # (A Aᵀ)^{-1} b
                resid = plan.residual(lam, g.contiguous(), transpose=True)   # g - Aᵀ lambda
                plan.outer(1.0, w, resid, grad)
        finally:
            pt.close()
            plan.close()
        grad_A = grad if ctx.csr else grad.view(m, n)
        return grad_A, lam, None, None, None, None


def cta_solve_autograd(A, b, **opts):
    """x = CTA solution of A x = b with gradients to A's values and to b.

    A: a CUDA float64 tensor (dense m x n, m <= n, full row rank) or
    CSR(rowptr, colidx, vals, shape) whose vals may require grad (the gradient lives on
    the nonzero pattern). Options are those of cta_solve (tol, max_iter, ...); FP64 only.
    """
    if opts.get("precision", PRECISION_FP64) != PRECISION_FP64:
        raise ValueError("the differentiable solve runs the FP64 path")
    if isinstance(A, CSR):
        return CTASolveFn.apply(A.vals, b, A.rowptr, A.colidx, tuple(A.shape), opts)
    return CTASolveFn.apply(A, b, None, None, tuple(A.shape), opts)
