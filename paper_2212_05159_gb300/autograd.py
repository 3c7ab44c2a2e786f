"""torch.autograd.Functions whose backward passes are the VJPs of Table 1.

Gradients of sparse inputs are plain value tensors on the input's own pattern
(Section 3.1); gradients of dense inputs are dense.
"""
from __future__ import annotations

import torch

from . import abi, ops
from .csr import CSR


class SpMM(torch.autograd.Function):
    """Y = A X with A = (pattern, values).  VJPs (Table 1, SpMV / SpDMM):
    dL/dA = (V X^T) masked to mask(A)  [SDDMM],  dL/dX = A^T V  [transpose-SpMM]."""

    @staticmethod
    def forward(ctx, values: torch.Tensor, X: torch.Tensor, A: CSR):
        ctx.A = A
        ctx.save_for_backward(values, X)
        return ops.spmm(A, X.contiguous(), values=values)

    @staticmethod
    def backward(ctx, V):
        values, X = ctx.saved_tensors
        A = ctx.A
        V = V.contiguous()
        if ctx.needs_input_grad[0] and ctx.needs_input_grad[1]:
            g_vals, g_X = ops.spmm_backward(A, V, X.contiguous(), values=values)   # one pass over A^T
            return g_vals, g_X, None
        g_vals = ops.sddmm(A, V, X.contiguous()) if ctx.needs_input_grad[0] else None
        g_X = ops.spmm_t(A, V, values=values) if ctx.needs_input_grad[1] else None
        return g_vals, g_X, None


def spmm(A: CSR, X: torch.Tensor, values: torch.Tensor | None = None) -> torch.Tensor:
    return SpMM.apply(A.values if values is None else values, X, A)


class SpGEMM(torch.autograd.Function):
    """values of C = A B on the plan's pattern.  VJPs (Table 1, SpSpMM):
    dL/dA = (V B^T) masked to A,  dL/dB = (A^T V) masked to B."""

    @staticmethod
    def forward(ctx, a_values, b_values, plan):
        ctx.plan = plan
        ctx.save_for_backward(a_values, b_values)
        return plan.numeric(a_values, b_values)

    @staticmethod
    def backward(ctx, gc):
        a_values, b_values = ctx.saved_tensors
        ga, gb = ctx.plan.backward(gc, a_values, b_values, ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        return ga, gb, None


class SpAdd(torch.autograd.Function):
    """values of C = alpha A + beta B on the plan's (union) pattern.  VJPs (Table 1,
    Sp + Sp): dL/dA = alpha V masked to A,  dL/dB = beta V masked to B."""

    @staticmethod
    def forward(ctx, a_values, b_values, plan, alpha: float, beta: float):
        ctx.plan, ctx.alpha, ctx.beta = plan, alpha, beta
        return plan.numeric(alpha, beta, a_values, b_values)

    @staticmethod
    def backward(ctx, gc):
        ga, gb = ctx.plan.backward(gc, ctx.alpha, ctx.beta, ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        return ga, gb, None, None, None


class SpTRSV(torch.autograd.Function):
    """x = L^-1 b for a batch of lower-triangular systems.  VJPs (Section 3.1.5, Table 1
    SpSolve rule): grad_b = L^-T v,  grad_L = -(L^-T v) x^T masked to mask(L)."""

    @staticmethod
    def forward(ctx, l_values, b, solver):
        x = solver.solve(b, l_values)
        ctx.solver = solver
        ctx.save_for_backward(l_values, x)
        return x

    @staticmethod
    def backward(ctx, v):
        l_values, x = ctx.saved_tensors
        lam = ctx.solver.solve(v.contiguous(), l_values, transpose=True)
        g_l = ops.masked_outer(ctx.solver.L, lam, x, -1.0) if ctx.needs_input_grad[0] else None
        return g_l, lam, None


class Permute(torch.autograd.Function):
    """out = values[perm] (e.g. A^T's values in A^T's order); the VJP gathers the gradient
    back through the inverse permutation."""

    @staticmethod
    def forward(ctx, values, perm, inv):
        ctx.inv = inv
        out = torch.empty_like(values)
        abi.spx_gather_values(perm, values.contiguous(), out)
        return out

    @staticmethod
    def backward(ctx, g):
        gv = torch.empty_like(g)
        abi.spx_gather_values(ctx.inv, g.contiguous(), gv)
        return gv, None, None


class Diagonal(torch.autograd.Function):
    """d_i = a_ii (0 where absent); the VJP puts g_i on the stored entry (i, i)."""

    @staticmethod
    def forward(ctx, values, A: CSR):
        pos = A.diagonal_positions()
        ctx.pos, ctx.nnz = pos, values.numel()
        nd = pos.numel()
        d = torch.empty(max(nd, 1), dtype=torch.float32, device=values.device)[:nd]
        abi.spx_csr_diagonal(A.struct(values.contiguous()), d, None)
        return d

    @staticmethod
    def backward(ctx, g):
        gv = torch.zeros(ctx.nnz, dtype=torch.float32, device=g.device)
        abi.spx_diagonal_backward(ctx.pos, g.contiguous(), gv)
        return gv, None
