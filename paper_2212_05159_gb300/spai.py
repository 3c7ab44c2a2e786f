"""Sparse approximate inverse by gradient descent (Section 4.6).

Minimises loss(M) = ||I - M A||_F^2 over the stored entries of M with mask(M) = mask(A),
from M = mask(A) (every stored entry 1), until the gradient norm is below `gtol` (0.01 in
the paper).  Every step runs on the device through the library:

    C = M A                       spx_spgemm_numeric (pattern of M A analysed once)
    gC = -2 (I - C)               spx_spai_residual
    g = (gC A^T) on mask(M)       spx_spgemm_backward (gradient w.r.t. the first operand)
    <g, g>, <g A, g A>            spx_spgemm_numeric for g A, spx_dot
    M -= (1/2) <g,g>/<gA,gA> g    spx_spai_update (exact minimiser along -g: the loss is
                                  quadratic in M; the paper gives no step size)

The host reads two numbers per step (the loss and the gradient norm) to decide when to stop.
"""
from __future__ import annotations

import torch

from . import abi
from .csr import CSR
from .ops import SpGEMMPlan


class SPAIDescent:
    """State of the descent for one sparse matrix A (square, float32 values on the device)."""

    def __init__(self, A: CSR):
        if A.m != A.n:
            raise ValueError("SPAI needs a square matrix")
        self.A = A
        dev = A.device
        self.M = A.with_values(torch.ones(A.nnz, dtype=torch.float32, device=dev))
        self.plan = SpGEMMPlan(self.M, A)                      # pattern of C = M A, once
        nc = self.plan.C.nnz
        self.c = torch.empty(nc, dtype=torch.float32, device=dev)
        self.gc = torch.empty(nc, dtype=torch.float32, device=dev)
        self.ga = torch.empty(nc, dtype=torch.float32, device=dev)
        self.scal = torch.zeros(3, dtype=torch.float64, device=dev)       # <gC,gC>, <g,g>, <gA,gA>
        self.diag = torch.zeros(1, dtype=torch.int32, device=dev)
        self.ws = abi.workspace(abi.spx_dot_workspace_size(max(nc, A.nnz)), dev)
        self.history: list[tuple[float, float]] = []

    @property
    def values(self) -> torch.Tensor:
        return self.M.values

    def gradient(self):
        """Loss and gradient at the current M; the gradient stays on the device."""
        A, plan = self.A, self.plan
        plan.numeric(self.M.values, A.values, out=self.c)
        abi.spx_spai_residual(plan.C.struct(self.c), -2.0, self.gc, self.diag)
        g, _ = plan.backward(self.gc, a_values=self.M.values, b_values=A.values, need_b=False)
        abi.spx_dot(self.gc, self.gc, self.scal[0:1], self.ws)
        abi.spx_dot(g, g, self.scal[1:2], self.ws)
        return g

    def step(self, g):
        """One exact line-search step along -g."""
        self.plan.numeric(g, self.A.values, out=self.ga)
        abi.spx_dot(self.ga, self.ga, self.scal[2:3], self.ws)
        abi.spx_spai_update(self.M.values, g, self.scal[1:2], self.scal[2:3])

    def run(self, gtol: float = 1e-2, max_it: int = 500):
        """Descends until ||grad|| < gtol (or max_it steps); returns the history of
        (loss, ||grad||) at every iterate, the last one included."""
        for _ in range(max_it + 1):
            g = self.gradient()
            s = self.scal.cpu()
            loss = float(s[0]) / 4.0 + (self.A.m - int(self.diag.cpu()))
            gn = float(s[1]) ** 0.5
            self.history.append((loss, gn))
            if gn < gtol or len(self.history) > max_it:
                break
            self.step(g)
        return self.history
