"""Differentiable batched sparse solve: PCG forward, PCG adjoint backward.

Table 1 (SpSolve): for x = A^{-1} b the VJPs are grad_b = A^{-T} v and
grad_A = -(A^{-T} v) x^T masked to mask(A).  The paper computes A^{-T} v with the LU
factors of its direct solve (Section 3.1.6); here A is SPD and block-diagonal (a batch of
independent systems), A^{-T} = A^{-1}, and both solves are the same batched PCG kernel.
The adjoint needs only x and v: no iterate of the forward solve is stored.
"""
from __future__ import annotations

import numpy as np
import torch

from . import abi
from .csr import CSR

PC = {"none": 0, "jacobi": 1, "llt": 2, "M": 3, "ic0": 4, "dia": 5}


class SystemBatch:
    """A block-diagonal batch of SPD systems on the device with its solver scratch."""

    def __init__(self, A: CSR, sys_ptr):
        self.A = A
        ptr = np.asarray(sys_ptr, dtype=np.int32)
        self.nsys = len(ptr) - 1
        self.sys_ptr_host = ptr
        self.sys_ptr = torch.from_numpy(ptr).to(A.device)
        sizes = np.diff(ptr.astype(np.int64))
        # largest systems first: the longest solves start first (load balance)
        self.order = torch.from_numpy(np.argsort(-sizes, kind="stable").astype(np.int32)).to(A.device)
        self.ws = abi.workspace(abi.spx_cg_workspace_size(A.m), A.device)
        self.mean_rows = float(sizes.mean()) if sizes.size else 1.0
        self.max_rows = float(sizes.max()) if sizes.size else 1.0
        self.launch = None          # (threads, cluster, max clusters); None = launch_for()
        self._dinv = None
        self.iters = torch.zeros(self.nsys, dtype=torch.int32, device=A.device)
        self.status = torch.zeros(self.nsys, dtype=torch.int32, device=A.device)
        self.relres = torch.zeros(self.nsys, dtype=torch.float64, device=A.device)

    def launch_for(self, kind: int):
        """Launch shape of spx_cg_batched: 1024-thread blocks and a cluster (power of two, at
        most 16).  With no preconditioner, Jacobi or an explicit M the cluster is the
        smallest whose blocks hold the largest system's private vectors in shared memory
        (8 rows per thread); measured on GB300 with 2D diffusion batches, 64 systems of
        256^2 run at 70 ms (Jacobi) and 102 ms (explicit M) with 8 blocks against 94 and
        133 ms with the vectors in global memory, and 256 systems of 32^2..256^2 at 105 ms
        against 127 ms.  IC(0) runs its triangular solves on one block per system while
        the cluster's other blocks wait, so it takes one block per system (128 systems of
        256^2: 1.15 s against 6.2 s with 8 blocks); L L^T keeps ~4 rows of an average
        system per thread."""
        if self.launch is not None:
            return self.launch
        if kind in (0, 1, 3, 5):
            want = self.max_rows / (8.0 * 1024.0)
            cl = 2 ** int(np.ceil(np.log2(max(want, 1.0))))
        elif kind == 4:
            cl = 1
        else:
            want = self.mean_rows / 4.0 / 1024.0
            cl = 2 ** int(round(np.log2(max(want, 1.0))))
        return (1024, int(min(16, max(1, cl))), 0)

    def dinv(self, values=None):
        if values is not None:
            d = torch.empty(self.A.m, dtype=torch.float32, device=self.A.device)
            return abi.spx_diag_inverse(self.A.struct(values), d)
        if self._dinv is None:
            self._dinv = torch.empty(self.A.m, dtype=torch.float32, device=self.A.device)
            abi.spx_diag_inverse(self.A.struct(), self._dinv)
        return self._dinv


class Factor:
    """M = L L^T with L lower-triangular on a fixed pattern (Section 4.3)."""

    def __init__(self, L: CSR):
        self.L = L
        t_ip, t_ix, perm = L.transpose_pattern()
        self.perm = perm
        self.lt_vals = torch.empty(L.nnz, dtype=torch.float32, device=L.device)
        self._t_ip, self._t_ix = t_ip, t_ix
        self.refresh()

    def refresh(self, values: torch.Tensor | None = None):
        if values is not None:
            self.L = self.L.with_values(values)
        abi.spx_gather_values(self.perm, self.L.values, self.lt_vals)
        return self

    def structs(self):
        lt = abi.csr_struct(self.L.n, self.L.m, self._t_ip, self._t_ix, self.lt_vals)
        return self.L.struct(), lt


class IC0:
    """Zero-fill incomplete Cholesky of every system of a batch (the IC(0) baseline)."""

    def __init__(self, batch: SystemBatch, values: torch.Tensor | None = None):
        A = batch.A
        dev = A.device
        l_ip, l_ix, self.l_src = abi.spx_tril_pattern(A.struct(), dev)
        self.Lpat = CSR(l_ip, l_ix, None, (A.m, A.m))
        self.levels = abi.spx_ic0_analyse(self.Lpat.struct(), batch.sys_ptr, batch.nsys, dev)
        self.values = torch.empty(l_ix.numel(), dtype=torch.float32, device=dev)
        self.status = torch.empty(batch.nsys, dtype=torch.int32, device=dev)
        self.t_ip, self.t_ix, self.perm = self.Lpat.transpose_pattern()
        self.lt_vals = torch.empty_like(self.values)
        self.batch = batch
        self.factor(values)

    def rebind(self, batch: SystemBatch):
        """Use this analysis (pattern, level schedule) for another batch of the same pattern
        and system partition (other values); call factor() next."""
        if batch.A.m != self.batch.A.m or batch.A.nnz != self.batch.A.nnz or \
                not np.array_equal(batch.sys_ptr_host, self.batch.sys_ptr_host):
            raise ValueError("IC0.rebind: a batch of another pattern")
        self.batch = batch
        return self

    def factor(self, values: torch.Tensor | None = None):
        A = self.batch.A
        v = A.values if values is None else values
        abi.spx_ic0_factor(self.Lpat.struct(), self.l_src, v, self.batch.nsys, self.levels, self.values,
                           self.status)
        abi.spx_gather_values(self.perm, self.values, self.lt_vals)
        return self

    def structs(self):
        n = self.batch.A.m
        return (self.Lpat.struct(self.values),
                abi.csr_struct(n, n, self.t_ip, self.t_ix, self.lt_vals))


class DiagonalFactor:
    """M = L L^T (Section 4.3) with L lower-triangular in diagonal form: per system at most
    three diagonals L_{i, i + off} (off <= 0), the values in BF16.  fill() also forms M's
    (at most four) lower diagonals (spx_dia_square); the PCG keeps each block's rows of them
    in shared memory for the whole solve and applies M in one pass (spx_cg_batched_dia).
    The analysis (offsets per system) depends on the pattern; fill() takes new values of L
    on the same pattern."""

    def __init__(self, batch: SystemBatch, Lpat: CSR):
        self.batch = batch
        self.Lpat = Lpat
        self.offsets, self.nd, self.supported = abi.spx_dia_analyse(Lpat.struct(), batch.sys_ptr, batch.nsys,
                                                                    Lpat.device)
        self.values = torch.zeros(abi.DIA_MAX * max(Lpat.m, 1), dtype=torch.bfloat16, device=Lpat.device)
        nsys = batch.nsys
        self.m_offsets = torch.zeros(max(nsys, 1) * abi.MDIA_MAX, dtype=torch.int32, device=Lpat.device)
        self.m_nd = torch.zeros(max(nsys, 1), dtype=torch.int32, device=Lpat.device)
        self.m_values = torch.zeros(abi.MDIA_MAX * max(Lpat.m, 1), dtype=torch.bfloat16, device=Lpat.device)

    def rebind(self, batch: SystemBatch):
        if batch.A.m != self.batch.A.m or not np.array_equal(batch.sys_ptr_host, self.batch.sys_ptr_host):
            raise ValueError("DiagonalFactor.rebind: a batch of another partition")
        self.batch = batch
        return self

    def fill(self, L_values: torch.Tensor):
        abi.spx_dia_fill(self.Lpat.struct(L_values), self.batch.sys_ptr, self.batch.nsys, self.offsets, self.nd,
                         self.values)
        abi.spx_dia_square(self.batch.sys_ptr, self.batch.nsys, self.Lpat.m, self.offsets, self.nd, self.values,
                           self.Lpat.device, out=(self.m_offsets, self.m_nd, self.m_values))
        return self


def cg(batch: SystemBatch, b: torch.Tensor, pc: str = "jacobi", factor: Factor | None = None,
       tol: float = 1e-8, maxit: int | None = None, delta: float = 0.1, values: torch.Tensor | None = None,
       x: torch.Tensor | None = None, M: CSR | None = None, ic0: IC0 | None = None,
       dia: DiagonalFactor | None = None):
    """Solve every system of the batch; returns (x float64, iters, status, relres) tensors.

    pc: "none", "jacobi", "llt" (factor: M = L L^T as two products), "M" (an explicit
    sparse SPD M, one product per iteration), "ic0" or "dia" (M = L L^T with L in diagonal
    form in shared memory: dia)."""
    A = batch.A
    if maxit is None:
        maxit = int(10 * np.diff(batch.sys_ptr_host).max(initial=1))
    x = x if x is not None else torch.empty(A.m, dtype=torch.float64, device=A.device)
    kind = PC[pc]
    if kind == 5:
        if dia is None:
            raise ValueError("pc='dia' needs a DiagonalFactor")
        abi.spx_cg_set_launch(*batch.launch_for(kind))
        abi.spx_cg_batched_dia(A.struct(values), batch.sys_ptr, batch.nsys, batch.order, b.contiguous(), x,
                               dia.m_offsets, dia.m_nd, dia.m_values, tol, maxit, delta, batch.iters, batch.status,
                               batch.relres, batch.ws)
        return x, batch.iters, batch.status, batch.relres
    dinv = batch.dinv(values) if kind == 1 else None
    L = LT = None
    if kind == 2:
        if factor is None:
            raise ValueError("pc='llt' needs a Factor")
        L, LT = factor.structs()
    if kind == 3:
        if M is None:
            raise ValueError("pc='M' needs M")
        L = M.struct()
    levels = None
    if kind == 4:
        if ic0 is None:
            raise ValueError("pc='ic0' needs an IC0")
        L, LT = ic0.structs()
        levels = ic0.levels
    abi.spx_cg_set_launch(*batch.launch_for(kind))
    abi.spx_cg_batched(A.struct(values), batch.sys_ptr, batch.nsys, batch.order, b.contiguous(), x, kind,
                       dinv, L, LT, tol, maxit, delta, batch.iters, batch.status, batch.relres, batch.ws,
                       ic0_levels=levels)
    return x, batch.iters, batch.status, batch.relres


class Solve(torch.autograd.Function):
    """x = A^{-1} b for a batch of SPD systems (float32 values and b, float64 x).
    Backward (Table 1, SpSolve): lam = A^{-T} v by the same PCG, grad_b = lam,
    grad_A = -(lam x^T) masked to mask(A)."""

    @staticmethod
    def forward(ctx, values, b, batch, pc="jacobi", tol=1e-8, maxit=None):
        x, _, status, _ = cg(batch, b, pc=pc, tol=tol, maxit=maxit, values=values)
        ctx.batch, ctx.pc, ctx.tol, ctx.maxit = batch, pc, tol, maxit
        ctx.save_for_backward(values, x)
        return x

    @staticmethod
    def backward(ctx, v):
        values, x = ctx.saved_tensors
        batch = ctx.batch
        lam, _, _, _ = cg(batch, v.to(torch.float32).contiguous(), pc=ctx.pc, tol=ctx.tol, maxit=ctx.maxit,
                          values=values)
        g_vals = None
        if ctx.needs_input_grad[0]:
            g_vals = torch.empty(batch.A.nnz, dtype=torch.float32, device=values.device)
            abi.spx_masked_outer_f64(batch.A.struct(values), lam, x, g_vals, -1.0)
        g_b = lam.to(torch.float32) if ctx.needs_input_grad[1] else None
        return g_vals, g_b, None, None, None, None
