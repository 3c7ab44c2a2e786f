"""Functional forms of the sparse kernels on :class:`CSR` matrices.

Each function allocates its output with torch (device memory only) and calls one
C-ABI entry point; all arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import abi
from .csr import CSR


def _workspace(nbytes: int, device):
    return abi.workspace(nbytes, device) if nbytes > 0 else None


def _as2d(t: torch.Tensor):
    return (t.unsqueeze(1), True) if t.dim() == 1 else (t, False)


def spmm(A: CSR, X: torch.Tensor, values: torch.Tensor | None = None, out=None,
         alpha: float = 1.0, beta: float = 0.0, use_plan: bool = True) -> torch.Tensor:
    """Y = alpha * A X + beta * out (Section 3.1.1 / 3.1.3); X 1-D gives SpMV."""
    X2, vec = _as2d(X)
    Y = out if out is not None else torch.empty(A.m, X2.shape[1], dtype=torch.float32, device=X.device)
    Y2, _ = _as2d(Y)
    st = A.struct(values)
    plan = A.plan() if use_plan else None
    ws = _workspace(abi.spx_spmm_workspace_size(st, X2.shape[1], plan), X.device)
    abi.spx_spmm(st, X2, Y2, alpha, beta, plan, ws)
    return Y2.squeeze(1) if vec else Y2


def sddmm(A: CSR, G: torch.Tensor, X: torch.Tensor, scale: float = 1.0, out=None) -> torch.Tensor:
    """Values on mask(A) of scale * G X^T (Table 1, gradient w.r.t. A)."""
    G2, _ = _as2d(G)
    X2, _ = _as2d(X)
    o = out if out is not None else torch.empty(A.nnz, dtype=torch.float32, device=G.device)
    if G2.shape[1] == 1 and G2.is_contiguous() and X2.is_contiguous():
        abi.spx_masked_outer(A.struct(), G2, X2, o, scale)
    else:
        st = A.struct()
        ws = _workspace(abi.spx_sddmm_workspace_size(st, G2.shape[1]), G.device)
        abi.spx_sddmm(st, G2, X2, o, scale, 0, ws, plan=A.plan())
    return o


def masked_outer(A: CSR, u: torch.Tensor, v: torch.Tensor, scale: float = 1.0, out=None):
    """scale * u v^T on mask(A) (k = 1 SDDMM)."""
    o = out if out is not None else torch.empty(A.nnz, dtype=torch.float32, device=u.device)
    abi.spx_masked_outer(A.struct(), u.contiguous(), v.contiguous(), o, scale)
    return o


def spmm_t(A: CSR, G: torch.Tensor, values: torch.Tensor | None = None, out=None,
           alpha: float = 1.0, beta: float = 0.0, use_plan: bool = True) -> torch.Tensor:
    """gX = alpha * A^T G + beta * out (Table 1, gradient w.r.t. the dense operand)."""
    G2, vec = _as2d(G)
    gX = out if out is not None else torch.empty(A.n, G2.shape[1], dtype=torch.float32, device=G.device)
    gX2, _ = _as2d(gX)
    _, _, perm = A.transpose_pattern()
    st = A.t_struct(values)
    plan = A.t_plan() if use_plan else None
    ws = _workspace(abi.spx_spmm_t_workspace_size(st, G2.shape[1], plan), G.device)
    abi.spx_spmm_t(st, perm, G2, gX2, alpha, beta, plan, ws)
    return gX2.squeeze(1) if vec else gX2


def spmm_backward(A: CSR, G: torch.Tensor, X: torch.Tensor, values: torch.Tensor | None = None):
    """(gA, gX) of Y = A X for the upstream gradient G: gA = (G X^T) on mask(A) and gX = A^T G
    (Table 1).  Widths k that are multiples of 4 up to 128 (with aligned rows) take one pass
    over A^T that gathers each row of G once for both (spx_spmm_t_sddmm); others the two
    products apart."""
    G2, vec = _as2d(G)
    X2, _ = _as2d(X)
    k = G2.shape[1]
    aligned = all(t.is_contiguous() and t.data_ptr() % 16 == 0 for t in (G2, X2))
    if k % 4 == 0 and 4 <= k <= 128 and aligned:
        v = A.values if values is None else values
        t_ip, t_ix, perm = A.transpose_pattern()
        gX = torch.empty(A.n, k, dtype=torch.float32, device=G.device)
        gA = torch.empty(A.nnz, dtype=torch.float32, device=G.device)
        abi.spx_spmm_t_sddmm(abi.csr_struct(A.n, A.m, t_ip, t_ix, None), perm, v, G2, X2, gX, gA,
                             plan=A.t_plan())
        return gA, (gX.squeeze(1) if vec else gX)
    return sddmm(A, G, X), spmm_t(A, G, values=values)


class SpGEMMPlan:
    """Pattern of C = A B and the per-row classes, built once per (pattern A, pattern B)."""

    def __init__(self, A: CSR, B: CSR):
        if A.n != B.m:
            raise ValueError("inner dimensions differ")
        self.A, self.B = A, B
        dev = A.device
        sA, sB = A.struct(), B.struct()
        self.ws = abi.workspace(abi.spx_spgemm_workspace_size(A.m), dev)
        self.products = abi.spx_spgemm_analyse(sA, sB, self.ws)
        scratch = abi.workspace(4 * self.products, dev)
        c_ip = torch.empty(A.m + 1, dtype=torch.int32, device=dev)
        nnz = abi.spx_spgemm_symbolic(sA, sB, c_ip, self.ws, scratch, self.products)
        c_ix = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
        abi.spx_spgemm_fill(sA, c_ip, c_ix, self.ws, scratch)
        del scratch
        self.C = CSR(c_ip, c_ix[:nnz], None, (A.m, B.n))

    def numeric(self, a_values=None, b_values=None, out=None) -> torch.Tensor:
        o = out if out is not None else torch.empty(self.C.nnz, dtype=torch.float32, device=self.A.device)
        abi.spx_spgemm_numeric(self.A.struct(a_values), self.B.struct(b_values), self.C.struct(), o, self.ws)
        return o

    def backward(self, gc: torch.Tensor, a_values=None, b_values=None, need_a=True, need_b=True):
        dev = self.A.device
        ga = torch.empty(self.A.nnz, dtype=torch.float32, device=dev) if need_a else None
        gb = torch.empty(self.B.nnz, dtype=torch.float32, device=dev) if need_b else None
        t_ip = t_ix = perm = None
        if need_b:
            t_ip, t_ix, perm = self.A.transpose_pattern()
        abi.spx_spgemm_backward(self.A.struct(a_values), self.B.struct(b_values), self.C.struct(),
                                gc.contiguous(), ga, gb, t_ip, t_ix, perm)
        return ga, gb


class TriangularSolver:
    """Level schedule and transpose of a block-diagonal batch of lower-triangular patterns
    (Section 3.1.5), built once per pattern; solves L x = b and L^T y = v on the device."""

    def __init__(self, L: CSR, sys_ptr):
        if L.m != L.n:
            raise ValueError("L must be square")
        self.L = L
        dev = L.device
        ptr_t = sys_ptr if isinstance(sys_ptr, torch.Tensor) else torch.as_tensor(sys_ptr, dtype=torch.int32)
        self.sys_ptr = ptr_t.to(device=dev, dtype=torch.int32)
        self.nsys = int(self.sys_ptr.numel()) - 1
        self.levels = abi.spx_ic0_analyse(L.struct(), self.sys_ptr, self.nsys, dev)
        self.t_ip, self.t_ix, self.perm = L.transpose_pattern()
        self.status = torch.zeros(self.nsys, dtype=torch.int32, device=dev)

    def solve(self, b: torch.Tensor, values: torch.Tensor | None = None, transpose: bool = False,
              out: torch.Tensor | None = None) -> torch.Tensor:
        v = self.L.values if values is None else values
        x = out if out is not None else torch.empty_like(b)
        if transpose:
            lt = torch.empty_like(v)
            abi.spx_gather_values(self.perm, v, lt)
            T = abi.csr_struct(self.L.n, self.L.m, self.t_ip, self.t_ix, lt)
        else:
            T = self.L.struct(v)
        abi.spx_sptrsv(T, transpose, self.nsys, self.levels, b.contiguous(), x, self.status)
        return x


class SpAddPlan:
    """Pattern of C = alpha A + beta B -- the union of the stored patterns, row by row
    (Section 3.1.4) -- and the maps between the three patterns, built once per pair."""

    def __init__(self, A: CSR, B: CSR):
        if A.shape != B.shape:
            raise ValueError("shapes differ")
        self.A, self.B = A, B
        dev = A.device
        i32 = dict(dtype=torch.int32, device=dev)
        c_ip = torch.empty(A.m + 1, **i32)
        nnz = abi.spx_spadd_symbolic(A.struct(), B.struct(), c_ip, dev)
        c_ix = torch.empty(max(nnz, 1), **i32)
        self.src_a = torch.empty(max(nnz, 1), **i32)
        self.src_b = torch.empty(max(nnz, 1), **i32)
        self.pos_a = torch.empty(max(A.nnz, 1), **i32)
        self.pos_b = torch.empty(max(B.nnz, 1), **i32)
        abi.spx_spadd_fill(A.struct(), B.struct(), c_ip, c_ix, self.src_a, self.src_b, self.pos_a, self.pos_b)
        self.src_a, self.src_b = self.src_a[:nnz], self.src_b[:nnz]
        self.pos_a, self.pos_b = self.pos_a[:A.nnz], self.pos_b[:B.nnz]
        self.C = CSR(c_ip, c_ix[:nnz], None, A.shape)

    def numeric(self, alpha=1.0, beta=1.0, a_values=None, b_values=None, out=None) -> torch.Tensor:
        a = self.A.values if a_values is None else a_values
        b = self.B.values if b_values is None else b_values
        o = out if out is not None else torch.empty(self.C.nnz, dtype=torch.float32, device=self.A.device)
        abi.spx_spadd_numeric(alpha, a, self.src_a, beta, b, self.src_b, o)
        return o

    def backward(self, gc: torch.Tensor, alpha=1.0, beta=1.0, need_a=True, need_b=True):
        dev = self.A.device
        ga = torch.empty(self.A.nnz, dtype=torch.float32, device=dev) if need_a else None
        gb = torch.empty(self.B.nnz, dtype=torch.float32, device=dev) if need_b else None
        abi.spx_spadd_backward(alpha, beta, gc.contiguous(), self.pos_a, self.pos_b, ga, gb)
        return ga, gb


def spadd(A: CSR, B: CSR, alpha: float = 1.0, beta: float = 1.0) -> CSR:
    """C = alpha A + beta B with the union pattern (Section 3.1.4)."""
    plan = SpAddPlan(A, B)
    return plan.C.with_values(plan.numeric(alpha, beta))


def spgemm(A: CSR, B: CSR) -> CSR:
    """C = A B with the structural pattern (Section 3.1.2)."""
    plan = SpGEMMPlan(A, B)
    return plan.C.with_values(plan.numeric())
