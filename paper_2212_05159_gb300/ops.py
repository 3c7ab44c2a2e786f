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
        abi.spx_sddmm(st, G2, X2, o, scale, 0, ws)
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
