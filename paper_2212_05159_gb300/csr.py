"""Device CSR matrix with per-pattern caches (transpose, load-balancing plans).

The pattern (indptr, indices) is fixed for the life of the object; the values may be
swapped (e.g. learned values) without invalidating the caches, because the transpose
and the row plans depend only on the pattern (Section 3.1: gradients live on the
input's pattern, so the pattern is known a priori).
"""
from __future__ import annotations

import numpy as np
import torch

from . import abi

LONG_ROW_THRESHOLD = 256
MEDIUM_ROW_THRESHOLD = 32


class CSR:
    """An m x n CSR matrix on a CUDA device (int32 pattern, float32 values)."""

    def __init__(self, indptr: torch.Tensor, indices: torch.Tensor, values: torch.Tensor | None,
                 shape: tuple[int, int]):
        self.indptr = indptr.to(torch.int32).contiguous()
        self.indices = indices.to(torch.int32).contiguous()
        self.values = None if values is None else values.to(torch.float32).contiguous()
        self.shape = (int(shape[0]), int(shape[1]))
        self.device = self.indptr.device
        self._plan = None
        self._t = None
        self._t_plan = None
        self._parts = {}
        self._t_parts = {}
        self._merge = {}
        self._t_merge = {}

    # ------------------------------------------------------------------ construction
    @classmethod
    def from_host(cls, A, device="cuda") -> "CSR":
        """From any object with m, n, indptr, indices, values (numpy arrays)."""
        ip = torch.from_numpy(np.ascontiguousarray(A.indptr, dtype=np.int32)).to(device)
        ix = torch.from_numpy(np.ascontiguousarray(A.indices, dtype=np.int32)).to(device)
        v = torch.from_numpy(np.ascontiguousarray(A.values, dtype=np.float32)).to(device)
        return cls(ip, ix, v, (A.m, A.n))

    def with_values(self, values: torch.Tensor) -> "CSR":
        """Same pattern (and caches), other values."""
        other = CSR.__new__(CSR)
        other.__dict__.update(self.__dict__)
        other.values = values.to(torch.float32).contiguous()
        return other

    @property
    def m(self):
        return self.shape[0]

    @property
    def n(self):
        return self.shape[1]

    @property
    def nnz(self):
        return int(self.indices.numel())

    def struct(self, values: torch.Tensor | None = None) -> abi.spx_csr:
        v = self.values if values is None else values
        return abi.csr_struct(self.m, self.n, self.indptr, self.indices, v)

    def validate(self) -> None:
        abi.spx_csr_validate(self.struct(), self.device)

    # ------------------------------------------------------------------ caches
    def plan(self):
        if self._plan is None:
            rows, plan = abi.spx_rowplan_build(self.struct(), LONG_ROW_THRESHOLD, self.device,
                                               MEDIUM_ROW_THRESHOLD)
            self._plan = (rows, plan)
        return self._plan[1]

    def parts(self, n_parts: int):
        """Column-range split of the rows into n_parts segments (cached per count)."""
        if n_parts <= 1:
            return None
        cache = self._parts
        if n_parts not in cache:
            cache[n_parts] = abi.spx_rowplan_build_parts(self.struct(), n_parts, self.device)
        return cache[n_parts]

    def t_parts(self, n_parts: int):
        """The same split for A^T (rows of A^T split by A's row ranges)."""
        if n_parts <= 1:
            return None
        cache = self._t_parts
        if n_parts not in cache:
            t_ip, t_ix, _ = self.transpose_pattern()
            st = abi.csr_struct(self.n, self.m, t_ip, t_ix, None)
            cache[n_parts] = abi.spx_rowplan_build_parts(st, n_parts, self.device)
        return cache[n_parts]

    def transpose_pattern(self):
        """(t_indptr, t_indices, perm) of A^T, computed once per pattern."""
        if self._t is None:
            self._t = abi.spx_csr_transpose(self.struct(), self.device)
        return self._t

    def t_struct(self, values: torch.Tensor | None = None) -> abi.spx_csr:
        """Pattern of A^T whose value pointer is A's values (gathered through perm)."""
        t_ip, t_ix, _ = self.transpose_pattern()
        v = self.values if values is None else values
        return abi.csr_struct(self.n, self.m, t_ip, t_ix, v)

    def t_plan(self):
        if self._t_plan is None:
            t_ip, t_ix, _ = self.transpose_pattern()
            st = abi.csr_struct(self.n, self.m, t_ip, t_ix, None)
            self._t_plan = abi.spx_rowplan_build(st, LONG_ROW_THRESHOLD, self.device, MEDIUM_ROW_THRESHOLD)
        return self._t_plan[1]

    def merge_plan(self, items: int):
        """Merge-path segments of `items` rows + entries (cached per size)."""
        if items not in self._merge:
            self._merge[items] = abi.spx_merge_plan_build(
                abi.csr_struct(self.m, self.n, self.indptr, self.indices, None), items, self.device)
        return self._merge[items][1]

    def t_merge_plan(self, items: int):
        """The same for A^T's pattern."""
        if items not in self._t_merge:
            t_ip, t_ix, _ = self.transpose_pattern()
            self._t_merge[items] = abi.spx_merge_plan_build(abi.csr_struct(self.n, self.m, t_ip, t_ix, None), items,
                                                            self.device)
        return self._t_merge[items][1]

    def diagonal_positions(self) -> torch.Tensor:
        """int32[min(m, n)]: index of entry (i, i) in indices / values, -1 if absent (cached)."""
        if getattr(self, "_diag_pos", None) is None:
            nd = min(self.m, self.n)
            pos = torch.empty(max(nd, 1), dtype=torch.int32, device=self.device)[:nd]
            abi.spx_csr_diagonal(abi.csr_struct(self.m, self.n, self.indptr, self.indices, None), None, pos)
            self._diag_pos = pos
        return self._diag_pos

    def inverse_transpose_perm(self) -> torch.Tensor:
        """The inverse of transpose_pattern()'s permutation: A.values = A^T.values[inv]."""
        if getattr(self, "_t_inv", None) is None:
            t_ip, t_ix, _ = self.transpose_pattern()
            _, _, inv = abi.spx_csr_transpose(abi.csr_struct(self.n, self.m, t_ip, t_ix, None), self.device)
            self._t_inv = inv
        return self._t_inv

    # ------------------------------------------------------------------ the paper's operator syntax
    def __matmul__(self, other):
        """A @ X for a dense 1-D or 2-D X (Section 3.1.1 / 3.1.3, differentiable in A's values
        and X) or A @ B for a CSR B (Section 3.1.2: the structural pattern, differentiable in
        both value arrays; the pattern is analysed on every call -- keep an ops.SpGEMMPlan to
        reuse it)."""
        from . import autograd
        if isinstance(other, CSR):
            from .ops import SpGEMMPlan
            plan = SpGEMMPlan(self, other)
            return plan.C.with_values(autograd.SpGEMM.apply(self.values, other.values, plan))
        return autograd.spmm(self, other)

    def __add__(self, other):
        """A + B for a CSR B of the same shape (Section 3.1.4): the union pattern, differentiable
        in both value arrays (dA = V masked to A, dB = V masked to B).  The pattern is analysed on
        every call -- keep an ops.SpAddPlan to reuse it."""
        return self._add(other, 1.0)

    def __sub__(self, other):
        """A - B, as A + (-1) B."""
        return self._add(other, -1.0)

    def _add(self, other, beta: float):
        if not isinstance(other, CSR):
            return NotImplemented
        from . import autograd
        from .ops import SpAddPlan
        plan = SpAddPlan(self, other)
        return plan.C.with_values(autograd.SpAdd.apply(self.values, other.values, plan, 1.0, beta))

    @property
    def T(self) -> "CSR":
        """A^T: the cached transposed pattern with A's values gathered through its
        permutation (differentiable: the gradient returns through the inverse permutation)."""
        from . import autograd
        t_ip, t_ix, perm = self.transpose_pattern()
        inv = self.inverse_transpose_perm()
        out = CSR(t_ip, t_ix, None, (self.n, self.m))
        out._t = (self.indptr, self.indices, inv)
        out._t_inv = perm
        if self.values is not None:
            out.values = autograd.Permute.apply(self.values, perm, inv)
        return out

    def diagonal(self) -> torch.Tensor:
        """The diagonal, length min(m, n), 0 where a row stores no diagonal entry;
        differentiable in A's values (the gradient lands on the stored entries (i, i))."""
        from . import autograd
        return autograd.Diagonal.apply(self.values, self)

    def __repr__(self):
        return f"CSR({self.m}x{self.n}, nnz={self.nnz}, device={self.device})"
