"""Multi-rank partitioning of the hot path (one process per GPU, torch.distributed).

The paper runs on one GPU; these are the partitions for several, and the only exchanges
they need:

  SpMM / SDDMM / A^T G (Table 1, SpDMM rows).  A is split into contiguous row blocks
  holding about the same number of stored entries (power-law rows make equal row counts
  badly unbalanced); rank r owns rows [r0, r1) of A, Y, G and gA, and a contiguous slice of
  X's rows (and of gX).
    forward   Y_r = A_r X            one all-gather of X before the product
    SDDMM     gA_r = (G_r X^T) on A_r's mask   X as gathered for the forward: no exchange
    A^T G     gX = sum_r A_r^T G_r   each rank forms its n x k partial; one reduce-scatter
                                     sums the partials and leaves each rank its slice of gX
  Batched PCG (Section 4.3 solves).  Systems are independent: they are split over the ranks
  by estimated cost (rows x expected iterations, largest first onto the least loaded rank),
  with no exchange.
  Network training (the learned preconditioner).  Data-parallel: each rank trains on its
  own batches and the parameter gradients are summed by one all-reduce before the optimiser
  step.

The orchestration takes the local products as callables, so the same code drives the
library's CUDA kernels over NCCL or any CPU implementation over gloo.  Every function here
moves data; the arithmetic of the products is the callables'.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def row_blocks_by_nnz(indptr, parts: int) -> np.ndarray:
    """Boundaries b[0..parts] of contiguous row blocks: block p = rows [b[p], b[p+1]) ends at
    the first row boundary where the prefix count of entries reaches (p + 1) nnz / parts, so
    a block holds at most nnz / parts entries plus one row's."""
    ip = np.asarray(indptr, np.int64)
    m = ip.size - 1
    nnz = int(ip[-1])
    b = np.zeros(parts + 1, np.int64)
    b[parts] = m
    for p in range(1, parts):
        cut = int(np.searchsorted(ip, (nnz * p) // parts, side="left"))
        b[p] = min(max(cut, int(b[p - 1])), m)
    return b


def even_slices(n: int, parts: int) -> np.ndarray:
    """Boundaries of `parts` contiguous slices of n rows of (nearly) equal size."""
    return np.array([(n * p) // parts for p in range(parts + 1)], np.int64)


def _padded(t: torch.Tensor, rows: int) -> torch.Tensor:
    if t.shape[0] == rows:
        return t.contiguous()
    out = torch.zeros((rows,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    out[: t.shape[0]] = t
    return out


def all_gather_rows(owned: torch.Tensor, bounds: np.ndarray, group=None) -> torch.Tensor:
    """The full matrix from every rank's slice of rows (bounds: even_slices)."""
    world = dist.get_world_size(group)
    chunk = int(max(bounds[p + 1] - bounds[p] for p in range(world)))
    parts = [torch.empty((chunk,) + tuple(owned.shape[1:]), dtype=owned.dtype, device=owned.device)
             for _ in range(world)]
    dist.all_gather(parts, _padded(owned, chunk), group=group)
    return torch.cat([parts[p][: bounds[p + 1] - bounds[p]] for p in range(world)], dim=0)


def reduce_scatter_rows(partial: torch.Tensor, bounds: np.ndarray, group=None) -> torch.Tensor:
    """The sum over ranks of `partial` (every rank's full-size contribution), of which this
    rank keeps its slice of rows.  Summed by the backend's reduce-scatter where it has one,
    else by an all-reduce of which the slice is kept (same sums)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    chunk = int(max(bounds[p + 1] - bounds[p] for p in range(world)))
    pieces = [_padded(partial[bounds[p]:bounds[p + 1]], chunk) for p in range(world)]
    out = torch.empty((chunk,) + tuple(partial.shape[1:]), dtype=partial.dtype, device=partial.device)
    try:
        dist.reduce_scatter(out, pieces, group=group)
    except (RuntimeError, NotImplementedError, ValueError):
        full = torch.cat(pieces, dim=0)
        dist.all_reduce(full, group=group)
        out = full[rank * chunk:(rank + 1) * chunk]
    return out[: bounds[rank + 1] - bounds[rank]]


class RowSharded:
    """Rank `rank`'s share of a sparse m x n matrix for the three products of a step."""

    def __init__(self, indptr, m: int, n: int, group=None):
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.rows = row_blocks_by_nnz(indptr, self.world)
        self.cols = even_slices(n, self.world)
        self.m, self.n = m, n
        self.r0, self.r1 = int(self.rows[self.rank]), int(self.rows[self.rank + 1])
        self.c0, self.c1 = int(self.cols[self.rank]), int(self.cols[self.rank + 1])

    def forward(self, local_spmm, X_owned: torch.Tensor):
        """(Y_r, X): the gathered X is returned for the SDDMM of the reverse pass."""
        X = all_gather_rows(X_owned, self.cols, self.group)
        return local_spmm(X), X

    def backward(self, local_sddmm, local_spmm_t, G_r: torch.Tensor, X: torch.Tensor):
        """(gA_r on A_r's entries, this rank's slice of gX)."""
        gA = local_sddmm(G_r, X)
        gX = reduce_scatter_rows(local_spmm_t(G_r), self.cols, self.group)
        return gA, gX


def allreduce_gradients(grad: torch.Tensor, group=None) -> torch.Tensor:
    """Data-parallel training: the sum of every rank's parameter gradient, in place."""
    dist.all_reduce(grad, group=group)
    return grad


def partition_systems(costs, parts: int) -> list[list[int]]:
    """Independent systems onto `parts` ranks: largest estimated cost first, each onto the
    least loaded rank (ties to the lower rank); returns the system ids of every rank."""
    costs = np.asarray(costs, np.float64)
    order = np.argsort(-costs, kind="stable")
    load = np.zeros(parts)
    out = [[] for _ in range(parts)]
    for s in order:
        p = int(np.argmin(load))
        out[p].append(int(s))
        load[p] += costs[s]
    return [sorted(x) for x in out]
