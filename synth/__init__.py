"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only *generates* inputs: sparsity patterns, matrix values and dense
operands.  It contains none of the arithmetic of the sparse operations themselves,
so both sides of a parity test can draw from it without sharing method code.

Every generator returns plain numpy arrays.  CSR triples are
``(indptr int32[m+1], indices int32[nnz], values float32[nnz])`` with column
indices sorted and unique within each row; float32 values are what the GPU path
consumes and the FP64 oracle promotes them exactly.

Workload recipes (see the model problems of Section 4 of the paper, Eq. for A_N and
its 2D Kronecker sum):

* ``poisson1d(N)``      -- the tridiagonal [-1 2 -1] matrix A_N.
* ``poisson2d(nx, ny)`` -- A_{nx x ny} = A_nx (x) I_ny + I_nx (x) A_ny (5-point).
* ``poisson3d(n)``      -- the 3D analogue (7-point stencil, n^3 rows).
* ``powerlaw_csr``      -- random rows with a power-law length tail (exponent 1.5,
  minimum scale 5.62 so the mean is 16 at n = 2^20, lengths capped at 4096),
  columns uniform and unique per row, values N(0,1).
* ``random_k_per_row``  -- exactly k uniform unique columns per row, values U(-1,1).
* ``diffusion2d``       -- variable-coefficient 5-point diffusion on an s x s grid:
  cell coefficients log-normal exp(sigma * N(0,1)), face weights the harmonic mean
  of the two cells, boundary faces (Dirichlet 0) weighted by the cell's own
  coefficient; symmetric positive definite and diagonally dominant.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "CSR", "poisson1d", "poisson2d", "poisson3d", "powerlaw_csr", "random_k_per_row",
    "diffusion2d", "diffusion_batch", "block_diag", "normal", "uniform", "with_values",
    "empty_rows_csr", "from_dense",
]


class CSR:
    """A host CSR matrix: ``indptr``/``indices`` int32, ``values`` float32."""

    __slots__ = ("m", "n", "indptr", "indices", "values")

    def __init__(self, m, n, indptr, indices, values):
        self.m = int(m)
        self.n = int(n)
        self.indptr = np.ascontiguousarray(indptr, dtype=np.int32)
        self.indices = np.ascontiguousarray(indices, dtype=np.int32)
        self.values = np.ascontiguousarray(values, dtype=np.float32)
        assert self.indptr.shape == (self.m + 1,)
        assert self.indices.shape == self.values.shape == (int(self.indptr[-1]),)

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    @property
    def shape(self):
        return (self.m, self.n)

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.indptr.astype(np.int64))

    def to_dense(self) -> np.ndarray:
        """Dense float64 copy (small matrices only)."""
        d = np.zeros((self.m, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.m), self.row_lengths())
        d[rows, self.indices] = self.values.astype(np.float64)
        return d

    def __repr__(self):
        return f"CSR({self.m}x{self.n}, nnz={self.nnz})"


def _from_coo_sorted(m, n, rows, cols, vals) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=m).astype(np.int64)
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    return CSR(m, n, indptr, cols, vals)


def from_dense(d: np.ndarray) -> CSR:
    """CSR of the nonzero entries of a small dense array."""
    d = np.asarray(d)
    rows, cols = np.nonzero(d)
    return _from_coo_sorted(d.shape[0], d.shape[1], rows, cols, d[rows, cols])


def with_values(A: CSR, values) -> CSR:
    return CSR(A.m, A.n, A.indptr, A.indices, values)


def normal(shape, seed: int, dtype=np.float32) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def uniform(shape, seed: int, lo=-1.0, hi=1.0, dtype=np.float32) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, shape).astype(dtype)


def poisson1d(N: int) -> CSR:
    """A_N: tridiagonal with 2 on the diagonal and -1 off it (Section 4, Eq. for A_N)."""
    i = np.arange(N)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[1:] - 1, i[:-1] + 1])
    vals = np.concatenate([np.full(N, 2.0), np.full(N - 1, -1.0), np.full(N - 1, -1.0)])
    return _from_coo_sorted(N, N, rows, cols, vals)


def poisson2d(nx: int, ny: int | None = None) -> CSR:
    """A_{nx x ny} = A_nx (x) I_ny + I_nx (x) A_ny, row index ix*ny + iy (Section 4)."""
    ny = nx if ny is None else ny
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    ix, iy = ix.ravel(), iy.ravel()
    idx = ix * ny + iy
    rows = [idx]
    cols = [idx]
    vals = [np.full(idx.size, 4.0)]
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        jx, jy = ix + dx, iy + dy
        ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny)
        rows.append(idx[ok])
        cols.append((jx * ny + jy)[ok])
        vals.append(np.full(int(ok.sum()), -1.0))
    return _from_coo_sorted(nx * ny, nx * ny, np.concatenate(rows), np.concatenate(cols),
                            np.concatenate(vals))


def poisson3d(n: int) -> CSR:
    """7-point 3D Poisson on an n^3 grid: the 3D Kronecker sum of A_n (row index (ix*n+iy)*n+iz)."""
    N = n * n * n
    idx = np.arange(N, dtype=np.int64)
    iz = idx % n
    iy = (idx // n) % n
    ix = idx // (n * n)
    rows = [idx]
    cols = [idx]
    vals = [np.full(N, 6.0)]
    for d, comp, stride in ((-1, ix, n * n), (1, ix, n * n), (-1, iy, n), (1, iy, n),
                            (-1, iz, 1), (1, iz, 1)):
        ok = (comp + d >= 0) & (comp + d < n)
        rows.append(idx[ok])
        cols.append(idx[ok] + d * stride)
        vals.append(np.full(int(ok.sum()), -1.0))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return _from_coo_sorted(N, N, rows, cols, vals)


def _unique_sorted_columns(lengths: np.ndarray, ncols: int, rng) -> np.ndarray:
    """Per row, ``lengths[i]`` distinct uniform columns in [0, ncols), sorted."""
    m = lengths.size
    assert int(lengths.max(initial=0)) <= ncols
    dense = lengths * 4 > ncols                 # near-full rows: draw without replacement
    if dense.any():
        out = np.zeros(int(lengths.sum()), dtype=np.int32)
        offs = np.zeros(m + 1, dtype=np.int64)
        np.cumsum(lengths, out=offs[1:])
        sparse_cols = _unique_sorted_columns(np.where(dense, 0, lengths), ncols, rng)
        sp_offs = np.zeros(m + 1, dtype=np.int64)
        np.cumsum(np.where(dense, 0, lengths), out=sp_offs[1:])
        for i in range(m):
            if dense[i]:
                out[offs[i]:offs[i + 1]] = np.sort(rng.choice(ncols, int(lengths[i]), replace=False))
            else:
                out[offs[i]:offs[i + 1]] = sparse_cols[sp_offs[i]:sp_offs[i + 1]]
        return out
    rows = np.repeat(np.arange(m, dtype=np.int64), lengths)
    cols = rng.integers(0, ncols, size=rows.size, dtype=np.int64)
    for _ in range(64):
        key = rows * ncols + cols
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(ks.size, dtype=bool)
        dup[1:] = ks[1:] == ks[:-1]
        if not dup.any():
            return cols[order].astype(np.int32)
        cols_sorted = cols[order]
        cols_sorted[dup] = rng.integers(0, ncols, size=int(dup.sum()), dtype=np.int64)
        rows = rows[order]
        cols = cols_sorted
    raise RuntimeError("could not draw unique columns")


def powerlaw_csr(n: int, seed: int, kmin: float = 5.62, exponent: float = 1.5,
                 max_len: int = 4096, ncols: int | None = None) -> CSR:
    """Random CSR with power-law row lengths min(max_len, floor(kmin * U^(-1/exponent)))."""
    ncols = n if ncols is None else ncols
    rng = np.random.default_rng(seed)
    u = 1.0 - rng.random(n)                     # U in (0, 1]
    lengths = np.minimum(np.minimum(max_len, ncols),
                         np.floor(kmin * u ** (-1.0 / exponent))).astype(np.int64)
    cols = _unique_sorted_columns(lengths, ncols, rng)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=indptr[1:])
    vals = rng.standard_normal(cols.size).astype(np.float32)
    return CSR(n, ncols, indptr, cols, vals)


def random_k_per_row(n: int, k: int, seed: int, ncols: int | None = None) -> CSR:
    """Exactly k distinct uniform columns per row, values U(-1, 1)."""
    ncols = n if ncols is None else ncols
    rng = np.random.default_rng(seed)
    lengths = np.full(n, k, dtype=np.int64)
    cols = _unique_sorted_columns(lengths, ncols, rng)
    indptr = np.arange(n + 1, dtype=np.int64) * k
    vals = rng.uniform(-1.0, 1.0, cols.size).astype(np.float32)
    return CSR(n, ncols, indptr, cols, vals)


def empty_rows_csr(m: int, n: int, seed: int, p_empty: float = 0.3, max_len: int = 40) -> CSR:
    """Ragged test matrix: a fraction of empty rows, one hub row, lengths 0..max_len."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, max_len + 1, size=m)
    lengths[rng.random(m) < p_empty] = 0
    if m > 2:
        lengths[m // 2] = min(n, 40 * max_len)      # one long hub row
    lengths = np.minimum(lengths, n).astype(np.int64)
    cols = _unique_sorted_columns(lengths, n, rng)
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=indptr[1:])
    vals = rng.standard_normal(cols.size).astype(np.float32)
    return CSR(m, n, indptr, cols, vals)


def diffusion2d(s: int, sigma: float, seed: int) -> CSR:
    """Variable-coefficient 2D diffusion, 5-point, s x s cells, Dirichlet 0 boundary.

    Coefficient per cell c = exp(sigma * N(0,1)); the weight of an interior face is the
    harmonic mean 2 c1 c2 / (c1 + c2); a boundary face is weighted by the cell's own c.
    Row (ix, iy) -> ix * s + iy; A_ii = sum of the cell's face weights, A_ij = -w_ij.
    """
    rng = np.random.default_rng(seed)
    c = np.exp(sigma * rng.standard_normal((s, s)))
    wx = 2.0 * c[1:, :] * c[:-1, :] / (c[1:, :] + c[:-1, :])    # faces between ix and ix+1
    wy = 2.0 * c[:, 1:] * c[:, :-1] / (c[:, 1:] + c[:, :-1])    # faces between iy and iy+1
    diag = np.zeros((s, s))
    diag[1:, :] += wx
    diag[:-1, :] += wx
    diag[:, 1:] += wy
    diag[:, :-1] += wy
    diag[0, :] += c[0, :]
    diag[-1, :] += c[-1, :]
    diag[:, 0] += c[:, 0]
    diag[:, -1] += c[:, -1]
    idx = np.arange(s * s).reshape(s, s)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [diag.ravel()]
    # x-neighbours
    rows += [idx[1:, :].ravel(), idx[:-1, :].ravel()]
    cols += [idx[:-1, :].ravel(), idx[1:, :].ravel()]
    vals += [-wx.ravel(), -wx.ravel()]
    rows += [idx[:, 1:].ravel(), idx[:, :-1].ravel()]
    cols += [idx[:, :-1].ravel(), idx[:, 1:].ravel()]
    vals += [-wy.ravel(), -wy.ravel()]
    return _from_coo_sorted(s * s, s * s, np.concatenate(rows), np.concatenate(cols),
                            np.concatenate(vals))


def block_diag(mats) -> tuple[CSR, np.ndarray]:
    """Block-diagonal concatenation; returns (CSR, sys_ptr int32[B+1]) with row offsets."""
    mats = list(mats)
    offs = np.zeros(len(mats) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([a.m for a in mats])
    noffs = np.zeros(len(mats) + 1, dtype=np.int64)
    noffs[1:] = np.cumsum([a.nnz for a in mats])
    indptr = np.concatenate([[0]] + [a.indptr[1:].astype(np.int64) + noffs[b]
                                      for b, a in enumerate(mats)])
    indices = np.concatenate([a.indices.astype(np.int64) + offs[b] for b, a in enumerate(mats)])
    values = np.concatenate([a.values for a in mats])
    return CSR(offs[-1], offs[-1], indptr, indices, values), offs.astype(np.int32)


def diffusion_batch(nsys: int, seed: int, side_lo: int = 32, side_hi: int = 256,
                    sigma: float | tuple = 1.0):
    """``nsys`` diffusion systems with sides ~ U{side_lo..side_hi} (sigma fixed or ~U[a,b]).

    Returns (block-diagonal CSR, sys_ptr, sides, sigmas)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=nsys)
    if isinstance(sigma, tuple):
        sigmas = rng.uniform(sigma[0], sigma[1], size=nsys)
    else:
        sigmas = np.full(nsys, float(sigma))
    seeds = rng.integers(0, 2**31 - 1, size=nsys)
    mats = [diffusion2d(int(s), float(sg), int(sd)) for s, sg, sd in zip(sides, sigmas, seeds)]
    A, ptr = block_diag(mats)
    return A, ptr, sides, sigmas


def diffusion_system_batch(nsys: int, seed: int, side_lo: int, side_hi: int, sigma=(0.5, 2.0)):
    """A block-diagonal batch of diffusion systems with N(0,1) right-hand sides:
    (CSR, sys_ptr int32[B+1], b float32[m]).  A plain function of its arguments, so it can
    run in a worker process."""
    A, ptr, _, _ = diffusion_batch(nsys, seed=seed, side_lo=side_lo, side_hi=side_hi, sigma=sigma)
    return A, ptr, normal(A.m, seed=seed + 7919)
