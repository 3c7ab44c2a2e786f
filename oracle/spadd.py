"""Sparse + sparse: C = alpha A + beta B and its vector-Jacobian products.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 3.1.4 of the paper: mask(C) = mask(A) union mask(B), row by row; the gradients are
alpha V on mask(A) and beta V on mask(B), V given on mask(C) (Table 1, Sp + Sp).  The
pattern is structural: an entry stored in A or B is stored in C even when alpha a + beta b
is zero.  Plain per-row Python loops in float64.
"""
from __future__ import annotations

import numpy as np


def spadd(A, B, alpha, beta):
    """(indptr int32, indices int32, values float64) of alpha A + beta B."""
    assert A.m == B.m and A.n == B.n
    ip = [0]
    ix, vals = [], []
    for i in range(A.m):
        acc = {}
        for e in range(A.indptr[i], A.indptr[i + 1]):
            acc[int(A.indices[e])] = acc.get(int(A.indices[e]), 0.0) + alpha * float(A.values[e])
        for e in range(B.indptr[i], B.indptr[i + 1]):
            acc[int(B.indices[e])] = acc.get(int(B.indices[e]), 0.0) + beta * float(B.values[e])
        for j in sorted(acc):
            ix.append(j)
            vals.append(acc[j])
        ip.append(len(ix))
    return np.array(ip, np.int32), np.array(ix, np.int32), np.array(vals, np.float64)


def spadd_backward(A, B, c_indptr, c_indices, gc, alpha, beta):
    """(alpha V on mask(A), beta V on mask(B)) for V = gc on mask(C)."""
    ga = np.empty(A.nnz, np.float64)
    gb = np.empty(B.nnz, np.float64)
    for i in range(A.m):
        row = {int(c_indices[e]): float(gc[e]) for e in range(c_indptr[i], c_indptr[i + 1])}
        for e in range(A.indptr[i], A.indptr[i + 1]):
            ga[e] = alpha * row[int(A.indices[e])]
        for e in range(B.indptr[i], B.indptr[i + 1]):
            gb[e] = beta * row[int(B.indices[e])]
    return ga, gb
