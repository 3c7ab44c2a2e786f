"""Sparse triangular solve L x = b and its vector-Jacobian product.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 3.1.5 of the paper: the forward solve by substitution (rows in order; each row needs
only earlier rows), and the backward pass from the sparse-solve rule of Table 1:
    grad_b = L^-T v,     grad_L = -(L^-T v) x^T masked to mask(L),
the transposed solve reusing the forward routine on L^T and the gradient of L a masked outer
product that reuses grad_b.  Float64, through this package's C substitution routines.
"""
from __future__ import annotations

import numpy as np

from . import trsv_lower, trsv_lower_t


def solve(l_indptr, l_indices, l_vals, b):
    """x with L x = b (L lower triangular, CSR with the diagonal stored)."""
    return trsv_lower(l_indptr, l_indices, l_vals, b)


def vjp(l_indptr, l_indices, l_vals, b, v):
    """(x, grad_b, grad_L) of the loss <v, x> with x = L^-1 b."""
    x = trsv_lower(l_indptr, l_indices, l_vals, b)
    lam = trsv_lower_t(l_indptr, l_indices, l_vals, v)
    rows = np.repeat(np.arange(len(l_indptr) - 1), np.diff(l_indptr))
    grad_l = -lam[rows] * x[np.asarray(l_indices)]
    return x, lam, grad_l
