"""Sparse approximate inverse by gradient descent, and the static-pattern SPAI it is
compared with.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 4.6 of the paper: minimise the Frobenius loss

    loss(M) = || I - M A ||_F^2                                   (SPAI loss)

over the stored entries of M, with mask(M) = mask(A) fixed and M initialised to mask(A)
(every stored entry 1), by gradient descent until the gradient norm is below 0.01.  The
gradient follows from Table 1 (SpSpMM w.r.t. the first operand) with the upstream
gradient -2 (I - M A) on the pattern of C = M A:

    grad = -2 mask_M( (I - M A) A^T ).

The paper does not give the step size.  Reading: the loss is a quadratic in M, so each
step moves along d = -grad by its exact minimiser eta = (1/2) <d, d> / <d A, d A> (the
derivative of ||R - eta d A||^2 vanishes there, and <R, d A> = <R A^T, d> = <d, d> / 2).

The reference solution: the loss splits into one least-squares problem per row of M,
    min over m (support J_i) of || e_i - A[J_i, :]^T m ||_2,
solved directly row by row (the static-pattern SPAI of Grote and Huckle).

Everything is FP64; sparse products go through this package's C routines.
"""
from __future__ import annotations

import numpy as np

from . import spgemm, spgemm_grad_a


class _Mat:
    """CSR holder with float64 values (A's pattern, M's values)."""

    def __init__(self, m, n, indptr, indices, values):
        self.m, self.n = m, n
        self.indptr, self.indices, self.values = indptr, indices, values
        self.nnz = int(indptr[-1])


def residual(A, m_vals):
    """(C pattern, R values) with C = M A and R = I - C on C's pattern, plus the count of
    diagonal entries of I that C's pattern lacks (each adds 1 to the loss)."""
    M = _Mat(A.m, A.n, A.indptr, A.indices, np.asarray(m_vals, np.float64))
    c_ip, c_ix, c_v = spgemm(M, A)
    rows = np.repeat(np.arange(A.m), np.diff(c_ip))
    on_diag = rows == c_ix
    R = on_diag.astype(np.float64) - c_v
    missing = A.m - int(on_diag.sum())
    return (c_ip, c_ix), R, missing


def loss_and_grad(A, m_vals):
    """The SPAI loss and its gradient on M's (= A's) stored entries."""
    (c_ip, c_ix), R, missing = residual(A, m_vals)
    loss = float(R @ R) + missing
    M = _Mat(A.m, A.n, A.indptr, A.indices, np.asarray(m_vals, np.float64))
    grad = spgemm_grad_a(M, A, c_ip, c_ix, -2.0 * R)
    return loss, grad


def step_length(A, d):
    """Exact minimiser of the loss along direction d (given on M's pattern)."""
    D = _Mat(A.m, A.n, A.indptr, A.indices, np.asarray(d, np.float64))
    _, _, da = spgemm(D, A)
    return 0.5 * float(d @ d) / float(da @ da)


def gradient_descent(A, gtol=1e-2, max_it=500, m0=None):
    """Descent on the stored entries of M from M = mask(A) until ||grad|| < gtol.
    Returns (m values, [(loss, ||grad||) per iterate])."""
    m = np.ones(A.nnz, np.float64) if m0 is None else np.array(m0, np.float64)
    hist = []
    for _ in range(max_it + 1):
        loss, g = loss_and_grad(A, m)
        gn = float(np.sqrt(g @ g))
        hist.append((loss, gn))
        if gn < gtol or len(hist) > max_it:
            break
        d = -g
        m = m + step_length(A, d) * d
    return m, hist


def static_pattern_spai(A):
    """Row-wise least-squares minimiser of the loss with mask(M) = mask(A)."""
    Ad = np.zeros((A.m, A.n))
    rows = np.repeat(np.arange(A.m), np.diff(A.indptr))
    Ad[rows, A.indices] = np.asarray(A.values, np.float64)
    m = np.empty(A.nnz, np.float64)
    for i in range(A.m):
        a, b = int(A.indptr[i]), int(A.indptr[i + 1])
        J = A.indices[a:b]
        e = np.zeros(A.n)
        e[i] = 1.0
        m[a:b] = np.linalg.lstsq(Ad[J, :].T, e, rcond=None)[0]
    return m
