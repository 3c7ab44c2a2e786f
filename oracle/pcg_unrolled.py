"""Unrolled PCG with a learned factor M = L L^T, its loss and its hand-written reverse.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 4.3 of the paper: PCG with an approximate inverse M = L L^T (L lower
triangular), run for N_it iterations from x0 = 0, and the weighted residual-history
loss

    loss = sum_{i=1..N_it} w_i ||r_i|| / ||b||,   w_i = gamma^(N_it - i) / sum_j gamma^(N_it - j)

where r_i is the residual after iteration i (recurrence residual, x0 = 0).  Systems of
a block-diagonal batch are independent; their losses are averaged.

The reverse pass is written out by hand from the chain rule (Section 2), one forward
statement at a time in reverse order; gradients w.r.t. L stay on L's pattern (Table 1:
the SpMV VJP w.r.t. the matrix is a masked outer product).  Everything is FP64.
"""
from __future__ import annotations

import numpy as np

from . import sddmm, spmm, spmm_t


def loss_weights(n_it: int, gamma: float) -> np.ndarray:
    w = gamma ** (n_it - np.arange(1, n_it + 1, dtype=np.float64))
    return w / w.sum()


class _Block:
    """A CSR block that keeps the dtype of its values (float64 for perturbations)."""

    def __init__(self, n, indptr, indices, values):
        self.m = self.n = n
        self.indptr, self.indices, self.values = indptr, indices, values
        self.nnz = int(indptr[-1])


class _Sys:
    """One system's slice of the batch: rows [r0, r1)."""

    def __init__(self, A, L, r0, r1):
        self.r0, self.r1 = r0, r1
        n = r1 - r0

        def sub(M):
            a, b = int(M.indptr[r0]), int(M.indptr[r1])
            ip = np.asarray(M.indptr[r0:r1 + 1], np.int64) - a
            return _Block(n, ip, np.asarray(M.indices[a:b], np.int64) - r0, M.values[a:b]), a, b
        self.A, _, _ = sub(A)
        self.L, self.la, self.lb = sub(L)


def _apply_M(L, r):
    """z = L (L^T r); returns (w, z) with w = L^T r."""
    w = spmm_t(L, r)
    return w, spmm(L, w)


def forward_backward(A, L, b, sys_ptr, n_it: int = 4, gamma: float = 0.6,
                     want_grad: bool = True):
    """Loss of the unrolled PCG and d loss / d L.values (on L's pattern).

    A, L: CSR (synth.CSR) of the block-diagonal batch, L lower-triangular;
    b: right-hand sides (float64 [n]); sys_ptr: row offsets of the systems.
    Returns (loss, grad_L float64[nnz_L], per-system relative residual histories)."""
    wts = loss_weights(n_it, gamma)
    nsys = len(sys_ptr) - 1
    gL = np.zeros(L.nnz)
    loss = 0.0
    hists = []
    for s in range(nsys):
        S = _Sys(A, L, int(sys_ptr[s]), int(sys_ptr[s + 1]))
        bs = np.asarray(b[S.r0:S.r1], np.float64)
        ls, g, h = _one_system(S.A, S.L, bs, n_it, wts, want_grad)
        loss += ls / nsys
        if want_grad:
            gL[S.la:S.lb] += g / nsys
        hists.append(h)
    return loss, gL, hists


def _one_system(A, L, b, n_it, wts, want_grad):
    bnorm = np.linalg.norm(b)
    # ---------------- forward, keeping every intermediate
    r = [b.copy()]
    w0, z0 = _apply_M(L, b)
    ws, zs = [w0], [z0]
    rz = [float(b @ z0)]
    p = [z0.copy()]
    q, s, alpha, beta = [None], [None], [None], [None]
    rn = [bnorm]
    for i in range(1, n_it + 1):
        qi = spmm(A, p[i - 1])
        si = float(p[i - 1] @ qi)
        ai = rz[i - 1] / si
        ri = r[i - 1] - ai * qi
        wi, zi = _apply_M(L, ri)
        rzi = float(ri @ zi)
        bi = rzi / rz[i - 1]
        pi = zi + bi * p[i - 1]
        q.append(qi); s.append(si); alpha.append(ai); r.append(ri)
        ws.append(wi); zs.append(zi); rz.append(rzi); beta.append(bi); p.append(pi)
        rn.append(float(np.linalg.norm(ri)))
    loss = float(sum(wts[i - 1] * rn[i] for i in range(1, n_it + 1)) / bnorm)
    hist = np.array(rn) / bnorm
    if not want_grad:
        return loss, None, hist

    # ---------------- reverse
    gL = np.zeros(L.nnz)
    rb = [np.zeros_like(b) for _ in range(n_it + 1)]
    pb = [np.zeros_like(b) for _ in range(n_it + 1)]
    rzb = [0.0] * (n_it + 1)
    for i in range(1, n_it + 1):                 # loss = sum w_i ||r_i|| / ||b||
        rb[i] += (wts[i - 1] / bnorm) * r[i] / rn[i]
    for i in range(n_it, 0, -1):
        # p_i = z_i + beta_i p_{i-1}
        zb = pb[i].copy()
        betab = float(pb[i] @ p[i - 1])
        pb[i - 1] += beta[i] * pb[i]
        # beta_i = rz_i / rz_{i-1}
        rzb[i] += betab / rz[i - 1]
        rzb[i - 1] -= betab * rz[i] / rz[i - 1] ** 2
        # rz_i = <r_i, z_i>
        rb[i] += rzb[i] * zs[i]
        zb += rzb[i] * r[i]
        # z_i = L w_i
        gL += sddmm(L, zb.reshape(-1, 1), ws[i].reshape(-1, 1))
        wb = spmm_t(L, zb)
        # w_i = L^T r_i
        gL += sddmm(L, r[i].reshape(-1, 1), wb.reshape(-1, 1))
        rb[i] += spmm(L, wb)
        # r_i = r_{i-1} - alpha_i q_i
        rb[i - 1] += rb[i]
        alphab = -float(rb[i] @ q[i])
        qb = -alpha[i] * rb[i]
        # alpha_i = rz_{i-1} / s_i
        rzb[i - 1] += alphab / s[i]
        sb = -alphab * rz[i - 1] / s[i] ** 2
        # s_i = <p_{i-1}, q_i>
        pb[i - 1] += sb * q[i]
        qb += sb * p[i - 1]
        # q_i = A p_{i-1}
        pb[i - 1] += spmm_t(A, qb)
    # p_0 = z_0; rz_0 = <r_0, z_0>; z_0 = L w_0; w_0 = L^T r_0 (r_0 = b is constant)
    zb = pb[0] + rzb[0] * r[0]
    gL += sddmm(L, zb.reshape(-1, 1), ws[0].reshape(-1, 1))
    wb = spmm_t(L, zb)
    gL += sddmm(L, r[0].reshape(-1, 1), wb.reshape(-1, 1))
    return loss, gL, hist
