"""Pins for the oracle's unrolled PCG loss and its hand-written reverse (CPU only).

* torch FP64 autograd of the same unrolled loop written with dense matrices
  (Section 4.3 loss, M = L L^T);
* central differences on a tiny batch;
* L = D^{-1/2} (Jacobi) reproduces the residual history of Jacobi PCG.
"""
import numpy as np
import torch

import synth
from oracle import pcg_unrolled


def _batch(sides, seed):
    mats = [synth.diffusion2d(s, 1.0, seed + i) for i, s in enumerate(sides)]
    return synth.block_diag(mats)


def _tril_values(orc, A, seed):
    l_ip, l_ix, keep = orc.tril_pattern(A)
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(A.m), np.diff(l_ip))
    d = orc.diagonal(A)
    v = rng.uniform(-0.2, 0.2, l_ix.size) / np.sqrt(d[rows])
    diag = rows == l_ix
    v[diag] = (1.0 + rng.uniform(-0.1, 0.1, int(diag.sum()))) / np.sqrt(d[rows[diag]])
    return synth.CSR(A.m, A.n, l_ip, l_ix, v.astype(np.float32)), rows


def _torch_loss(A, L, rows, b, ptr, n_it, gamma):
    lv = torch.tensor(L.values.astype(np.float64), requires_grad=True)
    Ad_all = torch.tensor(A.to_dense())
    Ld_all = torch.zeros(A.m, A.m, dtype=torch.float64).index_put(
        (torch.tensor(rows), torch.tensor(L.indices.astype(np.int64))), lv)
    w = torch.tensor(pcg_unrolled.loss_weights(n_it, gamma))
    loss = 0
    nsys = len(ptr) - 1
    for s in range(nsys):
        a, c = int(ptr[s]), int(ptr[s + 1])
        Ad = Ad_all[a:c, a:c]
        Ld = Ld_all[a:c, a:c]
        M = Ld @ Ld.T
        bs = torch.tensor(b[a:c])
        r = bs.clone()
        z = M @ r
        p = z.clone()
        rz = r @ z
        for i in range(n_it):
            q = Ad @ p
            al = rz / (p @ q)
            r = r - al * q
            z = M @ r
            rzn = r @ z
            p = z + (rzn / rz) * p
            rz = rzn
            loss = loss + w[i] * torch.linalg.norm(r) / torch.linalg.norm(bs) / nsys
    loss.backward()
    return float(loss.detach()), lv.grad.numpy()


def test_unrolled_pcg_grad_matches_torch_autograd(orc):
    A, ptr = _batch([4, 5, 3], seed=1)
    L, rows = _tril_values(orc, A, seed=2)
    b = synth.normal(A.m, seed=3).astype(np.float64)
    loss, g, _ = pcg_unrolled.forward_backward(A, L, b, ptr, n_it=4, gamma=0.6)
    tl, tg = _torch_loss(A, L, rows, b, ptr, 4, 0.6)
    assert abs(loss - tl) < 1e-13
    np.testing.assert_allclose(g, tg, rtol=1e-9, atol=1e-12)


def test_unrolled_pcg_grad_finite_differences(orc):
    A, ptr = _batch([3, 4], seed=5)
    L, _ = _tril_values(orc, A, seed=6)
    b = synth.normal(A.m, seed=7).astype(np.float64)
    Lv = L.values.astype(np.float64)
    _, g, _ = pcg_unrolled.forward_backward(A, L, b, ptr, n_it=3, gamma=0.6)

    class V:  # an L with float64 values (the oracle promotes values exactly)
        m, n, indptr, indices = L.m, L.n, L.indptr, L.indices
        nnz = L.nnz

    def f(vals):
        V.values = vals
        return pcg_unrolled.forward_backward(A, V, b, ptr, n_it=3, gamma=0.6,
                                             want_grad=False)[0]
    h = 1e-6
    for e in range(0, L.nnz, 2):
        vp, vm = Lv.copy(), Lv.copy()
        vp[e] += h
        vm[e] -= h
        fd = (f(vp) - f(vm)) / (2 * h)
        assert abs(fd - g[e]) < 1e-6 * (1 + abs(g[e]))


def test_jacobi_factor_reproduces_jacobi_pcg(orc):
    A, ptr = _batch([8], seed=9)
    d = orc.diagonal(A)
    n = A.m
    L = synth.CSR(n, n, np.arange(n + 1), np.arange(n), (1 / np.sqrt(d)).astype(np.float32))
    b = synth.normal(n, seed=1).astype(np.float64)
    _, _, hists = pcg_unrolled.forward_backward(A, L, b, ptr, n_it=5, want_grad=False)
    # Jacobi with the float32-rounded factor: M = diag(l^2)
    dd = 1.0 / (L.values.astype(np.float64) ** 2)
    _, _, it, h = orc.pcg(A, b, tol=1e-30, maxit=5, pc="jacobi", diag=dd, hist=True)
    np.testing.assert_allclose(hists[0], h, rtol=1e-9)
