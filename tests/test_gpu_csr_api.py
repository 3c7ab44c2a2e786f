"""The CSR class's operator syntax (A @ X, A @ B, A + B, A - B, A.T, A.diagonal()) on the
library's kernels, against the FP64 oracle, and its gradients against dense FP64 autograd on
tiny inputs (Section 3.1: gradients of sparse values live on the input's pattern)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import assert_close_normalised

pytestmark = pytest.mark.gpu
spx = pytest.importorskip("paper_2212_05159_gb300")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _dense(A):
    D = np.zeros((A.m, A.n))
    rows = np.repeat(np.arange(A.m), np.diff(np.asarray(A.indptr, np.int64)))
    D[rows, A.indices] = A.values
    return D


@pytest.fixture(scope="module")
def rect():
    return synth.empty_rows_csr(300, 250, seed=7, max_len=20)


def test_matmul_dense_and_sparse(rect):
    A = rect
    dA = spx.CSR.from_host(A)
    X = synth.normal((A.n, 8), seed=1)
    Y = host(dA @ dev(X))
    Yo = oracle.spmm(A, X.astype(np.float64))
    assert_close_normalised(Y, Yo, np.abs(_dense(A)) @ np.abs(X), what="A @ X")
    x = synth.normal(A.n, seed=2)
    assert_close_normalised(host(dA @ dev(x)), oracle.spmm(A, x.astype(np.float64)),
                            np.abs(_dense(A)) @ np.abs(x), what="A @ x")
    B = synth.empty_rows_csr(250, 180, seed=8, max_len=10)
    C = dA @ spx.CSR.from_host(B)
    ip, ix, vals = oracle.spgemm(A, B)
    np.testing.assert_array_equal(host(C.indptr), ip)
    np.testing.assert_array_equal(host(C.indices), ix)
    norm = (np.abs(_dense(A)) @ np.abs(_dense(B)))[np.repeat(np.arange(A.m), np.diff(ip)), ix]
    assert_close_normalised(host(C.values), vals, norm, what="A @ B")


def test_transpose_is_bit_exact_and_an_involution(rect):
    A = rect
    dA = spx.CSR.from_host(A)
    AT = dA.T
    t_ip, t_ix, perm = oracle.transpose(A)
    np.testing.assert_array_equal(host(AT.indptr), t_ip)
    np.testing.assert_array_equal(host(AT.indices), t_ix)
    np.testing.assert_array_equal(host(AT.values), np.asarray(A.values, np.float32)[perm])
    ATT = AT.T
    np.testing.assert_array_equal(host(ATT.indptr), A.indptr)
    np.testing.assert_array_equal(host(ATT.indices), A.indices)
    np.testing.assert_array_equal(host(ATT.values), A.values)


def test_transpose_gradient_returns_through_the_inverse(rect):
    A = rect
    dA = spx.CSR.from_host(A)
    v = dA.values.clone().requires_grad_(True)
    w = dev(synth.normal(A.nnz, seed=3))
    (dA.with_values(v).T.values * w).sum().backward()
    _, _, perm = oracle.transpose(A)
    expect = np.empty(A.nnz, np.float32)
    expect[perm] = host(w)                                  # d/dv[perm[e]] of sum_e v[perm[e]] w[e]
    np.testing.assert_array_equal(host(v.grad), expect)


def test_diagonal_and_its_gradient():
    """A square matrix with some diagonal entries missing, and a wide rectangular one."""
    rng = np.random.default_rng(4)
    for (m, n) in ((200, 200), (120, 200), (200, 90)):
        D = (rng.random((m, n)) < 0.05) * rng.normal(size=(m, n))
        k = min(m, n)
        keep = rng.random(k) < 0.7
        D[np.arange(k)[keep], np.arange(k)[keep]] = rng.normal(size=int(keep.sum()))
        D[np.arange(k)[~keep], np.arange(k)[~keep]] = 0.0
        r, c = np.nonzero(D)
        ip = np.concatenate([[0], np.cumsum(np.bincount(r, minlength=m))])
        A = synth.CSR(m, n, ip, c, D[r, c].astype(np.float32))
        dA = spx.CSR.from_host(A)
        d = dA.diagonal()
        np.testing.assert_array_equal(host(d), oracle.diagonal(A)[:k].astype(np.float32))
        v = dA.values.clone().requires_grad_(True)
        g = dev(synth.normal(k, seed=m + n))
        (dA.with_values(v).diagonal() * g).sum().backward()
        expect = np.zeros(A.nnz, np.float32)
        on = np.nonzero(r == c)[0]
        expect[on] = host(g)[r[on]]
        np.testing.assert_array_equal(host(v.grad), expect)


def test_composed_expression_gradients_match_dense_autograd():
    """loss = sum(w * (A^T (A x)) / diag(A)) through A @, .T and diagonal(), against the same
    expression on the dense FP64 matrix with torch autograd (CPU)."""
    A = synth.poisson2d(6)
    dA = spx.CSR.from_host(A)
    v = dA.values.clone().requires_grad_(True)
    x = dev(synth.normal(A.n, seed=5)).requires_grad_(True)
    w = synth.normal(A.n, seed=6)
    B = dA.with_values(v)
    loss = ((B.T @ (B @ x)) / B.diagonal() * dev(w)).sum()
    loss.backward()
    Dd = torch.tensor(_dense(A), requires_grad=True)
    xd = torch.tensor(synth.normal(A.n, seed=5).astype(np.float64), requires_grad=True)
    lossd = ((Dd.t() @ (Dd @ xd)) / torch.diagonal(Dd) * torch.tensor(w.astype(np.float64))).sum()
    lossd.backward()
    rows = np.repeat(np.arange(A.m), np.diff(A.indptr))
    gd = Dd.grad.numpy()[rows, A.indices]
    assert abs(float(loss.detach()) - float(lossd.detach())) <= 1e-5 * max(1.0, abs(float(lossd.detach())))
    assert np.abs(host(v.grad) - gd).max() <= 1e-4 * np.abs(gd).max()
    assert np.abs(host(x.grad) - xd.grad.numpy()).max() <= 1e-4 * np.abs(xd.grad.numpy()).max()


@pytest.mark.parametrize("op", ["+", "-"])
def test_add_and_sub_on_the_union_pattern(op):
    """A + B and A - B for two patterns that overlap in part (and rows empty in one of them):
    the union pattern bit-exact, values and both value gradients against the oracle."""
    from oracle.spadd import spadd as o_spadd, spadd_backward as o_spadd_bwd
    A = synth.empty_rows_csr(400, 300, seed=21, max_len=15)
    B = synth.empty_rows_csr(400, 300, seed=22, max_len=15)
    beta = 1.0 if op == "+" else -1.0
    dA, dB = spx.CSR.from_host(A), spx.CSR.from_host(B)
    va = dA.values.clone().requires_grad_(True)
    vb = dB.values.clone().requires_grad_(True)
    C = dA.with_values(va) + dB.with_values(vb) if op == "+" else dA.with_values(va) - dB.with_values(vb)
    ip, ix, vals = o_spadd(A, B, 1.0, beta)
    np.testing.assert_array_equal(host(C.indptr), ip)
    np.testing.assert_array_equal(host(C.indices), ix)
    _, _, norm = o_spadd(synth.CSR(A.m, A.n, A.indptr, A.indices, np.abs(A.values)),
                         synth.CSR(B.m, B.n, B.indptr, B.indices, np.abs(B.values)), 1.0, 1.0)
    assert_close_normalised(host(C.values), vals, norm, what=f"A {op} B")
    gc = synth.normal(ix.size, seed=23)
    (C.values * dev(gc)).sum().backward()
    ga, gb = o_spadd_bwd(A, B, ip, ix, gc, 1.0, beta)
    np.testing.assert_array_equal(host(va.grad), ga.astype(np.float32))
    np.testing.assert_array_equal(host(vb.grad), gb.astype(np.float32))


def test_sum_of_sparse_terms_gradients_match_dense_autograd():
    """loss = sum(w * ((A - B) @ x + (A + B).T @ x)) through +, -, @ and .T, against dense FP64
    autograd on the same matrices."""
    A = synth.poisson2d(5)
    B = synth.with_values(synth.random_k_per_row(A.m, 3, seed=24, ncols=A.n), synth.normal(A.m * 3, seed=25))
    dA, dB = spx.CSR.from_host(A), spx.CSR.from_host(B)
    va = dA.values.clone().requires_grad_(True)
    vb = dB.values.clone().requires_grad_(True)
    xh = synth.normal(A.n, seed=26)
    w = synth.normal(A.n, seed=27)
    x = dev(xh)
    SA, SB = dA.with_values(va), dB.with_values(vb)
    loss = ((((SA - SB) @ x) + ((SA + SB).T @ x)) * dev(w)).sum()
    loss.backward()
    Da = torch.tensor(_dense(A), requires_grad=True)
    Db = torch.tensor(_dense(B), requires_grad=True)
    xd = torch.tensor(xh.astype(np.float64))
    lossd = ((((Da - Db) @ xd) + ((Da + Db).t() @ xd)) * torch.tensor(w.astype(np.float64))).sum()
    lossd.backward()
    ra = np.repeat(np.arange(A.m), np.diff(A.indptr))
    rb = np.repeat(np.arange(B.m), np.diff(B.indptr))
    ga, gb = Da.grad.numpy()[ra, A.indices], Db.grad.numpy()[rb, B.indices]
    assert abs(float(loss.detach()) - float(lossd.detach())) <= 1e-5 * max(1.0, abs(float(lossd.detach())))
    assert np.abs(host(va.grad) - ga).max() <= 1e-5 * max(1.0, np.abs(ga).max())
    assert np.abs(host(vb.grad) - gb).max() <= 1e-5 * max(1.0, np.abs(gb).max())
