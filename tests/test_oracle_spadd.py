"""Pins of the sparse-add oracle (Section 3.1.4, Table 1 Sp + Sp): values against dense
alpha A + beta B, the pattern against the union of the stored patterns (cancellations kept),
and the gradients against dense masking and the linearity of <V, C>."""
import numpy as np
import pytest

import synth
from oracle import spadd


def dense(ip, ix, v, m, n):
    D = np.zeros((m, n))
    rows = np.repeat(np.arange(m), np.diff(ip))
    D[rows, ix] = v
    return D


def stored(ip, ix, m, n):
    S = np.zeros((m, n), bool)
    S[np.repeat(np.arange(m), np.diff(ip)), ix] = True
    return S


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (1.0, -1.0), (0.5, 2.0)])
def test_values_and_union_pattern(alpha, beta):
    A = synth.random_k_per_row(40, 5, seed=1, ncols=37)
    B = synth.empty_rows_csr(40, 37, seed=2, max_len=9)
    c_ip, c_ix, c_v = spadd.spadd(A, B, alpha, beta)
    Ad = dense(A.indptr, A.indices, A.values, A.m, A.n)
    Bd = dense(B.indptr, B.indices, B.values, B.m, B.n)
    np.testing.assert_allclose(dense(c_ip, c_ix, c_v, A.m, A.n), alpha * Ad + beta * Bd, rtol=0, atol=1e-12)
    union = stored(A.indptr, A.indices, A.m, A.n) | stored(B.indptr, B.indices, B.m, B.n)
    np.testing.assert_array_equal(stored(c_ip, c_ix, A.m, A.n), union)
    for i in range(A.m):
        assert np.all(np.diff(c_ix[c_ip[i]:c_ip[i + 1]]) > 0)       # sorted, unique


def test_cancellation_keeps_the_entry():
    A = synth.poisson2d(4)
    c_ip, c_ix, c_v = spadd.spadd(A, A, 1.0, -1.0)
    np.testing.assert_array_equal(c_ip, A.indptr)
    np.testing.assert_array_equal(c_ix, A.indices)
    assert np.all(c_v == 0.0)


def test_backward_is_the_masked_upstream_and_the_adjoint():
    A = synth.random_k_per_row(30, 4, seed=3, ncols=30)
    B = synth.random_k_per_row(30, 6, seed=4, ncols=30)
    alpha, beta = 0.75, -1.25
    c_ip, c_ix, _ = spadd.spadd(A, B, alpha, beta)
    gc = np.random.default_rng(5).standard_normal(c_ix.size)
    ga, gb = spadd.spadd_backward(A, B, c_ip, c_ix, gc, alpha, beta)
    V = dense(c_ip, c_ix, gc, A.m, A.n)
    rows_a = np.repeat(np.arange(A.m), np.diff(A.indptr))
    rows_b = np.repeat(np.arange(B.m), np.diff(B.indptr))
    np.testing.assert_allclose(ga, alpha * V[rows_a, A.indices], rtol=0, atol=1e-15)
    np.testing.assert_allclose(gb, beta * V[rows_b, B.indices], rtol=0, atol=1e-15)
    # adjoint identity: <V, alpha dA + beta dB> = <ga, dA> + <gb, dB> for perturbations on the patterns
    rng = np.random.default_rng(6)
    da = rng.standard_normal(A.nnz).astype(np.float32).astype(np.float64)      # exact in the float32 CSR
    db = rng.standard_normal(B.nnz).astype(np.float32).astype(np.float64)
    dA = synth.CSR(A.m, A.n, A.indptr, A.indices, da)
    dB = synth.CSR(B.m, B.n, B.indptr, B.indices, db)
    _, _, dc = spadd.spadd(dA, dB, alpha, beta)
    assert gc @ dc == pytest.approx(ga @ da + gb @ db, rel=1e-12)
