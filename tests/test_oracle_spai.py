"""Pins of the SPAI oracle (Section 4.6): the loss and gradient against dense linear
algebra and central differences, the static-pattern SPAI against its normal equations, and
gradient descent against the static-pattern minimiser."""
import numpy as np
import pytest

import synth
from oracle import spai


def dense(A, vals=None):
    D = np.zeros((A.m, A.n))
    rows = np.repeat(np.arange(A.m), np.diff(A.indptr))
    D[rows, A.indices] = A.values if vals is None else vals
    return D


@pytest.mark.parametrize("make", [lambda: synth.poisson2d(5), lambda: synth.random_k_per_row(30, 4, seed=2, ncols=30)])
def test_loss_and_grad_match_dense(make):
    A = make()
    rng = np.random.default_rng(0)
    m = rng.standard_normal(A.nnz)
    loss, g = spai.loss_and_grad(A, m)
    Ad, Md = dense(A), dense(A, m)
    R = np.eye(A.m) - Md @ Ad
    assert loss == pytest.approx(np.sum(R * R), rel=1e-12)
    G = -2.0 * R @ Ad.T
    rows = np.repeat(np.arange(A.m), np.diff(A.indptr))
    np.testing.assert_allclose(g, G[rows, A.indices], rtol=1e-12, atol=1e-12 * np.abs(G).max())


def test_grad_central_differences():
    A = synth.poisson2d(4)
    m = np.random.default_rng(1).standard_normal(A.nnz)
    _, g = spai.loss_and_grad(A, m)
    for e in (0, 7, A.nnz // 2, A.nnz - 1):
        h = 1e-3
        mp, mm = m.copy(), m.copy()
        mp[e] += h
        mm[e] -= h
        fd = (spai.loss_and_grad(A, mp)[0] - spai.loss_and_grad(A, mm)[0]) / (2 * h)
        assert fd == pytest.approx(g[e], rel=1e-9, abs=1e-9)     # quadratic: exact up to rounding


def test_step_length_is_the_line_minimum():
    A = synth.poisson2d(6)
    m = np.ones(A.nnz)
    _, g = spai.loss_and_grad(A, m)
    eta = spai.step_length(A, -g)
    f = lambda t: spai.loss_and_grad(A, m - t * g)[0]  # noqa: E731
    assert f(eta) < f(0.9 * eta) and f(eta) < f(1.1 * eta)


def test_static_pattern_spai_normal_equations():
    """Each row's residual e_i - A[J,:]^T m is orthogonal to the rows A[J,:]."""
    A = synth.poisson2d(8)
    m = spai.static_pattern_spai(A)
    Ad = dense(A)
    for i in range(A.m):
        a, b = A.indptr[i], A.indptr[i + 1]
        J = A.indices[a:b]
        r = np.eye(A.m)[i] - Ad[J, :].T @ m[a:b]
        np.testing.assert_allclose(Ad[J, :] @ r, 0.0, atol=1e-12)
    # and it is the global minimum: the gradient vanishes there
    _, g = spai.loss_and_grad(A, m)
    assert np.abs(g).max() < 1e-12


def test_gradient_descent_reaches_the_static_pattern_spai():
    """The paper's 8 x 8 Poisson case, from M = mask(A), stopping at ||grad|| < 0.01."""
    A = synth.poisson2d(8)
    m_gd, hist = spai.gradient_descent(A, gtol=1e-2)
    m_ls = spai.static_pattern_spai(A)
    loss_ls = spai.loss_and_grad(A, m_ls)[0]
    losses = [h[0] for h in hist]
    assert all(b <= a + 1e-12 for a, b in zip(losses, losses[1:]))          # monotone descent
    assert hist[-1][1] < 1e-2 and len(hist) < 200
    assert losses[-1] == pytest.approx(loss_ls, rel=1e-4)
    m_tight, _ = spai.gradient_descent(A, gtol=1e-9, max_it=5000)
    np.testing.assert_allclose(m_tight, m_ls, atol=1e-8)
