"""Pins of the triangular-solve oracle and its VJP (Section 3.1.5, Table 1 SpSolve rule):
the solves against dense LAPACK, the gradients against central differences and the
dense form -L^-T v x^T."""
import numpy as np
import pytest

from oracle import sptrsv


def random_lower(n, seed, density=0.2):
    rng = np.random.default_rng(seed)
    ip, ix, v = [0], [], []
    for i in range(n):
        cols = sorted(j for j in range(i) if rng.random() < density)
        ix += cols + [i]
        v += list(rng.uniform(-0.5, 0.5, len(cols))) + [rng.uniform(1.5, 2.5)]
        ip.append(len(ix))
    return np.array(ip, np.int32), np.array(ix, np.int32), np.array(v, np.float64)


def dense(ip, ix, v, n):
    D = np.zeros((n, n))
    D[np.repeat(np.arange(n), np.diff(ip)), ix] = v
    return D


def test_solve_matches_dense():
    ip, ix, v = random_lower(60, 1)
    b = np.random.default_rng(2).standard_normal(60)
    np.testing.assert_allclose(sptrsv.solve(ip, ix, v, b), np.linalg.solve(dense(ip, ix, v, 60), b),
                               rtol=1e-12, atol=1e-12)


def test_vjp_dense_form_and_central_differences():
    n = 40
    ip, ix, v = random_lower(n, 3)
    rng = np.random.default_rng(4)
    b, w = rng.standard_normal(n), rng.standard_normal(n)
    x, gb, gl = sptrsv.vjp(ip, ix, v, b, w)
    L = dense(ip, ix, v, n)
    lam = np.linalg.solve(L.T, w)
    np.testing.assert_allclose(gb, lam, rtol=1e-12, atol=1e-12)
    G = -np.outer(lam, x)
    np.testing.assert_allclose(gl, G[np.repeat(np.arange(n), np.diff(ip)), ix], rtol=1e-11, atol=1e-12)
    f = lambda vals, bb: w @ sptrsv.solve(ip, ix, vals, bb)  # noqa: E731
    h = 1e-6
    for e in (0, len(v) // 3, len(v) - 1):
        vp, vm = v.copy(), v.copy()
        vp[e] += h
        vm[e] -= h
        assert (f(vp, b) - f(vm, b)) / (2 * h) == pytest.approx(gl[e], rel=1e-6, abs=1e-9)
    for i in (0, n // 2, n - 1):
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        assert (f(v, bp) - f(v, bm)) / (2 * h) == pytest.approx(gb[i], rel=1e-6, abs=1e-9)
