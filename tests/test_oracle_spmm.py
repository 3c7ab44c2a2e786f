"""Pins for the oracle's SpMM, SDDMM, transpose and transpose-SpMM (CPU only).

Each pin is independent of the oracle's own loops: dense linear algebra on tiny
inputs, closed forms of the paper's model problems (Section 4, A_N and its 2D
Kronecker sum), finite differences of <G, A X> (the VJP contract of Section 2.2),
and structural identities.
"""
import numpy as np
import pytest

import synth


def _rand_csr(m, n, seed, density=0.3):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    d[m // 2, :] = 0.0                       # an empty row
    return synth.from_dense(d.astype(np.float32))


@pytest.mark.parametrize("m,n,k", [(7, 5, 1), (13, 17, 3), (32, 9, 8), (5, 40, 33)])
def test_spmm_matches_dense(orc, m, n, k):
    A = _rand_csr(m, n, seed=m * n + k)
    X = synth.normal((n, k), seed=k)
    Y = orc.spmm(A, X)
    np.testing.assert_allclose(Y, A.to_dense() @ X.astype(np.float64), rtol=1e-13, atol=1e-13)


def test_spmv_vector_shape(orc):
    A = _rand_csr(6, 4, seed=1)
    x = synth.normal(4, seed=2)
    y = orc.spmm(A, x)
    assert y.shape == (6,)
    np.testing.assert_allclose(y, A.to_dense() @ x.astype(np.float64), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("N", [1, 2, 9, 64])
def test_poisson1d_eigenvectors(orc, N):
    """A_N v_k = (2 - 2 cos(k pi/(N+1))) v_k with v_k(i) = sin(i k pi/(N+1))."""
    A = synth.poisson1d(N)
    i = np.arange(1, N + 1)
    for kk in (1, (N + 1) // 2, N):
        v = np.sin(i * kk * np.pi / (N + 1))
        lam = 2.0 - 2.0 * np.cos(kk * np.pi / (N + 1))
        np.testing.assert_allclose(orc.spmm(A, v), lam * v, atol=1e-12)


def test_poisson1d_row_sums(orc):
    """Row sums of A_N: 1 at both ends, 0 inside."""
    A = synth.poisson1d(50)
    s = orc.spmm(A, np.ones(50))
    expect = np.zeros(50)
    expect[0] = expect[-1] = 1.0
    np.testing.assert_array_equal(s, expect)


def test_poisson2d_eigenvector_and_count(orc):
    """Kronecker sum: eigenvalue lam_a(Nx) + lam_b(Ny) on sin x sin; nnz = 5 N^2 - 4 N."""
    nx, ny = 6, 9
    A = synth.poisson2d(nx, ny)
    assert A.nnz == 5 * nx * ny - 2 * nx - 2 * ny
    assert synth.poisson2d(64).nnz == 20224          # the 64 x 64 workload
    a, b = 2, 5
    ix, iy = np.meshgrid(np.arange(1, nx + 1), np.arange(1, ny + 1), indexing="ij")
    v = (np.sin(ix * a * np.pi / (nx + 1)) * np.sin(iy * b * np.pi / (ny + 1))).ravel()
    lam = (2 - 2 * np.cos(a * np.pi / (nx + 1))) + (2 - 2 * np.cos(b * np.pi / (ny + 1)))
    np.testing.assert_allclose(orc.spmm(A, v), lam * v, atol=1e-12)


def test_poisson3d_count():
    """7-point stencil on n^3: nnz = 7 n^3 - 6 n^2."""
    for n in (1, 3, 8):
        assert synth.poisson3d(n).nnz == 7 * n ** 3 - 6 * n ** 2


@pytest.mark.parametrize("m,n,k", [(9, 7, 1), (16, 11, 4), (6, 30, 17)])
def test_sddmm_matches_masked_dense(orc, m, n, k):
    A = _rand_csr(m, n, seed=3 * m + k)
    G = synth.normal((m, k), seed=10 + k)
    X = synth.normal((n, k), seed=20 + k)
    out = orc.sddmm(A, G, X)
    dense = G.astype(np.float64) @ X.astype(np.float64).T
    rows = np.repeat(np.arange(m), A.row_lengths())
    np.testing.assert_allclose(out, dense[rows, A.indices], rtol=1e-13, atol=1e-13)


def test_sddmm_is_gradient_of_spmm(orc):
    """d <G, A X> / d A_e by central differences equals sddmm (exact: linear map)."""
    A = _rand_csr(8, 6, seed=5)
    A = synth.with_values(A, np.round(A.values * 64) / 64)   # dyadic: v +- h stays exact
    X = synth.normal((6, 3), seed=6).astype(np.float64)
    G = synth.normal((8, 3), seed=7).astype(np.float64)
    grad = orc.sddmm(A, G, X)
    h = 0.5
    vals = A.values.astype(np.float64)
    for e in range(A.nnz):
        vp, vm = vals.copy(), vals.copy()
        vp[e] += h
        vm[e] -= h
        Ap = synth.CSR(A.m, A.n, A.indptr, A.indices, vp)
        Am = synth.CSR(A.m, A.n, A.indptr, A.indices, vm)
        # spmm promotes float32 values: keep h exactly representable
        fd = (np.sum(G * orc.spmm(Ap, X)) - np.sum(G * orc.spmm(Am, X))) / (2 * h)
        assert abs(fd - grad[e]) <= 1e-10 * (1 + abs(grad[e]))


def test_transpose_matches_dense_and_is_involution(orc):
    A = synth.empty_rows_csr(40, 23, seed=3, max_len=6)
    t_ip, t_ix, perm = orc.transpose(A)
    AT = synth.CSR(A.n, A.m, t_ip, t_ix, A.values[perm])
    np.testing.assert_array_equal(AT.to_dense(), A.to_dense().T)
    # rows of A^T are sorted (stable counting sort) and perm is a permutation
    for j in range(A.n):
        seg = t_ix[t_ip[j]:t_ip[j + 1]]
        assert np.all(np.diff(seg) > 0)
    assert np.array_equal(np.sort(perm), np.arange(A.nnz))
    t2_ip, t2_ix, perm2 = orc.transpose(AT)
    np.testing.assert_array_equal(t2_ip, A.indptr)
    np.testing.assert_array_equal(t2_ix, A.indices)
    np.testing.assert_array_equal(perm[perm2], np.arange(A.nnz))


@pytest.mark.parametrize("m,n,k", [(11, 7, 1), (8, 20, 5)])
def test_spmm_t_matches_dense_and_adjoint(orc, m, n, k):
    A = _rand_csr(m, n, seed=m + n + k)
    G = synth.normal((m, k), seed=1 + k).astype(np.float64)
    X = synth.normal((n, k), seed=2 + k).astype(np.float64)
    gX = orc.spmm_t(A, G)
    np.testing.assert_allclose(gX, A.to_dense().T @ G, rtol=1e-13, atol=1e-13)
    # <G, A X> = <A^T G, X>
    assert abs(np.sum(G * orc.spmm(A, X)) - np.sum(gX * X)) < 1e-11


def test_empty_matrix(orc):
    A = synth.CSR(3, 4, np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    assert np.all(orc.spmm(A, np.ones((4, 2))) == 0)
    assert orc.sddmm(A, np.ones((3, 2)), np.ones((4, 2))).size == 0
    t_ip, t_ix, perm = orc.transpose(A)
    assert np.all(t_ip == 0) and t_ix.size == 0


def test_row_parallel_variants_equal_the_serial_routines(orc):
    """The all-cores timing variants: the same sums in the same order, so bitwise equal
    (power-law rows, empty rows and a hub row, a rectangular matrix, 1 to 7 threads)."""
    A = synth.powerlaw_csr(3000, seed=4, max_len=400)
    R = synth.random_k_per_row(500, 3, seed=2, ncols=800)
    E = synth.empty_rows_csr(700, 900, seed=3)
    for M in (A, R, E):
        X = synth.normal((M.n, 5), seed=1)
        G = synth.normal((M.m, 5), seed=2)
        t = orc.transpose(M)
        for threads in (1, 3, 7):
            Y, used = orc.spmm_mt(M, X, threads)
            assert 1 <= used <= threads
            np.testing.assert_array_equal(Y, orc.spmm(M, X))
            np.testing.assert_array_equal(orc.sddmm_mt(M, G, X, threads)[0], orc.sddmm(M, G, X))
            np.testing.assert_array_equal(orc.spmm_t_mt(M, G, threads, t)[0], orc.spmm_t(M, G))
