"""Pins for the oracle's PCG, preconditioners, IC(0), triangular solves and the
sparse-solve adjoint (CPU only).

* PCG against a dense LAPACK solve on tiny SPD systems, and against the closed-form inverse
  of A_N (the discrete Green's function) with plain and Jacobi preconditioning;
* one-iteration convergence on an eigenvector right-hand side of A_N / 2D Poisson
  (Section 4 model problems);
* IC(0) of the tridiagonal A_N is its exact Cholesky factor (no fill), so IC(0)-PCG
  converges in one iteration;
* Jacobi with a constant diagonal reproduces the unpreconditioned iteration count,
  and M = L L^T with L = I is plain CG;
* the adjoint (Table 1, SpSolve rows) against central differences of g^T A^{-1} b;
* status codes for max-iterations, breakdown and non-finite input.
"""
import numpy as np
import pytest

import synth


def test_pcg_matches_dense_solve(orc):
    A = synth.diffusion2d(7, 1.0, seed=3)
    b = synth.normal(A.m, seed=4).astype(np.float64)
    x, st, it = orc.pcg(A, b, tol=1e-12)
    assert st == 0
    np.testing.assert_allclose(x, np.linalg.solve(A.to_dense(), b), rtol=1e-9, atol=1e-11)
    for pc in ("jacobi", "ic0"):
        L = orc.ic0(A) if pc == "ic0" else None
        x2, st2, it2 = orc.pcg(A, b, tol=1e-12, pc=pc, L=L)
        assert st2 == 0
        np.testing.assert_allclose(x2, x, rtol=1e-9, atol=1e-11)


def test_true_residual_reaches_tolerance(orc):
    A, _, _, _ = synth.diffusion_batch(1, seed=2, side_lo=20, side_hi=20)
    b = synth.normal(A.m, seed=5).astype(np.float64)
    x, st, it = orc.pcg(A, b, tol=1e-8, pc="jacobi")
    assert st == 0 and it > 1
    r = b - A.to_dense() @ x
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("which", ["1d", "2d"])
def test_eigenvector_rhs_one_iteration(orc, which):
    if which == "1d":
        N = 31
        A = synth.poisson1d(N)
        v = np.sin(np.arange(1, N + 1) * 3 * np.pi / (N + 1))
        lam = 2 - 2 * np.cos(3 * np.pi / (N + 1))
    else:
        N = 9
        A = synth.poisson2d(N)
        ix, iy = np.meshgrid(np.arange(1, N + 1), np.arange(1, N + 1), indexing="ij")
        v = (np.sin(ix * 2 * np.pi / (N + 1)) * np.sin(iy * 4 * np.pi / (N + 1))).ravel()
        lam = (2 - 2 * np.cos(2 * np.pi / (N + 1))) + (2 - 2 * np.cos(4 * np.pi / (N + 1)))
    x, st, it = orc.pcg(A, v, tol=1e-10)
    assert st == 0 and it == 1
    np.testing.assert_allclose(x, v / lam, atol=1e-12)


def test_ic0_of_tridiagonal_is_exact_cholesky(orc):
    N = 40
    A = synth.poisson1d(N)
    l_ip, l_ix, l_v = orc.ic0(A)
    Ld = synth.CSR(N, N, l_ip, l_ix, np.zeros(l_ix.size, np.float32)).to_dense()
    rows = np.repeat(np.arange(N), np.diff(l_ip))
    Ld[rows, l_ix] = l_v
    np.testing.assert_allclose(Ld, np.linalg.cholesky(A.to_dense()), atol=1e-13)
    b = synth.normal(N, seed=1).astype(np.float64)
    x, st, it = orc.pcg(A, b, tol=1e-10, pc="ic0", L=(l_ip, l_ix, l_v))
    assert st == 0 and it == 1


def test_ic0_matches_a_on_pattern(orc):
    """IC(0): (L L^T)_ij = a_ij on every stored (i, j) of tril(A)."""
    A = synth.diffusion2d(6, 1.0, seed=9)
    l_ip, l_ix, l_v = orc.ic0(A)
    n = A.m
    Ld = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(l_ip))
    Ld[rows, l_ix] = l_v
    LLt = Ld @ Ld.T
    Ad = A.to_dense()
    np.testing.assert_allclose(LLt[rows, l_ix], Ad[rows, l_ix], atol=1e-12)


def test_triangular_solves_match_dense(orc):
    A = synth.diffusion2d(5, 0.5, seed=1)
    l_ip, l_ix, l_v = orc.ic0(A)
    n = A.m
    Ld = np.zeros((n, n))
    Ld[np.repeat(np.arange(n), np.diff(l_ip)), l_ix] = l_v
    r = synth.normal(n, seed=2).astype(np.float64)
    np.testing.assert_allclose(orc.trsv_lower(l_ip, l_ix, l_v, r), np.linalg.solve(Ld, r),
                               atol=1e-12)
    np.testing.assert_allclose(orc.trsv_lower_t(l_ip, l_ix, l_v, r), np.linalg.solve(Ld.T, r),
                               atol=1e-12)


def test_constant_diagonal_jacobi_equals_cg(orc):
    A = synth.poisson2d(12)
    b = synth.normal(A.m, seed=8).astype(np.float64)
    _, _, it0, h0 = orc.pcg(A, b, tol=1e-8, hist=True)
    _, _, it1, h1 = orc.pcg(A, b, tol=1e-8, pc="jacobi", hist=True)
    assert it0 == it1
    np.testing.assert_allclose(h0, h1, rtol=1e-8)


def test_identity_factor_is_plain_cg(orc):
    A = synth.diffusion2d(9, 1.0, seed=4)
    b = synth.normal(A.m, seed=3).astype(np.float64)
    n = A.m
    L = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    _, _, it0, h0 = orc.pcg(A, b, tol=1e-8, hist=True)
    _, _, it1, h1 = orc.pcg(A, b, tol=1e-8, pc="llt", L=L, hist=True)
    assert it0 == it1
    np.testing.assert_allclose(h0, h1, rtol=1e-10)


def test_llt_matches_dense_preconditioned_cg(orc):
    """M = L L^T applied through two sparse products equals the dense M."""
    A = synth.diffusion2d(6, 1.0, seed=5)
    l_ip, l_ix, _ = orc.tril_pattern(A)
    rng = np.random.default_rng(0)
    l_v = rng.uniform(0.1, 0.3, l_ix.size)
    rows = np.repeat(np.arange(A.m), np.diff(l_ip))
    l_v[rows == l_ix] = 1.0
    Ld = np.zeros((A.m, A.m))
    Ld[rows, l_ix] = l_v
    M = Ld @ Ld.T
    b = synth.normal(A.m, seed=6).astype(np.float64)
    # one PCG iteration by hand with the dense M
    r0 = b
    z0 = M @ r0
    q = A.to_dense() @ z0
    alpha = (r0 @ z0) / (z0 @ q)
    x1 = alpha * z0
    x, st, it = orc.pcg(A, b, tol=1e-30, maxit=1, pc="llt", L=(l_ip, l_ix, l_v))
    assert st == 1 and it == 1
    np.testing.assert_allclose(x, x1, rtol=1e-12, atol=1e-14)


def test_status_codes(orc):
    A = synth.poisson2d(8)
    b = synth.normal(A.m, seed=1).astype(np.float64)
    _, st, it = orc.pcg(A, b, tol=1e-12, maxit=3)
    assert st == 1 and it == 3                         # max iterations
    bad = b.copy()
    bad[5] = np.nan
    _, st, _ = orc.pcg(A, bad, tol=1e-8)
    assert st == 3                                     # non-finite
    n = A.m
    L = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    # M = L L^T is semi-definite with a zero diagonal entry: r^T M r can vanish
    Lz = (L[0], L[1], np.where(np.arange(n) % 2 == 0, 0.0, 1.0))
    e = np.zeros(n)
    e[0] = 1.0                                         # r0 in the null space of M
    _, st, _ = orc.pcg(A, e, tol=1e-8, pc="llt", L=Lz)
    assert st == 2                                     # breakdown
    x, st, it = orc.pcg(A, np.zeros(n), tol=1e-8)
    assert st == 0 and it == 0 and np.all(x == 0)


def test_solve_adjoint_finite_differences(orc):
    """grad_A of J = g^T A^{-1} b is -(lam x^T) on mask(A) with lam = A^{-T} g."""
    A = synth.diffusion2d(4, 1.0, seed=7)
    A = synth.with_values(A, np.round(A.values * 256) / 256)
    b = synth.normal(A.m, seed=1).astype(np.float64)
    g = synth.normal(A.m, seed=2).astype(np.float64)
    x, st, _ = orc.pcg(A, b, tol=1e-14)
    lam, ga = orc.solve_adjoint(A, x, g, tol=1e-14)
    np.testing.assert_allclose(lam, np.linalg.solve(A.to_dense().T, g), rtol=1e-9, atol=1e-12)
    rows = np.repeat(np.arange(A.m), A.row_lengths())
    h = 1.0 / 256
    for e in range(0, A.nnz, 3):
        # perturb the single stored entry e (not its symmetric partner)
        Ad = A.to_dense()
        Ap, Am = Ad.copy(), Ad.copy()
        Ap[rows[e], A.indices[e]] += h
        Am[rows[e], A.indices[e]] -= h
        fd = (g @ np.linalg.solve(Ap, b) - g @ np.linalg.solve(Am, b)) / (2 * h)
        assert abs(fd - ga[e]) < 1e-4 * (1 + abs(ga[e]))


@pytest.mark.parametrize("N", [1, 2, 17, 64])
def test_a_n_solve_is_the_discrete_green_function(orc, N):
    """A_N (Section 4's 1D model problem) has the closed-form inverse
    (A_N^-1)_ij = min(i, j) (N + 1 - max(i, j)) / (N + 1), i, j = 1..N (the discrete Green's
    function); CG reaches it within N iterations (A_N has N distinct eigenvalues)."""
    A = synth.poisson1d(N)
    i = np.arange(1, N + 1)
    G = np.minimum.outer(i, i) * (N + 1 - np.maximum.outer(i, i)) / (N + 1)
    rng = np.random.default_rng(N)
    b = rng.normal(size=N)
    x, st, it = orc.pcg(A, b, tol=1e-13)
    assert st == 0 and it <= N
    np.testing.assert_allclose(x, G @ b, rtol=1e-10, atol=1e-12 * np.abs(G @ b).max())
    for j in (0, N - 1, N // 2):                       # columns of the inverse
        e = np.zeros(N)
        e[j] = 1.0
        xj, st, _ = orc.pcg(A, e, tol=1e-13, pc="jacobi")
        assert st == 0
        np.testing.assert_allclose(xj, G[:, j], rtol=1e-10, atol=1e-13)
