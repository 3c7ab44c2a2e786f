"""Pins for the oracle's SpGEMM forward and backward (CPU only).

* pattern: brute-force boolean product of the dense masks (structural reading of
  mask(.), no numerical-zero dropping);
* values: dense product;
* grads: torch FP64 autograd of <V, (A B) masked to mask(C)> w.r.t. the stored
  values of A and B (Table 1, SpSpMM rows), plus central differences;
* closed forms for the 3D 7-point Poisson square on a 64^3 grid.
"""
import json
import os

import numpy as np
import pytest
import torch

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_csr(m, n, seed, density):
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    vals = rng.uniform(-1, 1, (m, n)) * mask
    # keep explicit zeros in the pattern to exercise the structural mask
    d = np.where(mask, vals, 0.0)
    A = synth.from_dense(np.where(mask, 1.0, 0.0))
    rows = np.repeat(np.arange(m), A.row_lengths())
    v = d[rows, A.indices].astype(np.float32)
    if v.size:
        v[0] = 0.0                              # an explicit stored zero
    return synth.CSR(m, n, A.indptr, A.indices, v), mask


@pytest.mark.parametrize("m,n,p,da,db", [(6, 5, 7, 0.4, 0.4), (12, 9, 10, 0.2, 0.5),
                                          (1, 1, 1, 1.0, 1.0), (5, 8, 3, 0.0, 0.5)])
def test_spgemm_pattern_and_values(orc, m, n, p, da, db):
    A, ma = _rand_csr(m, n, seed=m + 10 * n, density=da)
    B, mb = _rand_csr(n, p, seed=p + 7, density=db)
    c_ip, c_ix, c_v = orc.spgemm(A, B)
    brute = (ma.astype(np.int64) @ mb.astype(np.int64)) > 0
    C = synth.CSR(m, p, c_ip, c_ix, np.ones(c_ix.size, np.float32))
    np.testing.assert_array_equal(C.to_dense() > 0, brute)
    for i in range(m):
        assert np.all(np.diff(c_ix[c_ip[i]:c_ip[i + 1]]) > 0)
    dense = A.to_dense() @ B.to_dense()
    rows = np.repeat(np.arange(m), np.diff(c_ip))
    np.testing.assert_allclose(c_v, dense[rows, c_ix], atol=1e-14)
    row_nnz, row_prod, tot = orc.spgemm_count(A, B)
    assert tot == c_ix.size
    np.testing.assert_array_equal(row_prod, (ma.astype(np.int64) @ mb.sum(1)))


def test_spgemm_grads_match_torch_autograd(orc):
    A, _ = _rand_csr(9, 7, seed=1, density=0.35)
    B, _ = _rand_csr(7, 8, seed=2, density=0.35)
    c_ip, c_ix, _ = orc.spgemm(A, B)
    gc = synth.normal(c_ix.size, seed=3).astype(np.float64)
    ga = orc.spgemm_grad_a(A, B, c_ip, c_ix, gc)
    gb = orc.spgemm_grad_b(A, B, c_ip, c_ix, gc)

    a_rows = np.repeat(np.arange(A.m), A.row_lengths())
    b_rows = np.repeat(np.arange(B.m), B.row_lengths())
    c_rows = np.repeat(np.arange(A.m), np.diff(c_ip))
    av = torch.tensor(A.values.astype(np.float64), requires_grad=True)
    bv = torch.tensor(B.values.astype(np.float64), requires_grad=True)
    Ad = torch.zeros(A.m, A.n, dtype=torch.float64).index_put(
        (torch.tensor(a_rows), torch.tensor(A.indices.astype(np.int64))), av)
    Bd = torch.zeros(B.m, B.n, dtype=torch.float64).index_put(
        (torch.tensor(b_rows), torch.tensor(B.indices.astype(np.int64))), bv)
    Cd = Ad @ Bd
    z = (Cd[torch.tensor(c_rows), torch.tensor(c_ix.astype(np.int64))] * torch.tensor(gc)).sum()
    z.backward()
    np.testing.assert_allclose(ga, av.grad.numpy(), atol=1e-13)
    np.testing.assert_allclose(gb, bv.grad.numpy(), atol=1e-13)


def test_spgemm_grads_finite_differences(orc):
    A, _ = _rand_csr(5, 6, seed=11, density=0.5)
    B, _ = _rand_csr(6, 4, seed=12, density=0.5)
    A = synth.with_values(A, np.round(A.values * 64) / 64)   # dyadic: v +- h stays exact
    B = synth.with_values(B, np.round(B.values * 64) / 64)
    c_ip, c_ix, _ = orc.spgemm(A, B)
    gc = synth.normal(c_ix.size, seed=13).astype(np.float64)
    ga = orc.spgemm_grad_a(A, B, c_ip, c_ix, gc)
    gb = orc.spgemm_grad_b(A, B, c_ip, c_ix, gc)

    def f(av, bv):
        _, _, cv = orc.spgemm(synth.with_values(A, av), synth.with_values(B, bv))
        return float(cv @ gc)
    h = 0.25                                    # exact in float32; f is bilinear
    for e in range(A.nnz):
        vp, vm = A.values.copy(), A.values.copy()
        vp[e] += h
        vm[e] -= h
        assert abs((f(vp, B.values) - f(vm, B.values)) / (2 * h) - ga[e]) < 1e-12
    for e in range(B.nnz):
        vp, vm = B.values.copy(), B.values.copy()
        vp[e] += h
        vm[e] -= h
        assert abs((f(A.values, vp) - f(A.values, vm)) / (2 * h) - gb[e]) < 1e-12


def _poisson3d_square_closed_form(n):
    """nnz of A^2 for the 7-point stencil: offsets with |d|_1 <= 2 that stay in the grid;
    products = sum over rows of len(row)^2 (A symmetric)."""
    nnz = n ** 3                                             # d = 0
    nnz += 6 * (n - 1) * n * n                               # one axis, |d| = 1
    nnz += 6 * (n - 2) * n * n                               # one axis, |d| = 2
    nnz += 12 * (n - 1) * (n - 1) * n                        # two axes, |d| = 1 each
    # per axis a point has 1 neighbour at the two ends and 2 inside
    counts = {1: 2, 2: n - 2}
    prods = 0
    for a, ca in counts.items():
        for b, cb in counts.items():
            for c, cc in counts.items():
                prods += ca * cb * cc * (1 + a + b + c) ** 2
    return nnz, prods


def test_poisson3d_square_counts(orc):
    with open(os.path.join(GOLDEN, "poisson3d_square_64.json")) as fh:
        gold = json.load(fh)
    n = gold["n"]
    nnz_cf, prods_cf = _poisson3d_square_closed_form(n)
    assert (nnz_cf, prods_cf) == (gold["nnz_C"], gold["products"])
    A = synth.poisson3d(n)
    row_nnz, row_prod, tot = orc.spgemm_count(A, A)
    assert tot == nnz_cf
    assert int(row_prod.sum()) == prods_cf
    # an interior row of A^2 has the 25 offsets of the |d|_1 <= 2 stencil
    mid = (n // 2 * n + n // 2) * n + n // 2
    assert row_nnz[mid] == 25


def test_poisson1d_square_values(orc):
    """A_N^2 is pentadiagonal [1 -4 6 -4 1] inside, with 5 and -4 in the corners."""
    N = 12
    A = synth.poisson1d(N)
    c_ip, c_ix, c_v = orc.spgemm(A, A)
    C = synth.CSR(N, N, c_ip, c_ix, c_v.astype(np.float32)).to_dense()
    mid = N // 2
    np.testing.assert_array_equal(C[mid, mid - 2: mid + 3], [1, -4, 6, -4, 1])
    assert C[0, 0] == 5 and C[0, 1] == -4 and C[0, 2] == 1
