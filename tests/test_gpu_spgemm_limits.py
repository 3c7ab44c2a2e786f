"""SpGEMM (Section 3.1.2, Table 1) on matrices built to sit on both sides of the limits where
the library switches paths: rows of A with 8 / 9 entries and rows of C with 64 / 65 columns
(the small-row kernels of the numeric phase and of gA), columns of A with 8 / 9 and more
entries and rows of B with 8 / 9 entries (gB's one-round path), with C's rows short and long.
Pattern bit-exact; values and both gradients within 1e-5 normalised of the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import abs_csr, assert_close_normalised

pytestmark = pytest.mark.gpu
spx = pytest.importorskip("paper_2212_05159_gb300")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def csr_from_rows(rows, ncols, seed):
    lens = np.array([len(r) for r in rows], dtype=np.int64)
    indptr = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=indptr[1:])
    idx = np.concatenate([np.sort(np.asarray(r, dtype=np.int64)) for r in rows]) if lens.sum() else np.zeros(0)
    return synth.CSR(len(rows), ncols, indptr, idx, synth.uniform(int(lens.sum()), seed=seed))


def wide_rows_pair():
    """B's rows have disjoint columns, so a row of C has exactly the summed lengths of the rows
    of B it picks: rows of A with 6..9 entries give rows of C with 48..81 columns, among them
    exactly 64 (eight rows of 8) and 65 (seven of 8, one of 9); C's rows average above 32."""
    rng = np.random.default_rng(3)
    nb = 3000
    blen = np.where(np.arange(nb) % 3 == 2, 9, 8)
    B = csr_from_rows([[16 * k + j for j in range(blen[k])] for k in range(nb)], 16 * nb, seed=4)
    eights, nines = np.flatnonzero(blen == 8), np.flatnonzero(blen == 9)
    rows = []
    for i in range(2400):
        kind = i % 6
        if kind == 0:                              # 8 entries, C row of 64
            ks = rng.choice(eights, 8, replace=False)
        elif kind == 1:                            # 8 entries, C row of 65
            ks = np.concatenate([rng.choice(eights, 7, replace=False), rng.choice(nines, 1)])
        elif kind == 2:                            # 9 entries (past the small-row limit)
            ks = rng.choice(nb, 9, replace=False)
        elif kind == 3:                            # 7 entries of 9: 63 columns
            ks = rng.choice(nines, 7, replace=False)
        else:
            ks = rng.choice(nb, int(rng.integers(0, 9)), replace=False)
        rows.append(ks.tolist())
    A = csr_from_rows(rows, nb, seed=5)
    return A, B


def deep_columns_pair():
    """Rows of A with one or two entries (C's rows stay short: mean below 32 columns) whose
    columns are chosen so that some columns of A hold exactly 8, 32, 33 and 40 entries (and
    the others about 9); rows of B with 8 or 9 overlapping columns."""
    rng = np.random.default_rng(7)
    nb, ncol_b = 600, 500
    m = 4000
    col_of = rng.integers(4, nb, size=m)
    first = 0
    for col, count in ((0, 32), (1, 33), (2, 8), (3, 40)):
        col_of[first:first + count] = col
        first += count
    rows = []
    for i in range(m):
        ks = {int(col_of[i])}
        if i % 2 == 1:
            ks.add(int(rng.integers(4, nb)))
        rows.append(sorted(ks))
    A = csr_from_rows(rows, nb, seed=8)
    blen = np.where(np.arange(nb) % 2 == 0, 8, 9)
    B = csr_from_rows([sorted({(7 * k + 3 * j) % ncol_b for j in range(blen[k])}) for k in range(nb)], ncol_b,
                      seed=9)
    return A, B


def group_layouts_pair():
    """Rows of A that put the symbolic phase's 8-lane groups in each of their layouts: one entry
    whose B row has 1, 33 or 64 columns (runs of 1 and 64 slots), two entries of 17..32 columns
    (runs of 32), eight of exactly 8 (a lane's registers each, 64 products), five with one row
    of 9..16 columns (packed: 5 x 16 > 64 slots), eight of mixed lengths summing to 64 and 65
    (packed at the product limit, and one past it), empty rows of A and of B; B's rows overlap
    heavily, so most products repeat a column."""
    rng = np.random.default_rng(11)
    ncol = 200
    lens = [0, 1, 8, 8, 8, 8, 8, 8, 8, 8, 9, 12, 16, 17, 25, 32, 33, 40, 64, 3, 2, 5, 7, 4, 6, 15, 1, 0]
    nb = len(lens)
    B = csr_from_rows([sorted(rng.choice(ncol, L, replace=False).tolist()) for L in lens], ncol, seed=12)
    by_len = {}
    for k, L in enumerate(lens):
        by_len.setdefault(L, []).append(k)
    eights = by_len[8]
    templates = [
        [], [by_len[1][0]], [by_len[33][0]], [by_len[64][0]], [by_len[0][0]], [by_len[0][0], by_len[0][1]],
        [by_len[17][0], by_len[32][0]], [by_len[25][0], by_len[17][0]],
        eights,                                                       # 8 x 8 = 64, runs of 8
        [by_len[12][0], by_len[1][0], by_len[2][0], by_len[3][0], by_len[4][0]],        # packed, 22 products
        [by_len[16][0], by_len[15][0], by_len[9][0], by_len[8][0], by_len[7][0],
         by_len[5][0], by_len[3][0], by_len[1][0]],                  # packed, 64 products
        [by_len[16][0], by_len[15][0], by_len[9][0], by_len[8][0], by_len[7][0],
         by_len[6][0], by_len[3][0], by_len[1][0]],                  # 65 products: the warp path
        [by_len[40][0], by_len[8][0], by_len[8][1]],                 # 56 products, R = 64: packed
    ]
    rows = [sorted(set(templates[i % len(templates)])) for i in range(3 * len(templates))]
    A = csr_from_rows(rows, nb, seed=13)
    return A, B


PAIRS = {"wide_rows": wide_rows_pair, "deep_columns": deep_columns_pair, "group_layouts": group_layouts_pair}


@pytest.fixture(scope="module", params=list(PAIRS))
def pair(request):
    A, B = PAIRS[request.param]()
    dA, dB = spx.CSR.from_host(A), spx.CSR.from_host(B)
    return request.param, A, B, spx.SpGEMMPlan(dA, dB)


def test_the_matrices_reach_the_limits(pair):
    name, A, B, plan = pair
    c_ip = host(plan.C.indptr).astype(np.int64)
    c_len, a_len = np.diff(c_ip), np.diff(A.indptr.astype(np.int64))
    at_len = np.bincount(A.indices, minlength=A.n)
    if name == "wide_rows":
        assert {64, 65} <= set(c_len[a_len == 8].tolist()) and (a_len == 9).any()
        assert c_len.mean() > 32
    elif name == "group_layouts":
        b_len = np.diff(B.indptr.astype(np.int64))
        prods = np.array([b_len[A.indices[A.indptr[i]:A.indptr[i + 1]]].sum() for i in range(A.m)])
        assert {0, 1, 22, 33, 49, 56, 64, 65} <= set(prods.tolist())
        assert (prods[a_len == 8] == 64).any() and (prods[a_len == 8] == 65).any()
        assert (c_len < prods).any()                  # repeated columns to merge
    else:
        assert {8, 32, 33, 40} <= set(at_len.tolist()) and {8, 9} <= set(np.diff(B.indptr).tolist())
        assert c_len.mean() <= 32


def test_pattern_values_and_gradients(pair):
    name, A, B, plan = pair
    r_ip, r_ix, r_v = oracle.spgemm(A, B)
    np.testing.assert_array_equal(host(plan.C.indptr), r_ip)
    np.testing.assert_array_equal(host(plan.C.indices), r_ix)
    _, _, n_v = oracle.spgemm(abs_csr(A), abs_csr(B))
    got = host(plan.numeric())
    assert_close_normalised(got, r_v, n_v, what=f"spgemm values {name}")
    assert np.array_equal(got, host(plan.numeric()))
    gc = synth.normal(r_ix.size, seed=13)
    ga, gb = plan.backward(dev(gc))
    assert_close_normalised(host(ga), oracle.spgemm_grad_a(A, B, r_ip, r_ix, gc),
                            oracle.spgemm_grad_a(A, abs_csr(B), r_ip, r_ix, np.abs(gc)), what=f"grad A {name}")
    assert_close_normalised(host(gb), oracle.spgemm_grad_b(A, B, r_ip, r_ix, gc),
                            oracle.spgemm_grad_b(abs_csr(A), B, r_ip, r_ix, np.abs(gc)), what=f"grad B {name}")
    ga2, gb2 = plan.backward(dev(gc))
    assert np.array_equal(host(ga), host(ga2)) and np.array_equal(host(gb), host(gb2))
