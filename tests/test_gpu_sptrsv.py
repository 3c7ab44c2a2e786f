"""GPU parity of the batched sparse triangular solve and its VJP (Section 3.1.5) against the
FP64 oracle: IC(0) factors of a diffusion batch, random lower-triangular systems of ragged
sizes (one of a single row), the transposed solve, the gradients through autograd, and the
zero-pivot status."""
import numpy as np
import pytest
import torch

import synth
from oracle import sptrsv as osp
from helpers import assert_close_normalised

pytestmark = pytest.mark.gpu

spx = pytest.importorskip("paper_2212_05159_gb300")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def random_lower_batch(sizes, seed):
    rng = np.random.default_rng(seed)
    ip, ix, v, ptr = [0], [], [], [0]
    for n in sizes:
        r0 = ptr[-1]
        for i in range(n):
            k = min(i, int(rng.integers(0, 6)))
            cols = sorted(rng.choice(i, k, replace=False)) if k else []
            ix += [r0 + c for c in cols] + [r0 + i]
            v += list(rng.uniform(-0.4, 0.4, len(cols))) + [float(rng.uniform(1.5, 2.5))]
            ip.append(len(ix))
        ptr.append(r0 + n)
    n = ptr[-1]
    return synth.CSR(n, n, np.array(ip, np.int32), np.array(ix, np.int32), np.array(v, np.float32)), \
        np.array(ptr, np.int32)


def ic0_batch():
    A, ptr, _, _ = synth.diffusion_batch(6, seed=3, side_lo=16, side_hi=40, sigma=1.0)
    import oracle
    l_ip, l_ix, l_v = oracle.ic0(A)
    return synth.CSR(A.m, A.m, l_ip, l_ix, l_v.astype(np.float32)), ptr


CASES = {"ic0_diffusion": ic0_batch,
         "random_ragged": lambda: random_lower_batch([1, 7, 300, 1000, 64], seed=1)}


@pytest.mark.parametrize("name", list(CASES))
def test_solves_and_vjp_match_oracle(name):
    L, ptr = CASES[name]()
    dL = spx.CSR.from_host(L)
    solver = spx.TriangularSolver(dL, ptr)
    b = synth.normal(L.m, seed=11)
    v = synth.normal(L.m, seed=12)
    lv = dL.values.clone().requires_grad_(True)
    bt = dev(b).requires_grad_(True)
    from paper_2212_05159_gb300.autograd import SpTRSV
    x = SpTRSV.apply(lv, bt, solver)
    (x * dev(v)).sum().backward()
    assert np.all(host(solver.status) == 0)
    xo, gbo, glo = osp.vjp(L.indptr, L.indices, L.values, b, v)
    # normaliser: the same solves with |L| and |b| (the size of the terms summed)
    Labs = np.abs(L.values.astype(np.float64))
    rows = np.repeat(np.arange(L.m), np.diff(L.indptr))
    on = rows == L.indices
    M = np.where(on, Labs, -Labs)        # comparison matrix: |diag| on the diagonal, -|offdiag| off it
    xa = osp.solve(L.indptr, L.indices, M, np.abs(b))
    assert_close_normalised(host(x), xo, np.abs(xa) + np.abs(xo), rel=2e-5, what=f"x {name}")
    assert_close_normalised(host(bt.grad), gbo, np.abs(gbo).max() * np.ones_like(gbo), rel=2e-5,
                            what=f"grad b {name}")
    assert_close_normalised(host(lv.grad), glo, np.abs(glo).max() * np.ones_like(glo), rel=2e-5,
                            what=f"grad L {name}")


def test_zero_pivot_status():
    L, ptr = random_lower_batch([5, 9], seed=2)
    vals = L.values.copy()
    vals[L.indptr[7] - 1] = 0.0                 # the pivot of row 6 (second system)
    L = synth.CSR(L.m, L.n, L.indptr, L.indices, vals)
    dL = spx.CSR.from_host(L)
    solver = spx.TriangularSolver(dL, ptr)
    solver.solve(dev(synth.normal(L.m, seed=1)))
    assert list(host(solver.status)) == [0, 6]                     # SPX_OK, SPX_BREAKDOWN
