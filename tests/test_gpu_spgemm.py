"""GPU parity of SpGEMM (pattern bit-exact, values and both gradients within 1e-5
normalised) against the FP64 oracle, through the C ABI (Section 3.1.2, Table 1)."""
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


def _explicit_zero(A):
    v = A.values.copy()
    if v.size:
        v[v.size // 3] = 0.0
    return synth.with_values(A, v)


PAIRS = {
    # the two SpGEMM workloads at full size (n = 262,144)
    "poisson3d_64_sq": lambda: (synth.poisson3d(64),) * 2,
    "random8_262k": lambda: (synth.random_k_per_row(262144, 8, seed=1),
                             synth.random_k_per_row(262144, 8, seed=2)),
    # small / ragged: empty rows, a hub row, explicit zeros, rectangular
    "ragged": lambda: (_explicit_zero(synth.empty_rows_csr(700, 500, seed=3, max_len=12)),
                       synth.empty_rows_csr(500, 900, seed=4, max_len=9)),
    # rows with more than 512 products (block path), several bitmap chunks (p > 262144)
    "big_rows_wide": lambda: (synth.powerlaw_csr(3000, seed=5, max_len=400),
                              synth.random_k_per_row(3000, 6, seed=6, ncols=600000)),
    "poisson1d_sq": lambda: (synth.poisson1d(1000),) * 2,
    # rows of A with more than 32 entries whose B rows are mostly empty (few products)
    "long_a_rows_empty_b": lambda: (synth.empty_rows_csr(600, 800, seed=7, p_empty=0.1, max_len=60),
                                    synth.empty_rows_csr(800, 300, seed=8, p_empty=0.93, max_len=3)),
}


@pytest.fixture(scope="module", params=list(PAIRS))
def pair(request):
    A, B = PAIRS[request.param]()
    if A.values is B.values:
        B = synth.with_values(B, synth.uniform(B.nnz, seed=9))
    A = synth.with_values(A, synth.uniform(A.nnz, seed=8) if A.nnz > 0 else A.values)
    dA, dB = spx.CSR.from_host(A), spx.CSR.from_host(B)
    plan = spx.SpGEMMPlan(dA, dB)
    return request.param, A, B, dA, dB, plan


def test_pattern_bit_exact(pair):
    name, A, B, dA, dB, plan = pair
    r_ip, r_ix, _ = oracle.spgemm(A, B)
    np.testing.assert_array_equal(host(plan.C.indptr), r_ip)
    np.testing.assert_array_equal(host(plan.C.indices), r_ix)
    _, row_prod, _ = oracle.spgemm_count(A, B)
    assert plan.products == int(row_prod.sum())
    # the same steps without the host read-backs (sizes known): the same pattern
    from paper_2212_05159_gb300 import abi
    sA, sB = dA.struct(), dB.struct()
    scratch = abi.workspace(4 * plan.products, "cuda")
    c_ip = torch.full_like(plan.C.indptr, -1)
    c_ix = torch.full((max(r_ix.size, 1),), -1, dtype=torch.int32, device="cuda")
    assert abi.spx_spgemm_analyse(sA, sB, plan.ws, read_back=False) is None
    assert abi.spx_spgemm_symbolic(sA, sB, c_ip, plan.ws, scratch, plan.products, read_back=False) is None
    abi.spx_spgemm_fill(sA, c_ip, c_ix, plan.ws, scratch)
    np.testing.assert_array_equal(host(c_ip), r_ip)
    np.testing.assert_array_equal(host(c_ix)[: r_ix.size], r_ix)


def test_values(pair):
    name, A, B, dA, dB, plan = pair
    _, _, r_v = oracle.spgemm(A, B)
    _, _, n_v = oracle.spgemm(abs_csr(A), abs_csr(B))
    got = host(plan.numeric())
    assert_close_normalised(got, r_v, n_v, what=f"spgemm values {name}")
    again = host(plan.numeric())
    assert np.array_equal(got, again)                      # deterministic


def test_backward(pair):
    name, A, B, dA, dB, plan = pair
    c_ip, c_ix = host(plan.C.indptr), host(plan.C.indices)
    gc = synth.normal(c_ix.size, seed=11)
    ga, gb = plan.backward(dev(gc))
    assert_close_normalised(host(ga), oracle.spgemm_grad_a(A, B, c_ip, c_ix, gc),
                            oracle.spgemm_grad_a(A, abs_csr(B), c_ip, c_ix, np.abs(gc)),
                            what=f"spgemm grad A {name}")
    assert_close_normalised(host(gb), oracle.spgemm_grad_b(A, B, c_ip, c_ix, gc),
                            oracle.spgemm_grad_b(abs_csr(A), B, c_ip, c_ix, np.abs(gc)),
                            what=f"spgemm grad B {name}")


def test_autograd_function(pair):
    name, A, B, dA, dB, plan = pair
    if A.m > 5000:
        pytest.skip("covered by test_backward at this size")
    from paper_2212_05159_gb300.autograd import SpGEMM
    av = dev(A.values).requires_grad_(True)
    bv = dev(B.values).requires_grad_(True)
    cv = SpGEMM.apply(av, bv, plan)
    gc = synth.normal(cv.numel(), seed=12)
    cv.backward(dev(gc))
    c_ip, c_ix = host(plan.C.indptr), host(plan.C.indices)
    assert_close_normalised(host(av.grad), oracle.spgemm_grad_a(A, B, c_ip, c_ix, gc),
                            oracle.spgemm_grad_a(A, abs_csr(B), c_ip, c_ix, np.abs(gc)), what="autograd gA")
    assert_close_normalised(host(bv.grad), oracle.spgemm_grad_b(A, B, c_ip, c_ix, gc),
                            oracle.spgemm_grad_b(abs_csr(A), B, c_ip, c_ix, np.abs(gc)), what="autograd gB")


def test_empty_product():
    A = synth.CSR(4, 3, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    B = synth.random_k_per_row(3, 2, seed=1)
    plan = spx.SpGEMMPlan(spx.CSR.from_host(A), spx.CSR.from_host(B))
    assert plan.C.nnz == 0 and np.all(host(plan.C.indptr) == 0)
