"""GPU parity of sparse + sparse (Section 3.1.4, Table 1 Sp + Sp) against the FP64 oracle:
the union pattern bit-exact, the values within the normalised tolerance, the gradients, the
ragged / empty cases, and the n = 2^20 power-law pair on sampled rows."""
import numpy as np
import pytest
import torch

import synth
from oracle import spadd as ospadd
from helpers import assert_close_normalised

pytestmark = pytest.mark.gpu

spx = pytest.importorskip("paper_2212_05159_gb300")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


PAIRS = {
    "poisson_vs_random": lambda: (synth.poisson2d(40), synth.random_k_per_row(1600, 7, seed=1, ncols=1600)),
    "ragged_empty_rows": lambda: (synth.empty_rows_csr(3001, 2500, seed=4, max_len=70),
                                  synth.empty_rows_csr(3001, 2500, seed=5, max_len=30)),
    "powerlaw_pair": lambda: (synth.powerlaw_csr(20000, seed=1, max_len=2000),
                              synth.powerlaw_csr(20000, seed=2, max_len=2000)),
    "same_pattern": lambda: (synth.poisson3d(12), synth.with_values(synth.poisson3d(12), synth.uniform(
        synth.poisson3d(12).nnz, seed=9))),
}


@pytest.mark.parametrize("name", list(PAIRS))
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (1.0, -1.0), (0.5, -2.5)])
def test_spadd_matches_oracle(name, alpha, beta):
    A, B = PAIRS[name]()
    dA, dB = spx.CSR.from_host(A), spx.CSR.from_host(B)
    plan = spx.SpAddPlan(dA, dB)
    c = host(plan.numeric(alpha, beta))
    c_ip, c_ix, c_v = ospadd.spadd(A, B, alpha, beta)
    np.testing.assert_array_equal(host(plan.C.indptr), c_ip)
    np.testing.assert_array_equal(host(plan.C.indices), c_ix)
    Aa = synth.CSR(A.m, A.n, A.indptr, A.indices, np.abs(A.values))
    Ba = synth.CSR(B.m, B.n, B.indptr, B.indices, np.abs(B.values))
    _, _, norm = ospadd.spadd(Aa, Ba, abs(alpha), abs(beta))
    assert_close_normalised(c, c_v, norm, what=f"spadd {name}")
    gc = synth.normal(c_ix.size, seed=7)
    ga, gb = plan.backward(dev(gc), alpha, beta)
    oa, ob = ospadd.spadd_backward(A, B, c_ip, c_ix, gc, alpha, beta)
    # one float32 product each: within one rounding of the exact value
    np.testing.assert_allclose(host(ga), oa, rtol=1e-7, atol=0)
    np.testing.assert_allclose(host(gb), ob, rtol=1e-7, atol=0)


def test_autograd_and_empty_operand():
    A = synth.poisson2d(16)
    Z = synth.CSR(A.m, A.n, np.zeros(A.m + 1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    dA, dZ = spx.CSR.from_host(A), spx.CSR.from_host(Z)
    plan = spx.SpAddPlan(dA, dZ)
    np.testing.assert_array_equal(host(plan.C.indices), A.indices)
    a = dA.values.clone().requires_grad_(True)
    b = torch.zeros(0, device="cuda", requires_grad=True)
    from paper_2212_05159_gb300.autograd import SpAdd
    c = SpAdd.apply(a, b, plan, 2.0, 3.0)
    np.testing.assert_allclose(host(c), 2.0 * A.values, rtol=1e-7)
    c.sum().backward()
    np.testing.assert_allclose(host(a.grad), 2.0, rtol=0)


def test_full_size_powerlaw_pair_sampled():
    """Two n = 2^20 power-law matrices (the benchmark's size): pattern and values of sampled
    rows against the oracle run on those rows alone."""
    A = synth.powerlaw_csr(1 << 20, seed=0)
    B = synth.powerlaw_csr(1 << 20, seed=3)
    dA, dB = spx.CSR.from_host(A), spx.CSR.from_host(B)
    plan = spx.SpAddPlan(dA, dB)
    c = host(plan.numeric(1.0, -0.5))
    c_ip, c_ix = host(plan.C.indptr), host(plan.C.indices)
    rng = np.random.default_rng(0)
    lens = np.diff(A.indptr)
    rows = np.concatenate([rng.choice(A.m, 300, replace=False), np.argsort(lens)[-10:]])
    for i in rows:
        sa = synth.CSR(1, A.n, np.array([0, lens[i]], np.int32), A.indices[A.indptr[i]:A.indptr[i + 1]],
                       A.values[A.indptr[i]:A.indptr[i + 1]])
        lb = B.indptr[i + 1] - B.indptr[i]
        sb = synth.CSR(1, B.n, np.array([0, lb], np.int32), B.indices[B.indptr[i]:B.indptr[i + 1]],
                       B.values[B.indptr[i]:B.indptr[i + 1]])
        _, ix, v = ospadd.spadd(sa, sb, 1.0, -0.5)
        np.testing.assert_array_equal(c_ix[c_ip[i]:c_ip[i + 1]], ix)
        np.testing.assert_allclose(c[c_ip[i]:c_ip[i + 1]], v, rtol=1e-6, atol=1e-7)
