"""GPU parity of SPAI by gradient descent (Section 4.6) against the FP64 oracle: the
residual, the deterministic inner product, one descent step, the whole descent on the
paper's 8 x 8 Poisson problem, and a 256^2 problem checked on its loss history."""
import numpy as np
import pytest
import torch

import synth
from oracle import spai as ospai
from helpers import assert_close_normalised

pytestmark = pytest.mark.gpu

spx = pytest.importorskip("paper_2212_05159_gb300")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def test_dot_is_exact_enough_and_reproducible():
    from paper_2212_05159_gb300 import abi
    rng = np.random.default_rng(0)
    for n in (0, 1, 255, 1000, 3_000_001):
        x = rng.standard_normal(n).astype(np.float32)
        y = rng.standard_normal(n).astype(np.float32)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        ws = abi.workspace(abi.spx_dot_workspace_size(n), "cuda")
        dx, dy = dev(x), dev(y)
        abi.spx_dot(dx, dy, out, ws)
        ref = float(np.dot(x.astype(np.float64), y.astype(np.float64)))
        scale = float(np.abs(x.astype(np.float64)) @ np.abs(y.astype(np.float64))) + 1e-300
        assert abs(float(host(out)[0]) - ref) <= 1e-12 * scale
        first = float(host(out)[0])
        abi.spx_dot(dx, dy, out, ws)
        assert float(host(out)[0]) == first                      # fixed order: bit-identical


def test_residual_and_gradient_match_oracle():
    A = synth.poisson2d(12)
    dA = spx.CSR.from_host(A)
    d = spx.spai.SPAIDescent(dA)
    rng = np.random.default_rng(3)
    m = rng.standard_normal(A.nnz).astype(np.float32)
    d.M.values.copy_(dev(m))
    g = d.gradient()
    loss_o, g_o = ospai.loss_and_grad(A, m)
    s = host(d.scal)
    loss = s[0] / 4.0 + (A.m - int(host(d.diag)[0]))
    assert loss == pytest.approx(loss_o, rel=1e-5)
    # normaliser: 2 ((I + |M||A|) |A|^T) on mask(M), the sum of the terms' magnitudes
    Ad = np.zeros((A.m, A.n))
    Md = np.zeros((A.m, A.n))
    rows = np.repeat(np.arange(A.m), np.diff(A.indptr))
    Ad[rows, A.indices] = np.abs(A.values)
    Md[rows, A.indices] = np.abs(m)
    norm = (2.0 * (np.eye(A.m) + Md @ Ad) @ Ad.T)[rows, A.indices]
    assert_close_normalised(host(g), g_o, norm, what="SPAI gradient")


def test_descent_matches_oracle_steps_and_reaches_the_static_pattern_spai():
    """The paper's problem: 2D Poisson 8 x 8, M = mask(A) to ||grad|| < 0.01."""
    A = synth.poisson2d(8)
    dA = spx.CSR.from_host(A)
    d = spx.spai.SPAIDescent(dA)
    hist = d.run(gtol=1e-2)
    m_o, hist_o = ospai.gradient_descent(A, gtol=1e-2)
    assert abs(len(hist) - len(hist_o)) <= 1
    n = min(len(hist), len(hist_o))
    for (l, gn), (lo, gno) in zip(hist[:n], hist_o[:n]):
        assert l == pytest.approx(lo, rel=2e-4, abs=1e-4)
    m = host(d.values)
    np.testing.assert_allclose(m, m_o, rtol=0, atol=2e-4 * np.abs(m_o).max())
    loss_ls = ospai.loss_and_grad(A, ospai.static_pattern_spai(A))[0]
    assert hist[-1][0] == pytest.approx(loss_ls, rel=1e-3)
    assert hist[-1][1] < 1e-2


def test_descent_256_squared_loss_history():
    """The paper's largest size (N = 65,536): the loss decreases at every step and the
    first steps match the oracle's."""
    A = synth.poisson2d(256)
    dA = spx.CSR.from_host(A)
    d = spx.spai.SPAIDescent(dA)
    hist = d.run(gtol=1e-2, max_it=4)
    _, hist_o = ospai.gradient_descent(A, gtol=1e-2, max_it=4)
    for (l, _), (lo, _) in zip(hist, hist_o):
        assert l == pytest.approx(lo, rel=1e-4)
    losses = [h[0] for h in hist]
    assert all(b < a for a, b in zip(losses, losses[1:]))
