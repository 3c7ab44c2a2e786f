"""Pins for the oracle's network (CPU only): closed forms on the 1D model problem
(Section 4, A_N), the Jacobi start, scale invariance and finite differences."""
import numpy as np
import torch

import synth
from oracle import mpnn


def test_features_closed_form_on_A_N():
    """A_N: e_ij = -1/2 off the diagonal; sums -1 inside and -1/2 at both ends."""
    N = 9
    A = synth.poisson1d(N)
    p = mpnn.params_to_torch(mpnn.init_params(0), requires_grad=False)
    _, _, g = mpnn.forward(A, p, want_graph=True)
    f = g["f"].numpy()
    np.testing.assert_allclose(f[:, 0], 1.0)
    expect = np.full(N, -1.0)
    expect[0] = expect[-1] = -0.5
    np.testing.assert_allclose(f[:, 1], expect, atol=1e-15)
    np.testing.assert_allclose(f[:, 2], -0.5, atol=1e-15)
    np.testing.assert_allclose(f[:, 3], -0.5, atol=1e-15)


def test_initial_factor_is_jacobi():
    A = synth.diffusion2d(6, 1.0, seed=3)
    p = mpnn.params_to_torch(mpnn.init_params(1), requires_grad=False)
    L, (ri, ci) = mpnn.forward(A, p)
    L = L.numpy()
    diag = ri == ci
    d = np.zeros(A.m)
    rows = np.repeat(np.arange(A.m), A.row_lengths())
    on = rows == A.indices
    d[rows[on]] = A.values[on]
    # bd is stored in float32, so softplus(bd) = 1 up to float32 rounding of log(e - 1)
    np.testing.assert_allclose(L[diag], 1 / np.sqrt(d), rtol=1e-8)
    assert np.all(L[~diag] == 0)


def test_scale_invariance():
    """Scaling A by c leaves e and the features unchanged, so L scales by c^(-1/2)."""
    A = synth.diffusion2d(5, 1.5, seed=2)
    p = mpnn.init_params(4)
    p["v"] = np.random.default_rng(0).normal(0, 0.5, p["v"].shape).astype(np.float32)
    tp = mpnn.params_to_torch(p, requires_grad=False)
    L1, _ = mpnn.forward(A, tp)
    A4 = synth.with_values(A, A.values * 4.0)
    L4, _ = mpnn.forward(A4, tp)
    np.testing.assert_allclose(L4.numpy(), L1.numpy() / 2.0, rtol=1e-12, atol=1e-15)


def test_aggregation_on_constant_state():
    """With h constant across nodes, E h = (1 + sum_{j!=i} e_ij) h row by row."""
    A = synth.poisson1d(7)
    p = mpnn.params_to_torch(mpnn.init_params(0), requires_grad=False)
    _, _, g = mpnn.forward(A, p, want_graph=True)
    e = g["e"]
    rows = torch.from_numpy(np.repeat(np.arange(A.m), A.row_lengths()))
    cols = torch.from_numpy(A.indices.astype(np.int64))
    h = torch.ones(A.m, 3, dtype=torch.float64)
    agg = torch.zeros(A.m, 3, dtype=torch.float64).index_add(0, rows, e[:, None] * h[cols])
    expect = 1.0 + g["f"][:, 1]
    np.testing.assert_allclose(agg.numpy(), np.repeat(expect.numpy()[:, None], 3, axis=1), atol=1e-15)


def test_gradients_by_finite_differences():
    A = synth.diffusion2d(3, 1.0, seed=1)
    p = mpnn.init_params(5)
    rng = np.random.default_rng(2)
    p["v"] = rng.normal(0, 0.5, p["v"].shape).astype(np.float32)
    tp = mpnn.params_to_torch(p)
    L, _ = mpnn.forward(A, tp)
    wts = torch.from_numpy(rng.normal(size=L.numel()))
    (L * wts).sum().backward()
    for name, idx in (("W1", (3, 5)), ("Ua", (2, 7)), ("v", (4,)), ("u", (1,)), ("bd", (0,))):
        base = {k: v.detach().clone() for k, v in tp.items()}
        h = 1e-6
        bp = {k: v.clone() for k, v in base.items()}
        bm = {k: v.clone() for k, v in base.items()}
        bp[name][idx] += h
        bm[name][idx] -= h
        fd = ((mpnn.forward(A, bp)[0] * wts).sum() - (mpnn.forward(A, bm)[0] * wts).sum()) / (2 * h)
        assert abs(float(fd) - float(tp[name].grad[idx])) <= 1e-6 * (1 + abs(float(fd))), name
