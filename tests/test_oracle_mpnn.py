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


def test_square_pattern_closed_forms():
    """A + A^2 structurally: pentadiagonal for the 1D model problem; for the 5-point grid
    of side s, interior row i holds i + {0, +-1, +-2, +-s, +-2s, +-(s-1), +-(s+1)} (13)."""
    N = 8
    rows = mpnn.square_pattern(synth.poisson1d(N))
    for i, cs in enumerate(rows):
        assert cs == [j for j in range(i - 2, i + 3) if 0 <= j < N]
    s = 7
    A = synth.diffusion2d(s, 1.0, seed=1)
    rows = mpnn.square_pattern(A)
    for y in range(2, s - 2):
        for x in range(2, s - 2):
            i = y * s + x
            offs = sorted({0, 1, -1, 2, -2, s, -s, 2 * s, -2 * s, s - 1, -(s - 1), s + 1, -(s + 1)})
            assert rows[i] == [i + o for o in offs]
    # brute force: the boolean product on a random small pattern
    rng = np.random.default_rng(0)
    D = (rng.random((9, 9)) < 0.25) | np.eye(9, dtype=bool)
    ip = np.concatenate([[0], np.cumsum(D.sum(1))])
    ix = np.nonzero(D)[1]
    B = synth.CSR(9, 9, ip, ix, np.ones(ix.size, np.float32))
    S = D | ((D.astype(int) @ D.astype(int)) > 0)
    assert mpnn.square_pattern(B) == [list(np.nonzero(S[i])[0]) for i in range(9)]


def test_square_pattern_factor_extends_the_tril_factor():
    """On tril(A + A^2) the entries of tril(A) take the same values as on tril(A); the others
    see e_ij = 0; at the Jacobi start every off-diagonal entry is 0."""
    A = synth.diffusion2d(6, 1.2, seed=4)
    p = mpnn.init_params(2)
    p["v"] = np.random.default_rng(1).normal(0, 0.4, p["v"].shape).astype(np.float32)
    p["bo"] = np.array([0.05], np.float32)
    tp = mpnn.params_to_torch(p, requires_grad=False)
    L1, (r1, c1) = mpnn.forward(A, tp)
    L2, (r2, c2) = mpnn.forward(A, tp, pattern="A2")
    assert len(r2) > len(r1)
    pos = {(int(r), int(c)): k for k, (r, c) in enumerate(zip(r2, c2))}
    k = np.array([pos[(int(r), int(c))] for r, c in zip(r1, c1)])
    np.testing.assert_allclose(L2.numpy()[k], L1.numpy(), rtol=1e-14, atol=0)
    _, _, g = mpnn.forward(A, tp, want_graph=True, pattern="A2")
    h, d = g["h"], None
    rows = np.repeat(np.arange(A.m), A.row_lengths())
    on = rows == A.indices
    d = np.zeros(A.m)
    d[rows[on]] = A.values[on]
    d = 1 / np.sqrt(d)
    extra = np.setdiff1d(np.arange(len(r2)), k)
    ri, ci = torch.from_numpy(np.asarray(r2)[extra]), torch.from_numpy(np.asarray(c2)[extra])
    t = torch.relu(h[ri] @ tp["Ua"] + h[ci] @ tp["Ub"] + tp["c"])
    want = d[ri.numpy()] * (t @ tp["v"] + tp["bo"]).numpy()
    np.testing.assert_allclose(L2.numpy()[extra], want, rtol=1e-13)
    p0 = mpnn.params_to_torch(mpnn.init_params(3), requires_grad=False)
    L0, (r0, c0) = mpnn.forward(A, p0, pattern="A2")
    assert np.all(L0.numpy()[np.asarray(r0) != np.asarray(c0)] == 0)
