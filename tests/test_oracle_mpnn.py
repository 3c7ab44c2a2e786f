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


def _rand_params(seed, scale=0.3):
    p = mpnn.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    p["v"] = rng.normal(0, scale, p["v"].shape).astype(np.float32)
    p["c"] = rng.normal(0, 0.1, p["c"].shape).astype(np.float32)
    for k in ("b0", "b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.1, p[k].shape).astype(np.float32)
    for k in ("W0", "W1", "W2", "W3", "Ua", "Ub"):        # BF16 weights, as the network stores them
        p[k] = torch.from_numpy(p[k]).to(torch.bfloat16).to(torch.float32).numpy()
    return p


def _rne_bf16_bits(x32: np.ndarray) -> np.ndarray:
    """BF16 rounding written on the float32 bit pattern: add 0x7FFF plus the lowest kept
    bit (ties to even) and clear the 16 dropped bits (finite inputs)."""
    b = x32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def test_bf16_round_is_round_to_nearest_even():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-30, 100), rng.normal(0, 1e30, 100)])
    # exact ties between two BF16 neighbours: 1 + (2k + 1) 2^-8 ties to the even neighbour
    ties = 1.0 + (2 * np.arange(20) + 1) * 2.0 ** -8
    x = np.concatenate([x, ties, -ties, [0.0, -0.0, 1.0, 2.0 ** -126]])
    got = mpnn.bf16_round(torch.from_numpy(x)).numpy()
    want = _rne_bf16_bits(x.astype(np.float32)).astype(np.float64)
    np.testing.assert_array_equal(got, want)
    # a float64 value is rounded to float32 first, as a kernel's float32 value would be
    y = np.float64(1.0 + 2.0 ** -8 + 2.0 ** -30)          # just above a tie; float32 rounds it onto it
    assert float(mpnn.bf16_round(torch.tensor([y]))[0]) == 1.0


def test_bf16_option_off_is_the_exact_network():
    A = synth.diffusion2d(5, 1.3, seed=6)
    p = _rand_params(8)
    tp = mpnn.params_to_torch(p, requires_grad=False)
    L0, pat0 = mpnn.forward(A, tp)
    L1, pat1 = mpnn.forward(A, tp, bf16=False, record={})
    assert torch.equal(L0, L1)
    np.testing.assert_array_equal(pat0[0], pat1[0])


def test_bf16_product_on_representable_operands_is_the_plain_product():
    """With X and the incoming gradient already BF16 values, rounding changes nothing:
    forward and both gradients equal float64 autograd of X W."""
    rng = np.random.default_rng(3)
    bf = lambda a: torch.from_numpy(a).to(torch.bfloat16).to(torch.float64)  # noqa: E731
    X = bf(rng.normal(size=(7, 5)).astype(np.float32)).requires_grad_(True)
    W = bf(rng.normal(size=(5, 4)).astype(np.float32)).requires_grad_(True)
    G = bf(rng.normal(size=(7, 4)).astype(np.float32))
    Y = mpnn._Bf16Product.apply(X, W)
    Y.backward(G)
    X2, W2 = X.detach().clone().requires_grad_(True), W.detach().clone().requires_grad_(True)
    (X2 @ W2).backward(G)
    assert torch.equal(Y.detach(), (X2 @ W2).detach())
    assert torch.equal(X.grad, X2.grad) and torch.equal(W.grad, W2.grad)


def test_bf16_network_within_the_bf16_error_bound():
    """Rounding the dense operands to BF16 (unit roundoff u = 2^-8) moves L by more than
    float64 rounding but within 2u of its normaliser elementwise; the parameter gradients
    move by well under a third in relative Frobenius norm (relu derivatives of
    pre-activations within a BF16 rounding of zero flip, so no elementwise bound holds
    for them).  A dropped term, a wrong sign or a transposed operand in the rounded
    reverse pass would move them by O(1)."""
    A = synth.diffusion2d(6, 1.0, seed=2)
    p = _rand_params(5)
    tp = mpnn.params_to_torch(p)
    tq = mpnn.params_to_torch(p)
    L, _ = mpnn.forward(A, tp)
    Lb, _ = mpnn.forward(A, tq, bf16=True)
    gL = np.random.default_rng(4).normal(size=L.numel())
    (L * torch.from_numpy(gL)).sum().backward()
    (Lb * torch.from_numpy(gL)).sum().backward()
    N_L, _ = mpnn.error_scale(A, p)
    u = 2.0 ** -8
    dl = np.abs(Lb.detach().numpy() - L.detach().numpy())
    assert dl.max() > 1e-3 * u * N_L.max()                # the option does round something
    assert np.all(dl <= 2 * u * N_L)
    for name in tp:
        a, b = tp[name].grad.numpy(), tq[name].grad.numpy()
        assert np.linalg.norm(b - a) <= 0.3 * max(np.linalg.norm(a), 1e-300), name


def test_bf16_network_on_representable_activations_is_exact():
    """On 2 A_N (diagonal 4, so d = 1/2 and e = -1/2 exactly; features -1, -1/2) with
    weights of a few dyadic values and zero biases, every activation that the option
    rounds is a BF16 value already, so L is the exact network's bit for bit: the option
    rounds nothing but those operands."""
    A = synth.poisson1d(12)
    A = synth.with_values(A, A.values * 2)
    rng = np.random.default_rng(6)
    p = mpnn.init_params(0)
    for name in ("W0", "W1", "W2", "W3", "Ua", "Ub"):
        shp = p[name].shape
        w = rng.choice([-1.0, -0.5, 0.5, 1.0], size=shp) * (rng.random(shp) < 1.5 / shp[0])
        p[name] = w.astype(np.float32)
    for name in ("b0", "b1", "b2", "b3"):
        p[name][:] = 0
    p["v"] = rng.normal(0, 0.3, p["v"].shape).astype(np.float32)
    p["c"] = rng.normal(0, 0.1, p["c"].shape).astype(np.float32)
    tp = mpnn.params_to_torch(p, requires_grad=False)
    rec = {}
    L, _ = mpnn.forward(A, tp, record=rec)
    for x in rec["X"] + [rec["h"]]:
        assert torch.equal(mpnn.bf16_round(x), x)          # the construction holds
    assert float(rec["h"].abs().max()) > 0
    Lb, _ = mpnn.forward(A, tp, bf16=True)
    assert torch.equal(L, Lb)


def test_error_scale_bounds_the_values_and_is_exact_on_nonnegative_data():
    """The normaliser is the absolute form of each output's last product, so it bounds the
    output (triangle inequality); with non-negative parameters, e (positive off-diagonal
    entries) and upstream gradient every relu passes its input, and the normaliser is
    2 L off the diagonal (|t| . |v| + |bo| = L / d_i, plus |Lhat|) and exactly each
    parameter gradient."""
    A = synth.diffusion2d(5, 1.0, seed=7)
    p = _rand_params(9)
    tp = mpnn.params_to_torch(p)
    L, _ = mpnn.forward(A, tp)
    gL = np.random.default_rng(2).normal(size=L.numel())
    (L * torch.from_numpy(gL)).sum().backward()
    N_L, N_g = mpnn.error_scale(A, p, gL)
    assert np.all(np.abs(L.detach().numpy()) <= N_L * (1 + 1e-12))
    for name in tp:
        assert np.all(np.abs(tp[name].grad.numpy()) <= N_g[name] * (1 + 1e-12) + 1e-300), name

    A = synth.diffusion2d(4, 1.0, seed=3)
    A = synth.with_values(A, np.abs(A.values))
    p = {k: np.abs(v) for k, v in _rand_params(2).items()}
    tp = mpnn.params_to_torch(p)
    L, (ri, ci) = mpnn.forward(A, tp)
    off = np.asarray(ri) != np.asarray(ci)
    gL = np.where(off, np.random.default_rng(1).random(L.numel()), 0.0)
    (L * torch.from_numpy(gL)).sum().backward()
    N_L, N_g = mpnn.error_scale(A, p, gL)
    np.testing.assert_allclose(N_L[off], 2 * L.detach().numpy()[off], rtol=1e-13)
    for name in tp:
        np.testing.assert_allclose(N_g[name], tp[name].grad.numpy(), rtol=1e-12, atol=1e-300, err_msg=name)
