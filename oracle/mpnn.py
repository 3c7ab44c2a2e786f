"""FP64 reference of the message-passing network that emits the learned factor L.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain PyTorch CPU float64 ops,
one statement per step of the architecture below; gradients come from torch autograd.

The network maps an SPD matrix A (CSR) to the values of a lower-triangular L on the
pattern of tril(A) -- or, as a richer factor, of tril(A + A^2) (the structural pattern of
the product, every entry any k reaches, plus A's own) -- used as the factored approximate
inverse M = L L^T of Section 4.3.
The architecture is chosen here (the paper gives none for this use; the closest is
the GNN of Section 4.5); parity of the trained weights themselves is unpinned.

  scale-free inputs   d_i = a_ii^(-1/2),  e_ij = d_i a_ij d_j  (e_ii = 1)
  node features       f_i = [1, sum_{j!=i} e_ij, min_{j!=i} e_ij, max_{j!=i} e_ij]
                      (0 for the last three when row i has no off-diagonal entry)
  encoder             h = relu(f W0 + b0)                          (4 -> 64)
  3 layers            g = E h  (sparse product on A's pattern with values e)
                      h = h + relu([h, g] Wl + bl)                 (128 -> 64)
  edge head, tril(S)  t_e = relu(h_i Ua + h_j Ub + e_ij u + c)     (e = (i, j), j <= i; S = A or A + A^2,
                                                                   e_ij = 0 where A has no entry)
                      o_e = t_e . v + (bd if i == j else bo)
  factor              Lhat_e = softplus(o_e) if i == j else o_e;   L_e = d_i Lhat_e
With v = 0, bo = 0 and softplus(bd) = 1 the factor is L = D^(-1/2): M = D^(-1) (Jacobi).

Two options of `forward` serve the parity tests of the GPU network:
  bf16=True      the operands of every dense product (the encoder, the three layers and
                 the two heads P = h Ua, Q = h Ub) are rounded to BF16 where a
                 tensor-core kernel rounds them: the activations in the forward product;
                 in the reverse pass the incoming gradient G of the product output, for
                 both dX = bf(G) W^T and dW = bf(X)^T bf(G).  Weights hold BF16 values
                 already; biases, the aggregation E h, the edge head and every sum stay
                 in float64.  A value is rounded as a float32 kernel value is: to float32
                 first, then to BF16 (round to nearest even).  With bf16=False the network
                 is unchanged (exact products).
`error_scale` gives the elementwise normaliser of the parity tests: for L and for every
parameter gradient, the last product that produces it evaluated on absolute values
(|X||W| + |b| forward, |X|^T |G| for a weight gradient), from this oracle's own float64
intermediates -- the |A||X| normaliser of a single sparse product, applied to the
network's final steps.
"""
from __future__ import annotations

import math

import numpy as np
import torch

H = 64
F_IN = 4
N_LAYERS = 3
BD_INIT = math.log(math.e - 1.0)            # softplus(BD_INIT) = 1


def param_shapes():
    s = {"W0": (F_IN, H), "b0": (H,)}
    for layer in range(N_LAYERS):
        s[f"W{layer + 1}"] = (2 * H, H)
        s[f"b{layer + 1}"] = (H,)
    s.update({"Ua": (H, H), "Ub": (H, H), "u": (H,), "c": (H,), "v": (H,), "bd": (1,), "bo": (1,)})
    return s


def init_params(seed: int, dtype=np.float32):
    """Seeded initial weights: Glorot-uniform matrices, zero biases, v = 0 (Jacobi start)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes().items():
        if len(shp) == 2:
            lim = math.sqrt(6.0 / (shp[0] + shp[1]))
            p[name] = rng.uniform(-lim, lim, shp).astype(dtype)
        else:
            p[name] = np.zeros(shp, dtype)
    p["u"] = rng.uniform(-1, 1, (H,)).astype(dtype)
    p["bd"] = np.array([BD_INIT], dtype)
    return p


def bf16_round(x: torch.Tensor) -> torch.Tensor:
    """x rounded as a kernel rounds a float32 value to BF16: to float32 (nearest), then
    to BF16 (nearest, ties to even); returned in float64."""
    return x.to(torch.float32).to(torch.bfloat16).to(torch.float64)


class _Bf16Product(torch.autograd.Function):
    """X W with BF16 operands: the forward rounds the activations X (W is BF16 already);
    the reverse rounds the incoming gradient G once and uses it in both products,
    dX = bf(G) W^T and dW = bf(X)^T bf(G), summed in float64."""

    @staticmethod
    def forward(ctx, X, W):
        Xr = bf16_round(X)
        ctx.save_for_backward(Xr, W)
        return Xr @ W

    @staticmethod
    def backward(ctx, G):
        Xr, W = ctx.saved_tensors
        Gr = bf16_round(G)
        return Gr @ W.t(), Xr.t() @ Gr


class _MagnitudeProduct(torch.autograd.Function):
    """X W forward; the reverse pass takes both products on absolute values,
    dX = |G| |W|^T and dW = S_X^T |G|, with S_X >= |X| the error scale of the forward
    operand (the first-order bound of rounding errors carried backwards, used by
    `error_scale`)."""

    @staticmethod
    def forward(ctx, X, W, S_X):
        ctx.save_for_backward(W, S_X)
        return X @ W

    @staticmethod
    def backward(ctx, G):
        W, S_X = ctx.saved_tensors
        Ga = G.abs()
        return Ga @ W.abs().t(), S_X.t() @ Ga, None


class _MagnitudeScale(torch.autograd.Function):
    """s[:, None] * X (s a fixed weight per row, X differentiable); reverse |s| |G|."""

    @staticmethod
    def forward(ctx, s, X):
        ctx.save_for_backward(s)
        return s[:, None] * X

    @staticmethod
    def backward(ctx, G):
        (s,) = ctx.saved_tensors
        return None, s.abs()[:, None] * G.abs()


def _product(bf16: bool, magnitude: bool = False):
    """X W as the chosen mode computes it; S (magnitude mode only) is X's error scale."""
    if magnitude:
        return lambda X, W, S=None: _MagnitudeProduct.apply(X, W, X.detach().abs() if S is None else S)
    if bf16:
        return lambda X, W, S=None: _Bf16Product.apply(X, W)
    return lambda X, W, S=None: X @ W


def _rows(indptr):
    ip = np.asarray(indptr, np.int64)
    return np.repeat(np.arange(len(ip) - 1), np.diff(ip))


def square_pattern(A):
    """Per-row sorted columns of the structural pattern of A + A^2: j is stored in row i when
    a_ij is stored or a_ik and a_kj are stored for some k (no cancellation)."""
    ip = np.asarray(A.indptr, np.int64)
    ix = np.asarray(A.indices, np.int64)
    rows = []
    for i in range(A.m):
        cols = set(ix[ip[i]:ip[i + 1]].tolist())
        for k in ix[ip[i]:ip[i + 1]]:
            cols.update(ix[ip[k]:ip[k + 1]].tolist())
        rows.append(sorted(cols))
    return rows


def forward(A, params: dict, want_graph=False, pattern: str = "A", bf16: bool = False,
            record: dict | None = None, magnitude: bool = False):
    """L values (float64 torch tensor on the pattern of tril(A), or of tril(A + A^2) with
    pattern="A2") and that pattern as (rows, cols).

    params: dict of torch float64 tensors (requires_grad as the caller wishes).
    bf16: see the module docstring.  record: if given, filled with the intermediates
    (features, layer inputs and pre-activations, heads, edge terms) for `error_scale`.
    magnitude: the same forward values, with a reverse pass that takes every product on
    absolute values (for `error_scale`); the forward operand of a weight gradient enters
    with its error scale: the absolute form of the operation that produced it, carried
    along the residual path (S_h + mask (|X||W| + |b|) for a layer output h + relu(X W + b),
    |E| |h| for an aggregate, mask (|h_i| |Ua| + |h_j| |Ub| + |e| |u| + |c|) for the
    edge activation)."""
    mm = _product(bf16, magnitude)
    mm_edge = _product(False, magnitude)          # the edge head is not a BF16 product
    scale = _MagnitudeScale.apply if magnitude else (lambda w, X: w[:, None] * X)
    act = torch.relu
    rec = record if record is not None else {}
    n = A.m
    rows = torch.from_numpy(_rows(A.indptr))
    cols = torch.from_numpy(np.asarray(A.indices, np.int64))
    a = torch.from_numpy(np.asarray(A.values, np.float64))
    diag_mask = rows == cols
    dvals = torch.zeros(n, dtype=torch.float64).index_put((rows[diag_mask],), a[diag_mask])
    d = dvals.rsqrt()
    e = d[rows] * a * d[cols]
    off = ~diag_mask
    # node features
    s = torch.zeros(n, dtype=torch.float64).index_add(0, rows[off], e[off])
    big = torch.full((n,), float("inf"), dtype=torch.float64)
    mn = big.scatter_reduce(0, rows[off], e[off], reduce="amin", include_self=True)
    mx = (-big).scatter_reduce(0, rows[off], e[off], reduce="amax", include_self=True)
    has = torch.zeros(n, dtype=torch.bool).index_fill(0, rows[off], True)
    mn = torch.where(has, mn, torch.zeros_like(mn))
    mx = torch.where(has, mx, torch.zeros_like(mx))
    f = torch.stack([torch.ones(n, dtype=torch.float64), s, mn, mx], dim=1)
    # encoder and message passing
    def absf(name):
        return params[name].detach().abs()

    with torch.no_grad():
        sf = torch.stack([torch.ones(n, dtype=torch.float64),
                          torch.zeros(n, dtype=torch.float64).index_add(0, rows[off], e[off].abs()),
                          mn.abs(), mx.abs()], dim=1)
    u = mm(f, params["W0"], sf) + params["b0"]
    rec["X"], rec["U"] = [f], [u]
    h = act(u)
    with torch.no_grad():
        sh = (u > 0) * (sf @ absf("W0") + absf("b0"))
    for layer in range(1, N_LAYERS + 1):
        g = torch.zeros(n, H, dtype=torch.float64).index_add(0, rows, scale(e, h[cols]))
        x = torch.cat([h, g], dim=1)
        with torch.no_grad():
            sg = torch.zeros(n, H, dtype=torch.float64).index_add(0, rows, e.abs()[:, None] * h.detach().abs()[cols])
            sx = torch.cat([sh, sg], dim=1)
        u = mm(x, params[f"W{layer}"], sx) + params[f"b{layer}"]
        rec["X"].append(x)
        rec["U"].append(u)
        with torch.no_grad():
            sh = sh + (u > 0) * (x.detach().abs() @ absf(f"W{layer}") + absf(f"b{layer}"))
        h = h + act(u)
    # edge head on tril(A) or tril(A + A^2)
    if pattern == "A":
        low = cols <= rows
        ri, ci, el = rows[low], cols[low], e[low]
    elif pattern == "A2":
        pos = {(int(r), int(c)): k for k, (r, c) in enumerate(zip(rows.tolist(), cols.tolist()))}
        pr, pc = [], []
        for i, cs in enumerate(square_pattern(A)):
            for j in cs:
                if j <= i:
                    pr.append(i)
                    pc.append(j)
        ri = torch.tensor(pr, dtype=torch.int64)
        ci = torch.tensor(pc, dtype=torch.int64)
        src = torch.tensor([pos.get((r, c), -1) for r, c in zip(pr, pc)], dtype=torch.int64)
        el = torch.where(src >= 0, e[src.clamp(min=0)], torch.zeros((), dtype=torch.float64))
    else:
        raise ValueError(f"unknown pattern {pattern!r}")
    P = mm(h, params["Ua"], sh)
    Q = mm(h, params["Ub"], sh)
    s_pre = P[ri] + Q[ci] + scale(el, params["u"].expand(len(el), H)) + params["c"]
    t = act(s_pre)
    with torch.no_grad():
        ha = h.detach().abs()
        st = (s_pre > 0) * ((ha @ absf("Ua"))[ri] + (ha @ absf("Ub"))[ci] + el.abs()[:, None] * absf("u") + absf("c"))
    isd = ri == ci
    o = mm_edge(t, params["v"][:, None], st)[:, 0] + torch.where(isd, params["bd"], params["bo"])
    lhat = torch.where(isd, torch.nn.functional.softplus(o), o)
    L = d[ri] * lhat
    rec.update({"h": h, "P": P, "Q": Q, "s": s_pre, "t": t, "el": el, "o": o, "lhat": lhat,
                "d": d, "ri": ri, "diag": isd})
    if want_graph:
        return L, (ri.numpy(), ci.numpy()), {"h": h, "e": e, "f": f}
    return L, (ri.numpy(), ci.numpy())


def params_to_torch(p: dict, requires_grad=True):
    return {k: torch.tensor(np.asarray(v, np.float64), requires_grad=requires_grad) for k, v in p.items()}


def error_scale(A, params: dict, gL=None, pattern: str = "A", bf16: bool = False):
    """Elementwise normaliser of the parity tests of the network, from float64 intermediates.

    Returns (N_L, N_grad).  N_L = d_i (|t_e| . |v| + |bias_e| + |Lhat_e|): the absolute
    form of the edge head's last product (plus the softplus value on the diagonal).  With
    an upstream gradient gL on L's entries, N_grad[name] is the parameter gradient of the
    reverse pass taken on absolute values from |gL| (`magnitude`): every product of the
    reverse pass as |G| |W|^T and |X|^T |G|, every fixed weight (e, d) by its absolute
    value, relu and softplus derivatives as they are.  It is the first-order bound of the
    rounding errors a float32 reverse pass accumulates, carried from |gL| to each
    parameter (the |A^T| |G| normaliser of a single transposed product, composed).
    params: dict of numpy arrays."""
    tp = params_to_torch(params, requires_grad=gL is not None)
    rec = {}
    L, _ = forward(A, tp, pattern=pattern, bf16=bf16, record=rec, magnitude=True)
    with torch.no_grad():
        bias = torch.where(rec["diag"], tp["bd"], tp["bo"]).abs()
        N_L = (rec["d"][rec["ri"]] * (rec["t"].abs() @ tp["v"].abs() + bias + rec["lhat"].abs())).numpy()
    if gL is None:
        return N_L, None
    (L * torch.from_numpy(np.abs(np.asarray(gL, np.float64)))).sum().backward()
    return N_L, {k: v.grad.numpy().copy() for k, v in tp.items()}
