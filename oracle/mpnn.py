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


def forward(A, params: dict, want_graph=False, pattern: str = "A"):
    """L values (float64 torch tensor on the pattern of tril(A), or of tril(A + A^2) with
    pattern="A2") and that pattern as (rows, cols).

    params: dict of torch float64 tensors (requires_grad as the caller wishes)."""
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
    h = torch.relu(f @ params["W0"] + params["b0"])
    for layer in range(1, N_LAYERS + 1):
        g = torch.zeros(n, H, dtype=torch.float64).index_add(0, rows, e[:, None] * h[cols])
        h = h + torch.relu(torch.cat([h, g], dim=1) @ params[f"W{layer}"] + params[f"b{layer}"])
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
    P = h @ params["Ua"]
    Q = h @ params["Ub"]
    t = torch.relu(P[ri] + Q[ci] + el[:, None] * params["u"] + params["c"])
    isd = ri == ci
    o = t @ params["v"] + torch.where(isd, params["bd"], params["bo"])
    lhat = torch.where(isd, torch.nn.functional.softplus(o), o)
    L = d[ri] * lhat
    if want_graph:
        return L, (ri.numpy(), ci.numpy()), {"h": h, "e": e, "f": f}
    return L, (ri.numpy(), ci.numpy())


def params_to_torch(p: dict, requires_grad=True):
    return {k: torch.tensor(np.asarray(v, np.float64), requires_grad=requires_grad) for k, v in p.items()}
