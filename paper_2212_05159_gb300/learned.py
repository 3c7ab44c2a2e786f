"""Learned preconditioner: a message-passing network emits L on tril(A); M = L L^T.

Section 4.3 learns a lower-triangular L with M = L L^T by minimising the weighted
residual history of N_it PCG iterations.  Here L's values come from a small
message-passing network applied to each system, so one set of weights serves every
system of a family; it is trained by back-propagating that loss through the library's
own kernels (spx_pcg_train for the unrolled PCG, then the network's reverse pass).

Network (hidden width 64, 3 message-passing layers, BF16 weights, FP32 accumulation):
  d_i = a_ii^-1/2, e_ij = d_i a_ij d_j,  f_i = [1, sum_{j!=i} e_ij, min, max]
  h = relu(f W0 + b0);  3 x { g = E h;  h = h + relu([h g] Wl + bl) }
  P = h Ua,  Q = h Ub;  for (i, j) in tril(A):
  o = relu(P_i + Q_j + e_ij u + c) . v + (bd | bo),  L_ij = d_i (softplus(o) | o)
At initialisation v = 0, bo = 0, softplus(bd) = 1, so L = D^-1/2 and M = D^-1 (Jacobi).
Every arithmetic step runs in a CUDA kernel of the library; this module allocates
buffers and sequences the calls.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import abi
from .csr import CSR
from .ops import SpAddPlan, SpGEMMPlan

H = 64
F_IN = 4
LAYERS = 3
BD_INIT = math.log(math.e - 1.0)

# name, shape, stored as BF16 for the dense kernels
PARAMS = [("W0", (F_IN, H), True), ("b0", (H,), False)]
for _l in range(1, LAYERS + 1):
    PARAMS += [(f"W{_l}", (2 * H, H), True), (f"b{_l}", (H,), False)]
PARAMS += [("Ua", (H, H), True), ("Ub", (H, H), True), ("u", (H,), False), ("c", (H,), False),
           ("v", (H,), False), ("bd", (1,), False), ("bo", (1,), False)]


def loss_weights(n_it: int, gamma: float) -> np.ndarray:
    w = gamma ** (n_it - np.arange(1, n_it + 1, dtype=np.float64))
    return (w / w.sum()).astype(np.float32)


def default_init(seed: int) -> dict:
    """Glorot-uniform matrices, zero biases, random u, v = 0, softplus(bd) = 1."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp, _ in PARAMS:
        if len(shp) == 2:
            lim = math.sqrt(6.0 / (shp[0] + shp[1]))
            p[name] = rng.uniform(-lim, lim, shp).astype(np.float32)
        else:
            p[name] = np.zeros(shp, np.float32)
    p["u"] = rng.uniform(-1, 1, (H,)).astype(np.float32)
    p["bd"] = np.array([BD_INIT], np.float32)
    return p


class Graph:
    """Per-batch inputs of the network: features, e on A and on the factor's pattern.

    pattern "A": L on tril(A); "A2": L on tril(A + A^2), the structural pattern of the
    product plus A's own (built with the library's SpGEMM symbolic phase and sparse add),
    with e_ij = 0 where A has no entry."""

    def __init__(self, A: CSR, pattern: str = "A"):
        dev = A.device
        self.A = A
        n = A.m
        self.n = n
        self.pattern = pattern
        self.d = torch.empty(n, dtype=torch.float32, device=dev)
        self.e = torch.empty(max(A.nnz, 1), dtype=torch.float32, device=dev)[: A.nnz]
        self.f = torch.empty(n, F_IN, dtype=torch.float32, device=dev)
        self.E = A.with_values(self.e)
        if pattern == "A":
            base, self._eplan = A, None
        elif pattern == "A2":
            sq = SpGEMMPlan(A, A).C
            self._zeros = torch.zeros(max(sq.nnz, 1), dtype=torch.float32, device=dev)[: sq.nnz]
            self._eplan = SpAddPlan(self.E, sq.with_values(self._zeros))
            base = self._eplan.C
            self._e_base = torch.empty(max(base.nnz, 1), dtype=torch.float32, device=dev)[: base.nnz]
        else:
            raise ValueError(f"unknown factor pattern {pattern!r}")
        l_ip, l_ix, self.l_src = abi.spx_tril_pattern(base.struct(), dev)
        self.Lpat = CSR(l_ip, l_ix, None, (n, n))
        self.e_low = torch.empty(l_ix.numel(), dtype=torch.float32, device=dev)
        self.lt_ip, self.lt_ix, self.lt_perm = self.Lpat.transpose_pattern()
        self.E.plan()
        self.features()

    def rebind(self, A: CSR):
        """Use this graph (patterns, transposes, plans) for another matrix of the same pattern
        (other values); call features() next."""
        if A.m != self.A.m or A.nnz != self.A.nnz:
            raise ValueError("Graph.rebind: a matrix of another pattern")
        self.A = A
        return self

    def features(self, values: torch.Tensor | None = None):
        """(Re)computes d, e and the node features for A's values (same pattern)."""
        abi.spx_mpnn_features(self.A.struct(values), self.d, self.e, self.f)
        if self._eplan is None:
            abi.spx_gather_values(self.l_src, self.e, self.e_low)
        else:
            self._eplan.numeric(1.0, 0.0, a_values=self.e, b_values=self._zeros, out=self._e_base)
            abi.spx_gather_values(self.l_src, self._e_base, self.e_low)
        return self

    def LT_struct(self, L_values: torch.Tensor, out: torch.Tensor):
        """A^T-pattern view of L with its values gathered into `out`."""
        abi.spx_gather_values(self.lt_perm, L_values, out)
        return abi.csr_struct(self.n, self.n, self.lt_ip, self.lt_ix, out)


class MPNN:
    """Weights (FP32 master + BF16 copy), Adam state, forward and reverse passes."""

    def __init__(self, device="cuda", seed: int = 0, params: dict | None = None):
        self.device = device
        self.offsets = {}
        o = 0
        for name, shp, _ in PARAMS:
            size = int(np.prod(shp))
            self.offsets[name] = (o, shp)
            o += size
        self.count = o
        self.flat = torch.zeros(o, dtype=torch.float32, device=device)
        self.flat16 = torch.zeros(o, dtype=torch.bfloat16, device=device)
        self.grad = torch.zeros(o, dtype=torch.float32, device=device)
        self.m = torch.zeros(o, dtype=torch.float32, device=device)
        self.v = torch.zeros(o, dtype=torch.float32, device=device)
        self.step_count = 0
        self.set_params(params if params is not None else default_init(seed))

    def view(self, buf, name):
        o, shp = self.offsets[name]
        return buf[o:o + int(np.prod(shp))].view(*shp)

    def set_params(self, params: dict):
        host = np.zeros(self.count, np.float32)
        for name, shp, _ in PARAMS:
            o, _ = self.offsets[name]
            host[o:o + int(np.prod(shp))] = np.asarray(params[name], np.float32).reshape(-1)
        self.flat.copy_(torch.from_numpy(host))
        abi.spx_to_bf16(self.flat, self.flat16)

    def get_params(self) -> dict:
        host = self.flat.cpu().numpy()
        out = {}
        for name, shp, _ in PARAMS:
            o, _ = self.offsets[name]
            out[name] = host[o:o + int(np.prod(shp))].reshape(shp).copy()
        return out

    def p(self, name):
        return self.view(self.flat, name)

    def p16(self, name):
        return self.view(self.flat16, name)

    def g(self, name):
        return self.view(self.grad, name)

    # ------------------------------------------------------------------ forward
    def forward(self, G: Graph, tensor_cores: bool = False, inference: bool = False):
        """L values on G.Lpat; returns (L, saved activations).

        tensor_cores: run the dense layers on tcgen05 (activations rounded to BF16); the
        default keeps FP32 activations (CUDA-core kernels).  inference (tensor cores only):
        the same L without what the reverse pass needs -- the residual layers keep no
        pre-activation and both heads come from one product (P | Q = h [Ua Ub]); returns
        (L, None)."""
        if inference and tensor_cores:
            return self._infer(G), None
        n, dev = G.n, self.device
        emp = lambda *s: torch.empty(*s, dtype=torch.float32, device=dev)  # noqa: E731
        dense = abi.spx_dense_forward_tc if tensor_cores else abi.spx_dense_forward
        h0 = emp(n, H)
        dense(n, G.f, F_IN, None, 0, self.p16("W0"), self.p("b0"), H, 1, None, h0)
        hs, gs, us = [h0], [], []
        Es = G.E.struct()
        plan = G.E.plan()
        for layer in range(1, LAYERS + 1):
            h = hs[-1]
            g = emp(n, H)
            abi.spx_spmm(Es, h, g, 1.0, 0.0, plan)
            u = emp(n, H)
            hn = emp(n, H)
            dense(n, h, H, g, H, self.p16(f"W{layer}"), self.p(f"b{layer}"), H, 2, h, hn, u)
            hs.append(hn)
            gs.append(g)
            us.append(u)
        hL = hs[-1]
        P, Q = emp(n, H), emp(n, H)
        dense(n, hL, H, None, 0, self.p16("Ua"), None, H, 0, None, P)
        dense(n, hL, H, None, 0, self.p16("Ub"), None, H, 0, None, Q)
        L = emp(G.Lpat.nnz)
        abi.spx_edge_forward(G.Lpat.struct(), G.e_low, G.d, P, Q, self.p("u"), self.p("c"), self.p("v"),
                             self.p("bd"), self.p("bo"), L)
        return L, {"hs": hs, "gs": gs, "us": us, "P": P, "Q": Q}

    def _infer(self, G: Graph):
        """forward(tensor_cores=True) without the saved activations (same arithmetic)."""
        n, dev = G.n, self.device
        emp = lambda *s: torch.empty(*s, dtype=torch.float32, device=dev)  # noqa: E731
        h = emp(n, H)
        abi.spx_dense_forward_tc(n, G.f, F_IN, None, 0, self.p16("W0"), self.p("b0"), H, 1, None, h)
        Es = G.E.struct()
        plan = G.E.plan()
        g = emp(n, H)
        hn = emp(n, H)
        for layer in range(1, LAYERS + 1):
            abi.spx_spmm(Es, h, g, 1.0, 0.0, plan)
            abi.spx_dense_forward_tc(n, h, H, g, H, self.p16(f"W{layer}"), self.p(f"b{layer}"), H, 3, h, hn)
            h, hn = hn, h
        heads = torch.cat((self.p16("Ua"), self.p16("Ub")), dim=1).contiguous()     # [Ua Ub]: 64 x 128
        P, Q = emp(n, H), emp(n, H)
        abi.spx_dense_forward_tc(n, h, H, None, 0, heads, None, 2 * H, 4, None, P, Q)
        L = emp(G.Lpat.nnz)
        abi.spx_edge_forward(G.Lpat.struct(), G.e_low, G.d, P, Q, self.p("u"), self.p("c"), self.p("v"),
                             self.p("bd"), self.p("bo"), L)
        return L

    # ------------------------------------------------------------------ reverse
    def backward(self, G: Graph, saved, gL: torch.Tensor, tensor_cores: bool = False):
        """Accumulates d loss / d params into self.grad (overwritten) from gL on G.Lpat.

        tensor_cores: the data gradients G W^T and the weight gradients X^T G of the dense
        layers run on tcgen05 (operands rounded to BF16, FP32 accumulation; bias gradients
        summed in FP32)."""
        n, dev = G.n, self.device
        bdata = abi.spx_dense_backward_data_tc if tensor_cores else abi.spx_dense_backward_data
        emp = lambda *s: torch.empty(*s, dtype=torch.float32, device=dev)  # noqa: E731
        hs, gs, us, P, Q = saved["hs"], saved["gs"], saved["us"], saved["P"], saved["Q"]
        gP, gQ = emp(n, H), emp(n, H)
        gpar = emp(3 * H + 2)
        ews = abi.workspace(abi._size("spx_edge_backward_workspace_size", int(n)), dev)
        abi.spx_edge_backward(G.Lpat.struct(), G.lt_ip, G.lt_ix, G.lt_perm, G.e_low, G.d, P, Q, self.p("u"),
                              self.p("c"), self.p("v"), self.p("bd"), self.p("bo"), gL, gP, gQ, gpar, ews)
        self.g("v").copy_(gpar[0:H])
        self.g("c").copy_(gpar[H:2 * H])
        self.g("u").copy_(gpar[2 * H:3 * H])
        self.g("bd").copy_(gpar[3 * H:3 * H + 1])
        self.g("bo").copy_(gpar[3 * H + 1:3 * H + 2])

        def wgrad(X1, K1, X2, K2, Gm, N, dW, db):
            sfx = "_tc" if tensor_cores else ""
            ws = abi.workspace(abi._size(f"spx_dense_backward_weight{sfx}_workspace_size", int(n), int(K1 + K2),
                                         int(N)), dev)
            getattr(abi, f"spx_dense_backward_weight{sfx}")(n, X1, K1, X2, K2, Gm, N, dW, db, ws)

        hL = hs[-1]
        wgrad(hL, H, None, 0, gP, H, self.g("Ua"), None)
        wgrad(hL, H, None, 0, gQ, H, self.g("Ub"), None)
        gh = emp(n, H)
        bdata(n, gP, H, self.p16("Ua"), H, 0, gh, None, 0)
        bdata(n, gQ, H, self.p16("Ub"), H, 0, gh, None, 1)
        Es = G.E.struct()
        plan = G.E.plan()
        for layer in range(LAYERS, 0, -1):
            h_in, g, u = hs[layer - 1], gs[layer - 1], us[layer - 1]
            gu = emp(n, H)
            abi.spx_relu_backward(gh, u, gu)
            wgrad(h_in, H, g, H, gu, H, self.g(f"W{layer}"), self.g(f"b{layer}"))
            gg = torch.zeros(n, H, dtype=torch.float32, device=dev)
            # h_out = h_in + relu(u): gh_in = gh_out + (gu W^T)[:, :H]; gg = (gu W^T)[:, H:]
            bdata(n, gu, H, self.p16(f"W{layer}"), H, H, gh, gg, 1)
            # g = E h_in  ->  gh_in += E^T gg  (E is symmetric for symmetric A)
            abi.spx_spmm(Es, gg, gh, 1.0, 1.0, plan)
        gu0 = emp(n, H)
        abi.spx_relu_backward(gh, hs[0], gu0)
        wgrad(G.f, F_IN, None, 0, gu0, H, self.g("W0"), self.g("b0"))
        return self.grad

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        abi.spx_adam_step(self.flat, self.grad, self.m, self.v, self.step_count, lr, beta1, beta2, eps,
                          self.flat16)


class Trainer:
    """Unrolled-PCG training of the network on block-diagonal batches of systems."""

    def __init__(self, net: MPNN, n_it: int = 4, gamma: float = 0.6, lr: float = 1e-3, tensor_cores: bool = False,
                 pattern: str = "A", checkpoint=0, max_workspace_bytes: int | None = None):
        """checkpoint: 0 keeps every unrolled iterate for the reverse pass; s (1..n_it-1) keeps
        every s-th state and recomputes the rest; "auto" keeps everything while the workspace
        fits max_workspace_bytes (default: half the free device memory) and otherwise takes
        the largest interval that fits (the least recomputation)."""
        self.net, self.n_it, self.gamma, self.lr = net, n_it, gamma, lr
        self.tensor_cores = tensor_cores
        self.pattern = pattern
        self.checkpoint = checkpoint
        self.max_workspace_bytes = max_workspace_bytes
        self.wts = torch.from_numpy(loss_weights(n_it, gamma)).to(net.device)

    def interval(self, n: int) -> int:
        """The checkpoint interval for an n-row batch (0: keep every iterate)."""
        if self.checkpoint != "auto":
            return int(self.checkpoint)
        size = lambda s: abi._size("spx_pcg_train_workspace_size", int(n), int(self.n_it), int(s))  # noqa: E731
        budget = self.max_workspace_bytes
        if budget is None:
            budget = torch.cuda.mem_get_info()[0] // 2
        if size(0) <= budget:
            return 0
        fits = [s for s in range(self.n_it - 1, 0, -1) if size(s) <= budget]
        return fits[0] if fits else min(range(1, self.n_it), key=size)

    def loss_and_grad(self, A: CSR, sys_ptr: torch.Tensor, nsys: int, b: torch.Tensor, G: Graph | None = None):
        """Mean loss over the systems and the L gradient (the network is not updated)."""
        G = G or Graph(A, self.pattern)
        L, saved = self.net.forward(G, tensor_cores=self.tensor_cores)
        lt_vals = torch.empty_like(L)
        LT = G.LT_struct(L, lt_vals)
        Ls = abi.csr_struct(G.n, G.n, G.Lpat.indptr, G.Lpat.indices, L)
        s = self.interval(G.n)
        ws = abi.workspace(abi._size("spx_pcg_train_workspace_size", int(G.n), int(self.n_it), s), A.device)
        loss = torch.empty(nsys, dtype=torch.float32, device=A.device)
        gL = torch.empty_like(L)
        abi.spx_pcg_train(A.struct(), sys_ptr, nsys, Ls, LT, b, self.n_it, self.wts, loss, gL, ws, ckpt_interval=s)
        return loss, gL, L, G, saved

    def step(self, A: CSR, sys_ptr: torch.Tensor, nsys: int, b: torch.Tensor):
        loss, gL, L, G, saved = self.loss_and_grad(A, sys_ptr, nsys, b)
        self.net.backward(G, saved, gL, tensor_cores=self.tensor_cores)
        self.net.adam(self.lr)
        return loss


def explicit_M(G: Graph, L_values: torch.Tensor):
    """M = L L^T formed once with the library's SpGEMM (one sparse product per PCG step)."""
    dev = L_values.device
    Lc = G.Lpat.with_values(L_values)
    lt_vals = torch.empty_like(L_values)
    abi.spx_gather_values(G.lt_perm, L_values, lt_vals)
    LTc = CSR(G.lt_ip, G.lt_ix, lt_vals, (G.n, G.n))
    plan = SpGEMMPlan(Lc, LTc)
    return plan.C.with_values(plan.numeric()), plan
