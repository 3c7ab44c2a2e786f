"""Learned preconditioner study: train on generated diffusion systems, then time PCG to a
relative residual of 1e-8 with Jacobi, the learned factor and IC(0) on held-out systems.

Workload (variable-coefficient 2D diffusion, 5-point, log-normal coefficients):
  training   systems with grid side ~ U{32..128} and sigma ~ U[0.5, 2], drawn fresh for
             every step (steps x batch systems in total), right-hand sides N(0,1);
  evaluation held-out 256 x 256 systems (sigma ~ U[0.5, 2], other seeds), N(0,1) rhs.
Timed per method with CUDA events on the solving stream, from preconditioner set-up
(network inference and the numeric SpGEMM forming M = L L^T; IC(0) numeric
factorisation) through convergence, plus the per-pattern analysis (SpGEMM symbolic,
IC(0) level schedule, transposes), host-timed once per pattern and added to the total.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import multiprocessing
import time

import numpy as np
import torch

from . import learned, solve
from .csr import CSR


def _gen(nsys, seed, lo, hi, sigma):
    import synth
    return synth.diffusion_system_batch(nsys, seed, lo, hi, sigma)


def train(net: learned.MPNN, steps: int, batch: int = 32, n_it: int = 64, gamma: float = 0.9,
          lr: float = 2e-3, seed: int = 1, time_budget_s: float | None = None, log=None,
          tensor_cores: bool = True, workers: int = 0, depth: int = 8, pattern: str = "A", epochs: int = 1):
    """Trains on `steps` fresh batches (steps * batch generated systems).  tensor_cores: the
    network's dense products forward and backward on tcgen05, the numerics of inference.
    Reports the wall time and the GPU time of the training steps (CUDA events).  pattern: the
    factor's pattern, tril(A) ("A") or tril(A + A^2) ("A2").  The batches are generated on the
    host `depth` steps ahead, by one background thread (workers = 0) or by `workers` spawned
    processes (the calling script must then guard its entry point with
    `if __name__ == "__main__"`, as spawned processes import it).  epochs: passes over the
    same `steps` batches (the training set stays steps * batch systems)."""
    tr = learned.Trainer(net, n_it=n_it, gamma=gamma, lr=lr, tensor_cores=tensor_cores, pattern=pattern)
    import synth
    losses, events = [], []
    t0 = time.perf_counter()
    st = torch.cuda.current_stream()
    step = -1
    pool = (cf.ProcessPoolExecutor(workers, mp_context=multiprocessing.get_context("spawn")) if workers > 0
            else cf.ThreadPoolExecutor(1))
    with pool as ex:
        args = lambda i: (batch, seed * 100003 + i % steps, 32, 128, (0.5, 2.0))  # noqa: E731
        total = steps * epochs
        futs = collections.deque(ex.submit(synth.diffusion_system_batch, *args(i))
                                 for i in range(min(depth, total)))
        for step in range(total):
            A, ptr, b = futs.popleft().result()
            if step + len(futs) + 1 < total:
                futs.append(ex.submit(synth.diffusion_system_batch, *args(step + len(futs) + 1)))
            dA = CSR.from_host(A)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            loss = tr.step(dA, torch.from_numpy(ptr).cuda(), len(ptr) - 1, torch.from_numpy(b).cuda())
            e1.record(st)
            events.append((e0, e1))
            if step % 20 == 0 or step == total - 1:
                losses.append((step, float(loss.mean())))
                if log:
                    log(f"step {step} loss {losses[-1][1]:.4f}")
            if time_budget_s is not None and time.perf_counter() - t0 > time_budget_s:
                for f in futs:
                    f.cancel()
                break
    torch.cuda.synchronize()
    gpu_ms = sum(a.elapsed_time(b) for a, b in events)
    return {"steps": step + 1, "systems": min(step + 1, steps) * batch, "epochs": epochs,
            "seconds": time.perf_counter() - t0,
            "gpu_seconds": gpu_ms * 1e-3, "generator_processes": workers,
            "loss_history": losses, "n_it": n_it, "gamma": gamma, "lr": lr, "batch": batch,
            "tensor_cores": tensor_cores, "pattern": pattern}


def _leading(A, ptr, b, k):
    """The first k systems of a block-diagonal batch (a leading principal block)."""
    import synth
    r = int(ptr[k])
    e = int(A.indptr[r])
    sub = synth.CSR(r, r, A.indptr[: r + 1], A.indices[:e], A.values[:e])
    return sub, ptr[: k + 1], b[:r]


def _timed(fn):
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    out = fn()
    b.record(st)
    torch.cuda.synchronize()
    return a.elapsed_time(b), out


def _pattern_key(A, ptr):
    return (A.m, A.nnz, hash(np.asarray(A.indptr).tobytes()), hash(np.asarray(A.indices).tobytes()),
            hash(np.asarray(ptr).tobytes()))


def evaluate(net: learned.MPNN, nsys: int = 128, per_batch: int = 64, side: int = 256, seed: int = 777,
             tol: float = 1e-8, methods=("jacobi", "learned", "ic0"), ic0_systems: int | None = None,
             learned_nets: dict | None = None):
    """Iterations and wall time to `tol` for each method over `nsys` held-out systems (IC(0)
    over the first `ic0_systems`).  learned_nets: method name -> (network, factor pattern[,
    "dia" | "M"]); by default "learned" is `net` on tril(A).  A learned factor is applied in
    diagonal form from shared memory when its pattern allows it ("dia", the default), else
    (or with "M") as the explicit M = L L^T formed by SpGEMM.

    Each method's time counts everything it needs: the per-batch set-up and solve (features,
    network inference on the tensor cores and the numeric SpGEMM forming M = L L^T; IC(0)'s
    numeric factorisation) timed with CUDA events, plus the per-pattern analysis (the
    factor's patterns and transposes, the SpGEMM symbolic phase; IC(0)'s pattern and level
    schedule), host-timed with synchronisation.  Batches of the same pattern (all held-out
    systems have one size) reuse the analysis, so it is paid once; it is reported apart as
    analysis_ms and included in total_ms and in the speed-ups."""
    nets = learned_nets if learned_nets is not None else {"learned": (net, "A")}
    ic0_systems = nsys if ic0_systems is None else ic0_systems
    res = {m: {"iters": [], "ms": 0.0, "setup_ms": 0.0, "converged": 0, "max_relres": 0.0, "systems": 0}
           for m in methods}
    analysis_ms = {m: 0.0 for m in methods}
    paths = {}                          # learned method -> "dia" (diagonal form in shared memory) or "M"
    cache = {}                          # (method, pattern) -> per-pattern objects

    def analysed(m, key, build):
        k = (m, key)
        if k not in cache:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cache[k] = build()
            torch.cuda.synchronize()
            analysis_ms[m] += (time.perf_counter() - t0) * 1e3
        return cache[k]

    done = 0
    bi = 0
    while done < nsys:
        k = min(per_batch, nsys - done)
        A, ptr, b = _gen(k, seed + bi, side, side, (0.5, 2.0))
        dA = CSR.from_host(A)
        batch = solve.SystemBatch(dA, ptr)
        bt = torch.from_numpy(b).cuda()
        maxit = 20 * side * side
        key = _pattern_key(A, ptr)
        for m in methods:
            if m == "ic0" and done >= ic0_systems:
                continue
            if m == "jacobi":
                ms, out = _timed(lambda: solve.cg(batch, bt, pc="jacobi", tol=tol, maxit=maxit,
                                                  values=dA.values))
                setup = 0.0
            elif m in nets:
                net_m, pattern = nets[m][:2]
                want_dia = len(nets[m]) < 3 or nets[m][2] == "dia"

                def build():
                    G = learned.Graph(dA, pattern)
                    F = solve.DiagonalFactor(batch, G.Lpat) if want_dia else None
                    if F is not None and F.supported:
                        return G, None, F
                    ones = torch.ones(G.Lpat.nnz, dtype=torch.float32, device=dA.device)
                    _, plan = learned.explicit_M(G, ones)        # the pattern of L L^T (symbolic)
                    return G, plan, None
                G, plan, F = analysed(m, key, build)
                G.rebind(dA)
                held = {}
                if F is not None:
                    F.rebind(batch)
                    paths[m] = "dia"

                    def prepare():
                        G.features(dA.values)
                        L2, _ = net_m.forward(G, tensor_cores=True, inference=True)   # tcgen05
                        F.fill(L2)

                    def run():
                        prepare()
                        return solve.cg(batch, bt, pc="dia", dia=F, tol=tol, maxit=maxit)
                    ms, out = _timed(run)
                    setup, _ = _timed(prepare)
                else:
                    paths[m] = "M"

                    def prepare():
                        G.features(dA.values)
                        L2, _ = net_m.forward(G, tensor_cores=True, inference=True)   # tcgen05
                        held["M"] = plan.C.with_values(plan.numeric(L2, _lt_values(G, L2)))

                    def run():
                        prepare()
                        return solve.cg(batch, bt, pc="M", M=held["M"], tol=tol, maxit=maxit)
                    ms, out = _timed(run)
                    setup, _ = _timed(prepare)
            else:
                kk = min(k, ic0_systems - done)              # IC(0) on the first ic0_systems only
                if kk < k:
                    As, ps, bs = _leading(A, ptr, b, kk)
                    dAs = CSR.from_host(As)
                    batch_ic, bt_ic = solve.SystemBatch(dAs, ps), torch.from_numpy(bs).cuda()
                    key_ic = _pattern_key(As, ps)
                else:
                    batch_ic, bt_ic, key_ic = batch, bt, key
                ic = analysed(m, key_ic, lambda: solve.IC0(batch_ic)).rebind(batch_ic)

                def run():
                    ic.factor()
                    return solve.cg(batch_ic, bt_ic, pc="ic0", ic0=ic, tol=tol, maxit=maxit)
                ms, out = _timed(run)
                setup, _ = _timed(lambda: ic.factor())
            _, it, st, rr = out
            r = res[m]
            r["iters"] += it.cpu().numpy().tolist()
            r["ms"] += ms
            r["setup_ms"] += setup
            r["converged"] += int((st.cpu().numpy() == 0).sum())
            r["max_relres"] = max(r["max_relres"], float(rr.cpu().numpy().max()))
            r["systems"] += int(it.numel())
        done += k
        bi += 1
    out = {"systems": nsys, "side": side, "tol": tol, "per_launch": per_batch,
           "timing": "total_ms = per-batch set-up and solve (CUDA events) + per-pattern analysis once "
                     "(host-timed); speed-ups use total_ms per system"}
    for m in methods:
        it = np.array(res[m]["iters"])
        ns = res[m]["systems"]
        total = res[m]["ms"] + analysis_ms[m]
        out[m] = {"systems": ns, "iters_median": float(np.median(it)), "iters_p90": float(np.percentile(it, 90)),
                  "iters_mean": float(it.mean()), "total_ms": total, "ms_per_system": total / ns,
                  "solve_and_setup_ms": res[m]["ms"], "numeric_setup_ms": res[m]["setup_ms"],
                  "numeric_setup": {"learned": "features, network inference, the factor's values (and M's by "
                                               "SpGEMM for the explicit M)",
                                    "ic0": "IC(0) numeric factorisation"}.get("ic0" if m == "ic0" else
                                                                              ("learned" if m in nets else ""), ""),
                  "analysis_ms": analysis_ms[m], "converged": res[m]["converged"],
                  "max_true_relres": res[m]["max_relres"]}
        if m in paths:
            out[m]["apply"] = {"dia": "M = L L^T by its diagonals in shared memory (spx_dia_square, spx_cg_batched_dia)",
                               "M": "explicit M = L L^T formed by SpGEMM, one gathered product"}[paths[m]]
    if "jacobi" in methods:
        for m in methods:
            if m != "jacobi":
                # per system, since IC(0) may cover a subset; the Jacobi figures of the same
                # systems are the first ones of its list
                ns = out[m]["systems"]
                j_it = np.array(res["jacobi"]["iters"][:ns])
                out[m]["speedup_vs_jacobi"] = out["jacobi"]["ms_per_system"] / out[m]["ms_per_system"]
                out[m]["iter_ratio_vs_jacobi"] = float(j_it.mean()) / out[m]["iters_mean"]
    return out


def _lt_values(G: learned.Graph, L: torch.Tensor):
    from . import abi
    out = torch.empty_like(L)
    abi.spx_gather_values(G.lt_perm, L, out)
    return out


def batch256_jacobi(graph_replay: bool = True, seed: int = 0, reps: int = 3):
    """The 256-system workload (sides U{32..256}, sigma 1): Jacobi PCG to 1e-8 in one persistent
    launch, captured once in a CUDA graph and replayed."""
    import synth
    A, ptr, sides, _ = synth.diffusion_batch(256, seed=seed, side_lo=32, side_hi=256, sigma=1.0)
    b = synth.normal(A.m, seed=seed + 1)
    dA = CSR.from_host(A)
    batch = solve.SystemBatch(dA, ptr)
    bt = torch.from_numpy(b).cuda()
    x = torch.empty(A.m, dtype=torch.float64, device="cuda")
    batch.dinv()
    maxit = 10 * 256 * 256
    solve.cg(batch, bt, pc="jacobi", x=x, maxit=maxit)           # warm-up
    torch.cuda.synchronize()
    if graph_replay:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                solve.cg(batch, bt, pc="jacobi", x=x, maxit=maxit)
        torch.cuda.current_stream().wait_stream(s)
        run = g.replay
    else:
        def run():
            solve.cg(batch, bt, pc="jacobi", x=x, maxit=maxit)
    times = []
    for _ in range(reps):
        ms, _ = _timed(run)
        times.append(ms)
    it = batch.iters.cpu().numpy()
    st = batch.status.cpu().numpy()
    rr = batch.relres.cpu().numpy()
    return {"systems": 256, "rows": int(A.m), "nnz": int(A.nnz), "ms": float(np.median(times)),
            "graph_replay": graph_replay, "iters_total": int(it.sum()), "iters_max": int(it.max()),
            "converged": int((st == 0).sum()), "max_true_relres": float(rr.max()),
            "row_iterations_per_s": float((np.diff(ptr) * it).sum() / (np.median(times) * 1e-3))}

