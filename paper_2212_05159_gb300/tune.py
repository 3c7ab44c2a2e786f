"""Autotuner for the launch parameters of the row-wise products and of SDDMM.

For a given pattern and dense width k it times the candidate column blocks (columns
gathered per pass), rows-per-group settings, gather engines and column-part splits (passes
over ranges of the dense operand's rows) with CUDA events on the current stream and keeps
the fastest.  Results are cached per (pattern statistics, k, kind) in
memory and in ``_build/tune_cache.json``.  Timing only: the kernels computed with any
candidate give results within the same tolerance (a column block changes only which pass
adds which columns; a column-part split sums each output as a fixed sequence of per-part
partial sums).
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import abi
from .csr import CSR

_CACHE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")
_lock = threading.Lock()
_cache: dict | None = None


def _load():
    global _cache
    if _cache is None:
        try:
            with open(_CACHE_PATH) as fh:
                _cache = json.load(fh)
        except (OSError, ValueError):
            _cache = {}
    return _cache


def _save():
    try:
        os.makedirs(os.path.dirname(_CACHE_PATH), exist_ok=True)
        tmp = _CACHE_PATH + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(_cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, _CACHE_PATH)
    except OSError:
        pass


def _key(A: CSR, k: int, kind: str) -> str:
    return f"{kind}:m={A.m}:n={A.n}:nnz={A.nnz}:k={k}"


def _time(fn, reps=3):
    fn()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        fn()
    b.record(st)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _col_blocks(k: int):
    c = sorted({k} | {b for b in (128, 64, 32, 16, 8, 4) if b < k and (k % 4 != 0 or b % 4 == 0)},
               reverse=True)
    return c


PART_COUNTS = (1, 2, 3, 4)


def _part_counts(rows_in: int, k: int):
    """Split counts worth timing: more than one only when the gathered operand exceeds ~32 MB."""
    return [p for p in PART_COUNTS if p == 1 or rows_in * k * 4 > (32 << 20) * (p - 1)]


def tune_rows(A: CSR, k: int, transposed: bool = False, force: bool = False):
    """Best (col_block, rows_per_group, engine, n_parts) for spx_spmm (or spx_spmm_t when
    transposed)."""
    kind = "spmm_t2" if transposed else "spmm2"
    key = _key(A, k, kind)
    with _lock:
        c = _load()
        if key in c and not force:
            return tuple(c[key]["best"])
    dev = A.device
    rows_in, rows_out = (A.m, A.n) if transposed else (A.n, A.m)
    X = torch.randn(rows_in, k, device=dev)
    Y = torch.empty(rows_out, k, device=dev)
    base = A.t_plan() if transposed else A.plan()
    best, best_ms, table = None, float("inf"), {}
    engines = (0, 1) if k % 4 == 0 else (0,)
    cands = [(cb, rpg, eng, 1) for cb in _col_blocks(k) for rpg in (1, 2, 4) for eng in engines]
    if k % 4 == 0:                                      # lean short rows: one pass over all k
        cands += [(k, rpg, 2, 1) for rpg in (1, 2, 4)]
    cands += [(cb, rpg, 0, np_) for cb in _col_blocks(k) for rpg in (1, 2, 4)
              for np_ in _part_counts(rows_in, min(cb, k)) if np_ > 1]
    for cb, rpg, eng, np_ in cands:
        if True:
            parts = (A.t_parts(np_) if transposed else A.parts(np_)) if np_ > 1 else None
            plan = base.with_params(cb, rpg, eng, parts)
            if transposed:
                _, _, perm = A.transpose_pattern()
                s = A.t_struct()
                ws = abi.workspace(abi.spx_spmm_t_workspace_size(s, k, plan), dev)
                fn = lambda: abi.spx_spmm_t(s, perm, X, Y, 1.0, 0.0, plan, ws)  # noqa: E731
            else:
                s = A.struct()
                ws = abi.workspace(abi.spx_spmm_workspace_size(s, k, plan), dev)
                fn = lambda: abi.spx_spmm(s, X, Y, 1.0, 0.0, plan, ws)  # noqa: E731
            ms = _time(fn)
            del ws
            table[f"{cb},{rpg},{eng},{np_}"] = ms
            if ms < best_ms:
                best, best_ms = (cb, rpg, eng, np_), ms
    with _lock:
        _load()[key] = {"best": list(best), "ms": best_ms, "table": table}
        _save()
    return best


def tune_sddmm(A: CSR, k: int, force: bool = False):
    """Best (column block, "rows" | "chunks", n_parts) for spx_sddmm."""
    key = _key(A, k, "sddmm3")
    with _lock:
        c = _load()
        if key in c and not force:
            return tuple(c[key]["best"])
    dev = A.device
    G = torch.randn(A.m, k, device=dev)
    X = torch.randn(A.n, k, device=dev)
    out = torch.empty(A.nnz, device=dev)
    s = A.struct()
    best, best_ms, table = None, float("inf"), {}
    base = A.plan()
    for cb in _col_blocks(k):
        for mode, np_ in [("chunks", 1)] + [("rows", p) for p in _part_counts(A.n, min(cb, k))]:
            ws = abi.workspace(abi.spx_sddmm_workspace_size(s, k, cb), dev)
            plan = base.with_params(cb, 2, 0, A.parts(np_)) if mode == "rows" else None
            ms = _time(lambda: abi.spx_sddmm(s, G, X, out, 1.0, cb, ws, plan=plan))
            table[f"{cb},{mode},{np_}"] = ms
            if ms < best_ms:
                best, best_ms = (cb, mode, np_), ms
    with _lock:
        _load()[key] = {"best": best, "ms": best_ms, "table": table}
        _save()
    return best


def tuned_plan(A: CSR, k: int, transposed: bool = False):
    base = A.t_plan() if transposed else A.plan()
    best = tune_rows(A, k, transposed)
    cb, rpg = best[0], best[1]
    eng = best[2] if len(best) > 2 else 0
    np_ = best[3] if len(best) > 3 else 1
    parts = (A.t_parts(np_) if transposed else A.parts(np_)) if np_ > 1 else None
    return base.with_params(cb, rpg, eng, parts)


def tuned_sddmm_plan(A: CSR, k: int):
    """(column block, plan or None) for spx_sddmm: plan None selects the entry-chunk kernel."""
    cb, mode, np_ = tune_sddmm(A, k)
    return cb, (A.plan().with_params(cb, 2, 0, A.parts(np_)) if mode == "rows" else None)


MERGE_KS = (4, 8, 16, 32, 64, 128)


def merge_items(A: CSR, k: int, blocks_per_sm: int, waves: int, transposed: bool = False) -> int:
    """Merged items (row ends + entries) per segment so that the segments fill `waves` rounds
    of the lane groups that `blocks_per_sm` resident 256-thread blocks per SM hold."""
    sms = torch.cuda.get_device_properties(A.device).multi_processor_count
    groups = sms * blocks_per_sm * 256 // (k // 4)
    rows = A.n if transposed else A.m
    return max(8, -(-(rows + A.nnz) // (groups * waves)))


def tune_engine(A: CSR, k: int, kind: str, force: bool = False):
    """Row plan or merge path for one product, by device timing on this pattern and width.

    kind: "spmm" (Y = A X), "spmm_t" (A^T G with A^T's values already gathered) or "sddmm".
    Returns ("rows",) or ("merge", items, variant)."""
    if k not in MERGE_KS:
        return ("rows",)
    key = _key(A, k, "engine:" + kind)
    with _lock:
        c = _load()
        if key in c and not force:
            return tuple(c[key]["best"])
    dev = A.device
    transposed = kind == "spmm_t"
    rows_in, rows_out = (A.m, A.n) if transposed else (A.n, A.m)
    if transposed:
        t_ip, t_ix, perm = A.transpose_pattern()
        tv = torch.empty(max(A.nnz, 1), device=dev)[: A.nnz]
        abi.spx_gather_values(perm, A.values, tv)
        s = abi.csr_struct(A.n, A.m, t_ip, t_ix, tv)
    else:
        s = A.struct()
    table = {}
    if kind == "sddmm":
        G = torch.randn(A.m, k, device=dev)
        X = torch.randn(A.n, k, device=dev)
        out = torch.empty(A.nnz, device=dev)
        cb, plan = tuned_sddmm_plan(A, k)
        ws = abi.workspace(abi.spx_sddmm_workspace_size(s, k, cb), dev)
        table["rows"] = _time(lambda: abi.spx_sddmm(s, G, X, out, 1.0, cb, ws, plan=plan))
    else:
        X = torch.randn(rows_in, k, device=dev)
        Y = torch.empty(rows_out, k, device=dev)
        plan = tuned_plan(A, k, transposed)
        ws = abi.workspace(abi.spx_spmm_workspace_size(s, k, plan), dev)
        table["rows"] = _time(lambda: abi.spx_spmm(s, X, Y, 1.0, 0.0, plan, ws))
    best, best_ms = ("rows",), table["rows"]
    for bps in (4, 6):
        for waves in (1, 2, 4, 8):
            items = merge_items(A, k, bps, waves, transposed)
            mp = A.t_merge_plan(items) if transposed else A.merge_plan(items)
            if kind == "sddmm":
                fns = {v: (lambda v=v: abi.spx_sddmm_merge(s, G, X, out, mp, variant=v)) for v in (0, 1, 2)}
            else:
                mws = abi.workspace(abi.spx_spmm_merge_workspace_size(s, k, mp), dev)
                fns = {v: (lambda v=v, mws=mws: abi.spx_spmm_merge(s, X, Y, mp, mws, variant=v)) for v in (0, 1, 2)}
            for v, fn in fns.items():
                ms = _time(fn)
                table[f"merge:{items},{v}"] = ms
                if ms < best_ms:
                    best, best_ms = ("merge", items, v), ms
    with _lock:
        _load()[key] = {"best": list(best), "ms": best_ms, "table": table}
        _save()
    return best
