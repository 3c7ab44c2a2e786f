"""ctypes binding of ``libspx.so`` (declared in ``include/spx.h``).

Argument marshalling only: every function here has the name of the C entry point it
calls, takes torch CUDA tensors (or host numpy arrays where the C side wants host
memory), passes their raw pointers and the current CUDA stream, and raises
:class:`SpxError` on a non-zero status.  No arithmetic of the method happens here.

The library is built in-tree (``paper_2212_05159_gb300/_build/libspx.so``) by
``paper_2212_05159_gb300.build``; if it is missing and cannot be built, importing a
compute function raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspx.so")
_lock = threading.Lock()
_lib = None

STATUS = {
    0: "SPX_OK", 1: "SPX_INVALID_ARG", 2: "SPX_BAD_PATTERN", 3: "SPX_UNSORTED",
    4: "SPX_OOM_WORKSPACE", 5: "SPX_MAXITER", 6: "SPX_BREAKDOWN", 7: "SPX_NONFINITE",
    8: "SPX_DEVICE_TIMEOUT", 9: "SPX_CUDA_ERROR", 10: "SPX_NOT_SUPPORTED",
}


class SpxError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


class spx_csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("indptr", ctypes.c_void_p), ("indices", ctypes.c_void_p),
                ("values", ctypes.c_void_p)]


class spx_rowplan(ctypes.Structure):
    _fields_ = [("long_rows", ctypes.c_void_p), ("n_long", ctypes.c_int32),
                ("threshold", ctypes.c_int32), ("col_block", ctypes.c_int32),
                ("rows_per_group", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("medium_rows", ctypes.c_void_p), ("n_medium", ctypes.c_int32),
                ("medium_threshold", ctypes.c_int32), ("part_ptr", ctypes.c_void_p),
                ("n_parts", ctypes.c_int32), ("short_rows", ctypes.c_void_p), ("n_short", ctypes.c_int32)]

    def with_params(self, col_block=0, rows_per_group=0, engine=0, parts=None, short_order=True):
        """A copy of this plan (same row lists) with other launch parameters; `parts` is a
        (part_ptr tensor, n_parts) pair from spx_rowplan_build_parts, None for one pass;
        short_order=False walks the short rows in natural order instead of the plan's."""
        pp, np_ = (parts[0].data_ptr(), int(parts[1])) if parts is not None and parts[1] > 1 else (None, 0)
        sr, ns = (self.short_rows, self.n_short) if short_order else (None, 0)
        return spx_rowplan(self.long_rows, self.n_long, self.threshold, col_block, rows_per_group, engine,
                           self.medium_rows, self.n_medium, self.medium_threshold, pp, np_, sr, ns)


class spx_mergeplan(ctypes.Structure):
    _fields_ = [("seg_row", ctypes.c_void_p), ("n_segments", ctypes.c_int32), ("items", ctypes.c_int64)]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_F = ctypes.c_float
_D = ctypes.c_double
_SZ = ctypes.c_size_t
_CSRP = ctypes.POINTER(spx_csr)
_PLANP = ctypes.POINTER(spx_rowplan)

# name -> argtypes (every entry point returns spx_status, an int)
SIGNATURES = {
    "spx_csr_validate": [_CSRP, _P, _SZ, _P],
    "spx_check_device": [_P],
    "spx_rowplan_workspace_size": [_I32, ctypes.POINTER(_SZ)],
    "spx_rowplan_build": [_CSRP, _I32, _P, ctypes.POINTER(_I32), _P, _SZ, _P],
    "spx_rowplan_build_short": [_CSRP, _I32, _P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), _P, _SZ, _P],
    "spx_rowplan_build_medium": [_CSRP, _I32, _I32, _P, ctypes.POINTER(_I32), _P, _SZ, _P],
    "spx_rowplan_build_parts": [_CSRP, _I32, _P, _P],
    "spx_spmm_workspace_size": [_CSRP, _I32, _PLANP, ctypes.POINTER(_SZ)],
    "spx_spmm": [_CSRP, _P, _I64, _I32, _P, _I64, _F, _F, _PLANP, _P, _SZ, _P],
    "spx_sddmm_workspace_size": [_CSRP, _I32, _I32, ctypes.POINTER(_SZ)],
    "spx_sddmm": [_CSRP, _P, _I64, _P, _I64, _I32, _F, _P, _I32, _PLANP, _P, _SZ, _P],
    "spx_masked_outer": [_CSRP, _P, _P, _F, _P, _P],
    "spx_transpose_workspace_size": [_I32, _I32, _I64, ctypes.POINTER(_SZ)],
    "spx_csr_transpose": [_CSRP, _P, _P, _P, _P, _SZ, _P],
    "spx_spmm_t_workspace_size": [_CSRP, _I32, _PLANP, ctypes.POINTER(_SZ)],
    "spx_spmm_t": [_CSRP, _P, _P, _I64, _I32, _P, _I64, _F, _F, _PLANP, _P, _SZ, _P],
    "spx_spmm_t_sddmm": [_CSRP, _P, _P, _P, _I64, _P, _I64, _I32, _P, _I64, _F, _F, _P, _F, _PLANP, _I32, _P],
    "spx_spmm_t_noalloc": [_CSRP, _P, _P, _I64, _I32, _P, _I64, _F, _F, _PLANP, _P],
    "spx_spgemm_workspace_size": [_I32, ctypes.POINTER(_SZ)],
    "spx_spgemm_analyse": [_CSRP, _CSRP, ctypes.POINTER(_I64), _P, _SZ, _P],
    "spx_spgemm_symbolic": [_CSRP, _CSRP, _I64, _P, ctypes.POINTER(_I64), _P, _SZ, _P, _SZ, _P],
    "spx_spgemm_fill": [_CSRP, _P, _P, _P, _SZ, _P, _P],
    "spx_spgemm_numeric": [_CSRP, _CSRP, _CSRP, _P, _P, _SZ, _P],
    "spx_spgemm_backward": [_CSRP, _CSRP, _CSRP, _P, _P, _P, _P, _P, _P, _P],
    "spx_gather_values": [_I64, _P, _P, _P, _P],
    "spx_merge_plan_segments": [_CSRP, _I64, ctypes.POINTER(_I32)],
    "spx_merge_plan_build": [_CSRP, _I64, _P, _I32, _P],
    "spx_spmm_merge_workspace_size": [_CSRP, _I32, ctypes.POINTER(spx_mergeplan), ctypes.POINTER(_SZ)],
    "spx_spmm_merge": [_CSRP, _P, _P, _I64, _I32, _P, _I64, _F, _F, ctypes.POINTER(spx_mergeplan), _I32, _P, _SZ,
                       _P],
    "spx_sddmm_merge": [_CSRP, _P, _I64, _P, _I64, _I32, _F, _P, ctypes.POINTER(spx_mergeplan), _I32, _P],
    "spx_dia_analyse": [_CSRP, _P, _I32, _P, _P, ctypes.POINTER(_I32), _P],
    "spx_dia_fill": [_CSRP, _P, _I32, _P, _P, _P, _P],
    "spx_dia_square": [_P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P],
    "spx_cg_batched_dia": [_CSRP, _P, _I32, _P, _P, _P, _P, _P, _P, _D, _I32, _D, _P, _P, _P, _P, _SZ, _P],
    "spx_gather_probe": [_P, _I64, _I32, _P, _I64, _I32, _I32, _I32, _P, _I64, _P],
    "spx_csr_diagonal": [_CSRP, _P, _P, _P],
    "spx_diagonal_backward": [_I32, _P, _P, _P, _P],
    "spx_cg_workspace_size": [_I32, ctypes.POINTER(_SZ)],
    "spx_cg_batched": [_CSRP, _P, _I32, _P, _P, _P, _I32, _P, _CSRP, _CSRP, ctypes.POINTER(_P), _D, _I32, _D,
                       _P, _P, _P, _P, _SZ, _P],
    "spx_ic0_workspace_size": [_I32, _I32, ctypes.POINTER(_SZ)],
    "spx_ic0_analyse": [_CSRP, _P, _I32, _P, _P, _P, _P, _SZ, _P],
    "spx_ic0_factor": [_CSRP, _P, _P, _I32, _P, _P, _P, _P, _P, _P],
    "spx_diag_inverse": [_CSRP, _P, _P],
    "spx_cg_set_launch": [_I32, _I32, _I32],
    "spx_cg_set_vector_residency": [_I32],
    "spx_masked_outer_f64": [_CSRP, _P, _P, _D, _P, _P],
    "spx_pcg_train_workspace_size": [_I32, _I32, _I32, ctypes.POINTER(_SZ)],
    "spx_pcg_train": [_CSRP, _P, _I32, _CSRP, _CSRP, _P, _I32, _I32, _P, _P, _P, _P, _SZ, _P],
    "spx_mpnn_features": [_CSRP, _P, _P, _P, _P],
    "spx_dense_forward": [_I64, _P, _I32, _P, _I32, _P, _P, _I32, _I32, _P, _P, _P, _P],
    "spx_dense_forward_tc": [_I64, _P, _I32, _P, _I32, _P, _P, _I32, _I32, _P, _P, _P, _P],
    "spx_dense_backward_data": [_I64, _P, _I32, _P, _I32, _I32, _P, _P, _I32, _P],
    "spx_dense_backward_weight_workspace_size": [_I64, _I32, _I32, ctypes.POINTER(_SZ)],
    "spx_dense_backward_weight": [_I64, _P, _I32, _P, _I32, _P, _I32, _P, _P, _P, _SZ, _P],
    "spx_relu_backward": [_I64, _P, _P, _P, _P],
    "spx_tril_workspace_size": [_I32, ctypes.POINTER(_SZ)],
    "spx_tril_pattern": [_CSRP, _P, _P, _P, ctypes.POINTER(_I64), _P, _SZ, _P],
    "spx_edge_forward": [_CSRP, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "spx_edge_backward_workspace_size": [_I32, ctypes.POINTER(_SZ)],
    "spx_edge_backward": [_CSRP, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                          _SZ, _P],
    "spx_adam_step": [_I64, _P, _P, _P, _P, _I32, _F, _F, _F, _F, _P, _P],
    "spx_to_bf16": [_I64, _P, _P, _P],
    "spx_spai_residual": [_CSRP, _F, _P, _P, _P],
    "spx_dense_backward_data_tc": [_I64, _P, _I32, _P, _I32, _I32, _P, _P, _I32, _P],
    "spx_tc_set_pipeline": [_I32],
    "spx_dense_backward_weight_tc_workspace_size": [_I64, _I32, _I32, ctypes.POINTER(_SZ)],
    "spx_dense_backward_weight_tc": [_I64, _P, _I32, _P, _I32, _P, _I32, _P, _P, _P, _SZ, _P],
    "spx_precond_apply": [_I32, _I64, _P, _P, _P, _CSRP, _CSRP, _I32, _P, _P, _P],
    "spx_cg_adjoint": [_CSRP, _P, _I32, _P, _P, _P, _P, _P, _I32, _P, _CSRP, _CSRP, _P, _D, _I32, _D, _P, _P, _P,
                       _P, _SZ, _P],
    "spx_spmm_autotune": [_CSRP, _P, _I64, _I32, _P, _I64, _PLANP, ctypes.POINTER(_F), _P],
    "spx_sync_status": [_P, _I32, _P, _P],
    "spx_sptrsv": [_CSRP, _I32, _I32, _P, _P, _P, _P, _P, _P, _P],
    "spx_spadd_workspace_size": [_I32, ctypes.POINTER(_SZ)],
    "spx_spadd_symbolic": [_CSRP, _CSRP, _P, ctypes.POINTER(_I64), _P, _SZ, _P],
    "spx_spadd_fill": [_CSRP, _CSRP, _P, _P, _P, _P, _P, _P, _P],
    "spx_spadd_numeric": [_I64, _F, _P, _P, _F, _P, _P, _P, _P],
    "spx_spadd_backward": [_I64, _I64, _F, _F, _P, _P, _P, _P, _P, _P],
    "spx_dot_workspace_size": [_I64, ctypes.POINTER(_SZ)],
    "spx_dot": [_I64, _P, _P, _P, _P, _SZ, _P],
    "spx_spai_update": [_I64, _P, _P, _P, _P, _P],
}


def lib():
    """The loaded library (built first if needed).  Raises if it cannot be had."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                from .build import build
                build()
            L = ctypes.CDLL(LIB_PATH)
            L.spx_last_error.restype = ctypes.c_char_p
            L.spx_status_name.restype = ctypes.c_char_p
            L.spx_version.restype = ctypes.c_int32
            for name, args in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = ctypes.c_int
                f.argtypes = args
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != 0:
        msg = lib().spx_last_error().decode(errors="replace")
        raise SpxError(status, where, msg)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def ptr(t):
    """Device pointer of a tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def csr_struct(m, n, indptr, indices, values=None) -> spx_csr:
    for t, dt in ((indptr, torch.int32), (indices, torch.int32)):
        if t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
            raise ValueError("indptr/indices must be contiguous int32 CUDA tensors")
    if values is not None and (values.dtype != torch.float32 or not values.is_contiguous()):
        raise ValueError("values must be a contiguous float32 CUDA tensor")
    return spx_csr(int(m), int(n), int(indices.numel()), indptr.data_ptr(), indices.data_ptr(),
                   values.data_ptr() if values is not None else None)


def workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


def _dense(t, name):
    if t.dtype != torch.float32 or t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be a float32 2-D tensor with unit column stride")
    return ctypes.c_void_p(t.data_ptr()), t.stride(0)


# ------------------------------------------------------------------ entry points
def spx_version() -> int:
    return int(lib().spx_version())


def spx_check_device() -> None:
    """Raises SpxError(SPX_DEVICE_TIMEOUT) if a bounded device-side wait ran out."""
    _check(lib().spx_check_device(_stream()), "spx_check_device")


def spx_csr_validate(A: spx_csr, device) -> None:
    ws = workspace(16, device)
    _check(lib().spx_csr_validate(ctypes.byref(A), ptr(ws), ws.numel(), _stream()),
           "spx_csr_validate")


def spx_rowplan_build(A: spx_csr, threshold: int, device, medium_threshold: int = 0, short_order: bool = True):
    """Returns (row-list tensors, spx_rowplan); medium_threshold > 0 adds the medium bin;
    short_order adds the length-grouped order of the short rows."""
    sz = _SZ(0)
    _check(lib().spx_rowplan_workspace_size(A.m, ctypes.byref(sz)), "spx_rowplan_workspace_size")
    ws = workspace(sz.value, device)
    rows = torch.empty(max(A.m, 1), dtype=torch.int32, device=device)
    n_long = _I32(0)
    _check(lib().spx_rowplan_build(ctypes.byref(A), int(threshold), ptr(rows), ctypes.byref(n_long),
                                   ptr(ws), ws.numel(), _stream()), "spx_rowplan_build")
    rows = rows[: n_long.value].clone() if n_long.value > 0 else rows[:0]
    med = rows[:0]
    n_med = _I32(0)
    if medium_threshold > 0 and A.m > 0:
        med = torch.empty(max(A.m, 1), dtype=torch.int32, device=device)
        _check(lib().spx_rowplan_build_medium(ctypes.byref(A), int(medium_threshold), int(threshold), ptr(med),
                                              ctypes.byref(n_med), ptr(ws), ws.numel(), _stream()),
               "spx_rowplan_build_medium")
        med = med[: n_med.value].clone() if n_med.value > 0 else med[:0]
    short = rows[:0]
    n_short, n_groups = _I32(0), _I32(0)
    if short_order and A.m > 0:
        short = torch.empty(max(A.m, 1), dtype=torch.int32, device=device)
        short_thr = int(medium_threshold) if n_med.value > 0 else int(threshold)
        _check(lib().spx_rowplan_build_short(ctypes.byref(A), short_thr, ptr(short), ctypes.byref(n_short),
                                             ctypes.byref(n_groups), ptr(ws), ws.numel(), _stream()),
               "spx_rowplan_build_short")
        short = short[: n_short.value].clone() if n_short.value > 0 else short[:1]
    use_short = short_order and A.m > 0 and n_groups.value > 1       # one group: the natural order
    plan = spx_rowplan(rows.data_ptr() if n_long.value > 0 else None, n_long.value, int(threshold), 0, 0, 0,
                       med.data_ptr() if n_med.value > 0 else None, n_med.value,
                       int(medium_threshold) if n_med.value > 0 else 0, None, 0,
                       short.data_ptr() if use_short else None, n_short.value if use_short else 0)
    return (rows, med, short), plan


def spx_rowplan_build_parts(A: spx_csr, n_parts: int, device):
    """Column-range split of A's rows into n_parts segments: (part_ptr tensor, n_parts)."""
    out = torch.empty(max((n_parts - 1) * A.m, 1), dtype=torch.int32, device=device)
    _check(lib().spx_rowplan_build_parts(ctypes.byref(A), int(n_parts), ptr(out), _stream()),
           "spx_rowplan_build_parts")
    return out, int(n_parts)


def _planp(plan):
    return ctypes.byref(plan) if plan is not None else None


def _wsargs(ws):
    return (ptr(ws), ws.numel()) if ws is not None else (None, 0)


def spx_spmm_workspace_size(A: spx_csr, k: int, plan: spx_rowplan | None = None) -> int:
    sz = _SZ(0)
    _check(lib().spx_spmm_workspace_size(ctypes.byref(A), int(k), _planp(plan), ctypes.byref(sz)),
           "spx_spmm_workspace_size")
    return sz.value


def spx_spmm(A: spx_csr, X, Y, alpha=1.0, beta=0.0, plan: spx_rowplan | None = None, ws=None):
    px, ldx = _dense(X, "X")
    py, ldy = _dense(Y, "Y")
    _check(lib().spx_spmm(ctypes.byref(A), px, ldx, X.shape[1], py, ldy, float(alpha), float(beta),
                          _planp(plan), *_wsargs(ws), _stream()), "spx_spmm")
    return Y


def spx_merge_plan_build(A: spx_csr, items: int, device):
    """Merge-path partition of A's rows + entries into segments of `items` items: returns
    (seg_row tensor, spx_mergeplan)."""
    ns = _I32(0)
    _check(lib().spx_merge_plan_segments(ctypes.byref(A), int(items), ctypes.byref(ns)), "spx_merge_plan_segments")
    seg = torch.empty(ns.value + 1, dtype=torch.int32, device=device)
    _check(lib().spx_merge_plan_build(ctypes.byref(A), int(items), seg.data_ptr(), ns.value, _stream()),
           "spx_merge_plan_build")
    return seg, spx_mergeplan(seg.data_ptr(), ns.value, int(items))


def spx_spmm_merge_workspace_size(A: spx_csr, k: int, plan: spx_mergeplan) -> int:
    sz = _SZ(0)
    _check(lib().spx_spmm_merge_workspace_size(ctypes.byref(A), int(k), ctypes.byref(plan), ctypes.byref(sz)),
           "spx_spmm_merge_workspace_size")
    return sz.value


def spx_spmm_merge(A: spx_csr, X, Y, plan: spx_mergeplan, ws, alpha=1.0, beta=0.0, perm=None, variant=0):
    px, ldx = _dense(X, "X")
    py, ldy = _dense(Y, "Y")
    _check(lib().spx_spmm_merge(ctypes.byref(A), ptr(perm) if perm is not None else None, px, ldx, X.shape[1], py,
                                ldy, float(alpha), float(beta), ctypes.byref(plan), int(variant), *_wsargs(ws),
                                _stream()), "spx_spmm_merge")
    return Y


def spx_sddmm_merge(A: spx_csr, G, X, out, plan: spx_mergeplan, scale=1.0, variant=0):
    pg, ldg = _dense(G, "G")
    px, ldx = _dense(X, "X")
    _check(lib().spx_sddmm_merge(ctypes.byref(A), pg, ldg, px, ldx, G.shape[1], float(scale), ptr(out),
                                 ctypes.byref(plan), int(variant), _stream()), "spx_sddmm_merge")
    return out


def spx_sddmm_workspace_size(A: spx_csr, k: int, col_block: int = 0) -> int:
    sz = _SZ(0)
    _check(lib().spx_sddmm_workspace_size(ctypes.byref(A), int(k), int(col_block), ctypes.byref(sz)),
           "spx_sddmm_workspace_size")
    return sz.value


def spx_sddmm(A: spx_csr, G, X, out, scale=1.0, col_block=0, ws=None, plan: spx_rowplan | None = None):
    pg, ldg = _dense(G, "G")
    px, ldx = _dense(X, "X")
    _check(lib().spx_sddmm(ctypes.byref(A), pg, ldg, px, ldx, G.shape[1], float(scale), ptr(out),
                           int(col_block), _planp(plan), *_wsargs(ws), _stream()), "spx_sddmm")
    return out


def spx_masked_outer(A: spx_csr, u, v, out, scale=1.0):
    _check(lib().spx_masked_outer(ctypes.byref(A), ptr(u), ptr(v), float(scale), ptr(out), _stream()),
           "spx_masked_outer")
    return out


def spx_csr_transpose(A: spx_csr, device):
    """Returns (t_indptr, t_indices, perm) int32 CUDA tensors."""
    sz = _SZ(0)
    _check(lib().spx_transpose_workspace_size(A.m, A.n, A.nnz, ctypes.byref(sz)),
           "spx_transpose_workspace_size")
    ws = workspace(sz.value, device)
    t_ip = torch.empty(A.n + 1, dtype=torch.int32, device=device)
    t_ix = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=device)
    perm = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=device)
    _check(lib().spx_csr_transpose(ctypes.byref(A), ptr(t_ip), ptr(t_ix), ptr(perm), ptr(ws), ws.numel(),
                                   _stream()), "spx_csr_transpose")
    return t_ip, t_ix[: A.nnz], perm[: A.nnz]


def spx_spmm_t_workspace_size(AT: spx_csr, k: int, plan: spx_rowplan | None = None) -> int:
    sz = _SZ(0)
    _check(lib().spx_spmm_t_workspace_size(ctypes.byref(AT), int(k), _planp(plan), ctypes.byref(sz)),
           "spx_spmm_t_workspace_size")
    return sz.value


def spx_spmm_t_noalloc(AT: spx_csr, perm, G, gX, alpha=1.0, beta=0.0, plan: spx_rowplan | None = None):
    """spx_spmm_t staging A^T's values in the library's built-in scratch (no allocation)."""
    pg, ldg = _dense(G, "G")
    px, ldx = _dense(gX, "gX")
    _check(lib().spx_spmm_t_noalloc(ctypes.byref(AT), ptr(perm), pg, ldg, G.shape[1], px, ldx, float(alpha),
                                    float(beta), _planp(plan), _stream()), "spx_spmm_t_noalloc")
    return gX


def spx_spmm_t(AT: spx_csr, perm, G, gX, alpha=1.0, beta=0.0, plan: spx_rowplan | None = None,
               ws=None):
    pg, ldg = _dense(G, "G")
    px, ldx = _dense(gX, "gX")
    _check(lib().spx_spmm_t(ctypes.byref(AT), ptr(perm), pg, ldg, G.shape[1], px, ldx, float(alpha),
                            float(beta), _planp(plan), *_wsargs(ws), _stream()), "spx_spmm_t")
    return gX


def spx_spmm_t_sddmm(AT: spx_csr, perm, a_values, G, X, gX, gA, alpha=1.0, beta=0.0, scale=1.0,
                     plan: spx_rowplan | None = None, variant: int = 0):
    """gX = alpha A^T G + beta gX and gA = scale (G X^T) on A's pattern, in one pass."""
    pg, ldg = _dense(G, "G")
    pxx, ldx = _dense(X, "X")
    px, ldgx = _dense(gX, "gX")
    _check(lib().spx_spmm_t_sddmm(ctypes.byref(AT), ptr(perm), ptr(a_values), pg, ldg, pxx, ldx, G.shape[1], px,
                                  ldgx, float(alpha), float(beta), ptr(gA), float(scale), _planp(plan), int(variant),
                                  _stream()),
           "spx_spmm_t_sddmm")
    return gX, gA


# ------------------------------------------------------------------ SpGEMM
def spx_spgemm_workspace_size(m: int) -> int:
    sz = _SZ(0)
    _check(lib().spx_spgemm_workspace_size(int(m), ctypes.byref(sz)), "spx_spgemm_workspace_size")
    return sz.value


def spx_spgemm_analyse(A: spx_csr, B: spx_csr, ws, read_back: bool = True):
    """The number of products (synchronises), or None without the read-back (asynchronous)."""
    prods = _I64(0)
    _check(lib().spx_spgemm_analyse(ctypes.byref(A), ctypes.byref(B), ctypes.byref(prods) if read_back else None,
                                    ptr(ws), ws.numel(), _stream()), "spx_spgemm_analyse")
    return prods.value if read_back else None


def spx_spgemm_symbolic(A: spx_csr, B: spx_csr, c_indptr, ws, scratch, products: int, read_back: bool = True):
    """nnz(C) (synchronises), or None without the read-back (asynchronous)."""
    nnz = _I64(0)
    _check(lib().spx_spgemm_symbolic(ctypes.byref(A), ctypes.byref(B), int(products), ptr(c_indptr),
                                     ctypes.byref(nnz) if read_back else None, ptr(ws), ws.numel(), ptr(scratch),
                                     scratch.numel(), _stream()), "spx_spgemm_symbolic")
    return nnz.value if read_back else None


def spx_spgemm_fill(A: spx_csr, c_indptr, c_indices, ws, scratch):
    _check(lib().spx_spgemm_fill(ctypes.byref(A), ptr(c_indptr), ptr(c_indices), ptr(ws), ws.numel(),
                                 ptr(scratch), _stream()), "spx_spgemm_fill")


def spx_spgemm_numeric(A: spx_csr, B: spx_csr, C: spx_csr, c_values, ws):
    _check(lib().spx_spgemm_numeric(ctypes.byref(A), ctypes.byref(B), ctypes.byref(C), ptr(c_values),
                                    ptr(ws), ws.numel(), _stream()), "spx_spgemm_numeric")


def spx_spgemm_backward(A: spx_csr, B: spx_csr, C: spx_csr, gc, ga, gb, at_indptr=None, at_indices=None,
                        a_perm=None):
    _check(lib().spx_spgemm_backward(ctypes.byref(A), ctypes.byref(B), ctypes.byref(C), ptr(gc), ptr(ga),
                                     ptr(gb), ptr(at_indptr), ptr(at_indices), ptr(a_perm), _stream()),
           "spx_spgemm_backward")


# ------------------------------------------------------------------ solve
def spx_csr_diagonal(A: spx_csr, diag, pos):
    _check(lib().spx_csr_diagonal(ctypes.byref(A), ptr(diag), ptr(pos), _stream()), "spx_csr_diagonal")


def spx_diagonal_backward(pos, g_diag, g_values):
    _check(lib().spx_diagonal_backward(int(pos.numel()), ptr(pos), ptr(g_diag), ptr(g_values), _stream()),
           "spx_diagonal_backward")


def spx_gather_probe(indices, n, X, unroll=2, blocks_per_sm=8, out=None):
    """Reads X's rows in the order of the column stream `indices` (a measurement of the
    gather bound); returns the per-thread sums buffer."""
    if out is None:
        out = torch.zeros(16 * 256 * torch.cuda.get_device_properties(X.device).multi_processor_count,
                          device=X.device)
    _check(lib().spx_gather_probe(ptr(indices), int(indices.numel()), int(n), ptr(X), int(X.stride(0)),
                                  int(X.shape[1]), int(unroll), int(blocks_per_sm), ptr(out), int(out.numel()),
                                  _stream()), "spx_gather_probe")
    return out


def spx_gather_values(perm, src, dst):
    _check(lib().spx_gather_values(int(perm.numel()), ptr(perm), ptr(src), ptr(dst), _stream()),
           "spx_gather_values")
    return dst


def spx_cg_workspace_size(n: int) -> int:
    sz = _SZ(0)
    _check(lib().spx_cg_workspace_size(int(n), ctypes.byref(sz)), "spx_cg_workspace_size")
    return sz.value


def spx_cg_batched(A: spx_csr, sys_ptr, nsys: int, order, b, x, pc_kind: int, dinv, L: spx_csr | None,
                   LT: spx_csr | None, tol: float, maxit: int, delta: float, iters, status, relres, ws,
                   ic0_levels=None):
    lev = None
    if ic0_levels is not None:
        lev = (ctypes.c_void_p * 3)(*[t.data_ptr() for t in ic0_levels])
    _check(lib().spx_cg_batched(ctypes.byref(A), ptr(sys_ptr), int(nsys), ptr(order), ptr(b), ptr(x),
                                int(pc_kind), ptr(dinv), ctypes.byref(L) if L is not None else None,
                                ctypes.byref(LT) if LT is not None else None, lev, float(tol), int(maxit),
                                float(delta), ptr(iters), ptr(status), ptr(relres), ptr(ws), ws.numel(),
                                _stream()), "spx_cg_batched")


DIA_MAX = 3
MDIA_MAX = 4


def spx_dia_analyse(L: spx_csr, sys_ptr, nsys: int, device):
    """Diagonal form of a lower-triangular pattern per system: (offsets int32[nsys * 3],
    counts int32[nsys], every system supported)."""
    offs = torch.zeros(max(nsys, 1) * DIA_MAX, dtype=torch.int32, device=device)
    nd = torch.zeros(max(nsys, 1), dtype=torch.int32, device=device)
    ok = _I32(0)
    _check(lib().spx_dia_analyse(ctypes.byref(L), ptr(sys_ptr), int(nsys), ptr(offs), ptr(nd), ctypes.byref(ok),
                                 _stream()), "spx_dia_analyse")
    return offs, nd, bool(ok.value)


def spx_dia_fill(L: spx_csr, sys_ptr, nsys: int, offs, nd, out_bf16):
    _check(lib().spx_dia_fill(ctypes.byref(L), ptr(sys_ptr), int(nsys), ptr(offs), ptr(nd), ptr(out_bf16),
                              _stream()), "spx_dia_fill")
    return out_bf16


def spx_dia_square(sys_ptr, nsys: int, n: int, l_offs, l_nd, l_vals_bf16, device, out=None):
    """M = L L^T by its lower diagonals: (offsets int32[nsys * 4], counts int32[nsys],
    values BF16[4 * n]), written into `out` (the same three tensors) when given."""
    if out is None:
        out = (torch.zeros(max(nsys, 1) * MDIA_MAX, dtype=torch.int32, device=device),
               torch.zeros(max(nsys, 1), dtype=torch.int32, device=device),
               torch.zeros(MDIA_MAX * max(n, 1), dtype=torch.bfloat16, device=device))
    m_offs, m_nd, m_vals = out
    _check(lib().spx_dia_square(ptr(sys_ptr), int(nsys), int(n), ptr(l_offs), ptr(l_nd), ptr(l_vals_bf16),
                                ptr(m_offs), ptr(m_nd), ptr(m_vals), _stream()), "spx_dia_square")
    return m_offs, m_nd, m_vals


def spx_cg_batched_dia(A: spx_csr, sys_ptr, nsys: int, order, b, x, offs, nd, vals_bf16, tol: float, maxit: int,
                       delta: float, iters, status, relres, ws):
    _check(lib().spx_cg_batched_dia(ctypes.byref(A), ptr(sys_ptr), int(nsys), ptr(order), ptr(b), ptr(x), ptr(offs),
                                    ptr(nd), ptr(vals_bf16), float(tol), int(maxit), float(delta), ptr(iters),
                                    ptr(status), ptr(relres), ptr(ws), ws.numel(), _stream()), "spx_cg_batched_dia")


def spx_ic0_analyse(Lpat: spx_csr, sys_ptr, nsys: int, device):
    """Returns (sys_lev_off, lev_ptr, lev_rows) int32 tensors."""
    sz = _SZ(0)
    _check(lib().spx_ic0_workspace_size(int(Lpat.m), int(nsys), ctypes.byref(sz)), "spx_ic0_workspace_size")
    ws = workspace(sz.value, device)
    off = torch.empty(nsys + 1, dtype=torch.int32, device=device)
    lp = torch.empty(Lpat.m + nsys + 1, dtype=torch.int32, device=device)
    rows = torch.empty(max(Lpat.m, 1), dtype=torch.int32, device=device)
    _check(lib().spx_ic0_analyse(ctypes.byref(Lpat), ptr(sys_ptr), int(nsys), ptr(off), ptr(lp), ptr(rows), ptr(ws),
                                 ws.numel(), _stream()), "spx_ic0_analyse")
    return off, lp, rows


def spx_ic0_factor(Lpat: spx_csr, l_src, a_values, nsys: int, levels, l_values, status):
    off, lp, rows = levels
    _check(lib().spx_ic0_factor(ctypes.byref(Lpat), ptr(l_src), ptr(a_values), int(nsys), ptr(off), ptr(lp),
                                ptr(rows), ptr(l_values), ptr(status), _stream()), "spx_ic0_factor")


def spx_diag_inverse(A: spx_csr, dinv):
    _check(lib().spx_diag_inverse(ctypes.byref(A), ptr(dinv), _stream()), "spx_diag_inverse")
    return dinv


def spx_masked_outer_f64(A: spx_csr, u, v, out, scale=1.0):
    _check(lib().spx_masked_outer_f64(ctypes.byref(A), ptr(u), ptr(v), float(scale), ptr(out), _stream()),
           "spx_masked_outer_f64")
    return out


# ------------------------------------------------------------------ learned preconditioner
def _size(fn, *args):
    sz = _SZ(0)
    _check(getattr(lib(), fn)(*args, ctypes.byref(sz)), fn)
    return sz.value


def spx_pcg_train(A: spx_csr, sys_ptr, nsys, L: spx_csr, LT: spx_csr, b, n_it, weights, loss, grad_L, ws,
                  ckpt_interval=0):
    _check(lib().spx_pcg_train(ctypes.byref(A), ptr(sys_ptr), int(nsys), ctypes.byref(L), ctypes.byref(LT),
                               ptr(b), int(n_it), int(ckpt_interval), ptr(weights), ptr(loss), ptr(grad_L), ptr(ws),
                               ws.numel(), _stream()), "spx_pcg_train")


def spx_mpnn_features(A: spx_csr, d, e_vals, feats):
    _check(lib().spx_mpnn_features(ctypes.byref(A), ptr(d), ptr(e_vals), ptr(feats), _stream()),
           "spx_mpnn_features")


def spx_dense_forward(n, X1, K1, X2, K2, W16, bias, N, mode, Hin, Y, U=None):
    _check(lib().spx_dense_forward(int(n), ptr(X1), int(K1), ptr(X2), int(K2), ptr(W16), ptr(bias), int(N),
                                   int(mode), ptr(Hin), ptr(Y), ptr(U), _stream()), "spx_dense_forward")


def spx_dense_forward_tc(n, X1, K1, X2, K2, W16, bias, N, mode, Hin, Y, U=None):
    _check(lib().spx_dense_forward_tc(int(n), ptr(X1), int(K1), ptr(X2), int(K2), ptr(W16), ptr(bias), int(N),
                                      int(mode), ptr(Hin), ptr(Y), ptr(U), _stream()), "spx_dense_forward_tc")


def spx_dense_backward_data(n, G, N, W16, K1, K2, dX1, dX2, accumulate):
    _check(lib().spx_dense_backward_data(int(n), ptr(G), int(N), ptr(W16), int(K1), int(K2), ptr(dX1), ptr(dX2),
                                         int(accumulate), _stream()), "spx_dense_backward_data")


def spx_dense_backward_data_tc(n, G, N, W16, K1, K2, dX1, dX2, accumulate):
    _check(lib().spx_dense_backward_data_tc(int(n), ptr(G), int(N), ptr(W16), int(K1), int(K2), ptr(dX1),
                                            ptr(dX2), int(accumulate), _stream()), "spx_dense_backward_data_tc")


def spx_tc_set_pipeline(enabled: bool):
    _check(lib().spx_tc_set_pipeline(1 if enabled else 0), "spx_tc_set_pipeline")


def spx_dense_backward_weight_tc(n, X1, K1, X2, K2, G, N, dW, db, ws):
    _check(lib().spx_dense_backward_weight_tc(int(n), ptr(X1), int(K1), ptr(X2), int(K2), ptr(G), int(N), ptr(dW),
                                              ptr(db), ptr(ws), ws.numel(), _stream()),
           "spx_dense_backward_weight_tc")


def spx_dense_backward_weight(n, X1, K1, X2, K2, G, N, dW, db, ws):
    _check(lib().spx_dense_backward_weight(int(n), ptr(X1), int(K1), ptr(X2), int(K2), ptr(G), int(N), ptr(dW),
                                           ptr(db), ptr(ws), ws.numel(), _stream()), "spx_dense_backward_weight")


def spx_relu_backward(gh, u, gu):
    _check(lib().spx_relu_backward(int(gh.numel()), ptr(gh), ptr(u), ptr(gu), _stream()), "spx_relu_backward")


def spx_tril_pattern(A: spx_csr, device):
    """Returns (l_indptr, l_indices, l_src) int32 tensors of tril(A)."""
    ws = workspace(_size("spx_tril_workspace_size", int(A.m)), device)
    ip = torch.empty(A.m + 1, dtype=torch.int32, device=device)
    nnz = _I64(0)
    _check(lib().spx_tril_pattern(ctypes.byref(A), ptr(ip), None, None, ctypes.byref(nnz), ptr(ws), ws.numel(),
                                  _stream()), "spx_tril_pattern")
    ix = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=device)
    src = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=device)
    _check(lib().spx_tril_pattern(ctypes.byref(A), ptr(ip), ptr(ix), ptr(src), ctypes.byref(nnz), ptr(ws),
                                  ws.numel(), _stream()), "spx_tril_pattern")
    return ip, ix[: nnz.value], src[: nnz.value]


def spx_edge_forward(Lpat: spx_csr, e_low, d, P, Q, u, c, v, bd, bo, L_values):
    _check(lib().spx_edge_forward(ctypes.byref(Lpat), ptr(e_low), ptr(d), ptr(P), ptr(Q), ptr(u), ptr(c), ptr(v),
                                  ptr(bd), ptr(bo), ptr(L_values), _stream()), "spx_edge_forward")


def spx_edge_backward(Lpat: spx_csr, lt_ip, lt_ix, lt_perm, e_low, d, P, Q, u, c, v, bd, bo, gL, gP, gQ,
                      gparams, ws):
    _check(lib().spx_edge_backward(ctypes.byref(Lpat), ptr(lt_ip), ptr(lt_ix), ptr(lt_perm), ptr(e_low), ptr(d),
                                   ptr(P), ptr(Q), ptr(u), ptr(c), ptr(v), ptr(bd), ptr(bo), ptr(gL), ptr(gP),
                                   ptr(gQ), ptr(gparams), ptr(ws), ws.numel(), _stream()), "spx_edge_backward")


def spx_adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, params_bf16=None):
    _check(lib().spx_adam_step(int(params.numel()), ptr(params), ptr(grads), ptr(m), ptr(v), int(step),
                               float(lr), float(beta1), float(beta2), float(eps), ptr(params_bf16), _stream()),
           "spx_adam_step")


def spx_to_bf16(src, dst):
    _check(lib().spx_to_bf16(int(src.numel()), ptr(src), ptr(dst), _stream()), "spx_to_bf16")


def spx_sptrsv(T: spx_csr, upper: bool, nsys: int, levels, b, x, status=None):
    off, lp, rows = levels
    _check(lib().spx_sptrsv(ctypes.byref(T), int(bool(upper)), int(nsys), ptr(off), ptr(lp), ptr(rows), ptr(b),
                            ptr(x), ptr(status), _stream()), "spx_sptrsv")
    return x


def _levels_arg(levels):
    if levels is None:
        return None
    arr = (ctypes.c_void_p * 3)(*[t.data_ptr() for t in levels])
    return ctypes.cast(arr, ctypes.c_void_p), arr            # keep arr alive with the pointer


def spx_precond_apply(kind: int, r, z, dinv=None, L: spx_csr | None = None, LT: spx_csr | None = None,
                      nsys: int = 0, levels=None, tmp=None):
    lv = _levels_arg(levels)
    _check(lib().spx_precond_apply(int(kind), int(r.numel()), ptr(r), ptr(z), ptr(dinv),
                                   ctypes.byref(L) if L is not None else None,
                                   ctypes.byref(LT) if LT is not None else None, int(nsys),
                                   lv[0] if lv else None, ptr(tmp), _stream()), "spx_precond_apply")
    return z


def spx_cg_adjoint(A: spx_csr, sys_ptr, nsys, order, x, g, lam, grad_A, pc_kind, dinv, L, LT, tol, maxit, delta,
                   iters, status, relres, ws, ic0_levels=None):
    lv = _levels_arg(ic0_levels)
    _check(lib().spx_cg_adjoint(ctypes.byref(A), ptr(sys_ptr), int(nsys), ptr(order), ptr(x), ptr(g), ptr(lam),
                                ptr(grad_A), int(pc_kind), ptr(dinv), ctypes.byref(L) if L is not None else None,
                                ctypes.byref(LT) if LT is not None else None, lv[0] if lv else None, float(tol),
                                int(maxit), float(delta), ptr(iters), ptr(status), ptr(relres), ptr(ws), ws.numel(),
                                _stream()), "spx_cg_adjoint")


def spx_spmm_autotune(A: spx_csr, X, Y, plan: spx_rowplan):
    """Times spx_spmm's launch parameters on the device; returns (plan, ms per call)."""
    px, ldx = _dense(X, "X")
    py, ldy = _dense(Y, "Y")
    p = spx_rowplan.from_buffer_copy(plan)
    ms = _F(0.0)
    _check(lib().spx_spmm_autotune(ctypes.byref(A), px, ldx, int(X.shape[1]), py, ldy, ctypes.byref(p),
                                   ctypes.byref(ms), _stream()), "spx_spmm_autotune")
    return p, float(ms.value)


def spx_sync_status(status_dev):
    """Host copy of the status words; raises SpxError on the first one that is not SPX_OK."""
    out = (ctypes.c_int32 * max(int(status_dev.numel()), 1))()
    _check(lib().spx_sync_status(ptr(status_dev), int(status_dev.numel()), out, _stream()), "spx_sync_status")
    return list(out)[: int(status_dev.numel())]


def spx_spadd_symbolic(A: spx_csr, B: spx_csr, c_indptr, device) -> int:
    sz = _SZ(0)
    _check(lib().spx_spadd_workspace_size(A.m, ctypes.byref(sz)), "spx_spadd_workspace_size")
    ws = workspace(sz.value, device)
    nnz = _I64(0)
    _check(lib().spx_spadd_symbolic(ctypes.byref(A), ctypes.byref(B), ptr(c_indptr), ctypes.byref(nnz), ptr(ws),
                                    ws.numel(), _stream()), "spx_spadd_symbolic")
    return nnz.value


def spx_spadd_fill(A: spx_csr, B: spx_csr, c_indptr, c_indices, src_a, src_b, pos_a, pos_b):
    _check(lib().spx_spadd_fill(ctypes.byref(A), ctypes.byref(B), ptr(c_indptr), ptr(c_indices), ptr(src_a),
                                ptr(src_b), ptr(pos_a), ptr(pos_b), _stream()), "spx_spadd_fill")


def spx_spadd_numeric(alpha, a_vals, src_a, beta, b_vals, src_b, c_vals):
    _check(lib().spx_spadd_numeric(int(c_vals.numel()), float(alpha), ptr(a_vals), ptr(src_a), float(beta),
                                   ptr(b_vals), ptr(src_b), ptr(c_vals), _stream()), "spx_spadd_numeric")
    return c_vals


def spx_spadd_backward(alpha, beta, gc, pos_a, pos_b, ga=None, gb=None):
    _check(lib().spx_spadd_backward(int(pos_a.numel()), int(pos_b.numel()), float(alpha), float(beta), ptr(gc),
                                    ptr(pos_a), ptr(pos_b), ptr(ga), ptr(gb), _stream()), "spx_spadd_backward")


def spx_spai_residual(C: spx_csr, scale: float, out, diag_count=None):
    _check(lib().spx_spai_residual(ctypes.byref(C), float(scale), ptr(out), ptr(diag_count), _stream()),
           "spx_spai_residual")
    return out


def spx_dot_workspace_size(n: int) -> int:
    sz = _SZ(0)
    _check(lib().spx_dot_workspace_size(int(n), ctypes.byref(sz)), "spx_dot_workspace_size")
    return sz.value


def spx_dot(x, y, out, ws):
    """out (device float64 scalar tensor) = <x, y>."""
    _check(lib().spx_dot(int(x.numel()), ptr(x), ptr(y), ptr(out), ptr(ws), ws.numel(), _stream()), "spx_dot")
    return out


def spx_spai_update(m, g, gg, dada):
    _check(lib().spx_spai_update(int(m.numel()), ptr(m), ptr(g), ptr(gg), ptr(dada), _stream()),
           "spx_spai_update")


def spx_cg_set_vector_residency(shared_memory: int = 1):
    _check(lib().spx_cg_set_vector_residency(int(shared_memory)), "spx_cg_set_vector_residency")


def spx_cg_set_launch(threads_per_block: int = 0, cluster_size: int = 0, max_clusters: int = 0):
    _check(lib().spx_cg_set_launch(int(threads_per_block), int(cluster_size), int(max_clusters)),
           "spx_cg_set_launch")
