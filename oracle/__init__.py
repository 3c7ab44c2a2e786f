"""FP64 CPU oracle for the sparse forward / reverse-mode operations.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The product path (the CUDA
library and its Python binding) never imports, links or executes anything here, and
this package imports nothing from the product.

The arithmetic lives in ``spx_oracle.c`` (plain serial C loops in double precision,
compiled with gcc by :func:`build`); this module only marshals numpy arrays.  Inputs
arrive as float32 (what the GPU consumes) and are promoted exactly to float64.

Submodules: ``pcg_unrolled`` (the unrolled-PCG loss of Section 4.3 and its reverse),
``mpnn`` (the learned-preconditioner network), ``spai`` (Section 4.6: SPAI by gradient
descent and the static-pattern SPAI), ``spadd`` and ``sptrsv`` (sparse add and the
triangular solve with their gradients), ``adam`` (the optimiser that trains the network).

Parity pins: every function here is checked by ``tests/test_oracle_*.py`` against
dense linear algebra, closed forms of the model problems, finite differences or
brute force on tiny inputs (see the test files for which pin covers which routine).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spx_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

PC_NONE, PC_JACOBI, PC_LLT, PC_IC0 = 0, 1, 2, 3
STATUS_NAMES = {0: "converged", 1: "maxiter", 2: "breakdown", 3: "nonfinite"}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I = ctypes.c_int64


def _declare(lib):
    sig = {
        "orc_spmm": (None, [_I, _P, _P, _P, _P, _I, _P]),
        "orc_sddmm": (None, [_I, _P, _P, _P, _P, _I, _P]),
        "orc_transpose": (None, [_I, _I, _P, _P, _P, _P, _P]),
        "orc_spmm_t": (None, [_I, _I, _P, _P, _P, _P, _I, _P]),
        "orc_spmm_mt": (ctypes.c_int, [_I, _P, _P, _P, _P, _I, _P, ctypes.c_int]),
        "orc_sddmm_mt": (ctypes.c_int, [_I, _P, _P, _P, _P, _I, _P, ctypes.c_int]),
        "orc_spmm_t_mt": (ctypes.c_int, [_I, _P, _P, _P, _P, _P, _I, _P, ctypes.c_int]),
        "orc_spgemm_count": (_I, [_I, _I, _P, _P, _P, _P, _P, _P]),
        "orc_spgemm_fill": (None, [_I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
        "orc_spgemm_grad_a": (None, [_I, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
        "orc_spgemm_grad_b": (None, [_I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
        "orc_trsv_lower": (None, [_I, _P, _P, _P, _P, _P]),
        "orc_trsv_lower_t": (None, [_I, _P, _P, _P, _P, _P]),
        "orc_ic0": (ctypes.c_int, [_I, _P, _P, _P, _P, _P, _P]),
        "orc_pcg": (ctypes.c_int, [_I, _P, _P, _P, _P, _P, ctypes.c_int, _P, _P, _P, _P,
                                   ctypes.c_double, _I, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


# ----------------------------------------------------------------------------- ops
def spmm(A, X):
    """Y = A X (SpMV when X is 1-D).  Section 3.1.1 / 3.1.3."""
    X = _f64(X)
    vec = X.ndim == 1
    X2 = X.reshape(A.n, -1)
    k = X2.shape[1]
    Y = np.empty((A.m, k), dtype=np.float64)
    ip, ix, v = _i32(A.indptr), _i32(A.indices), _f64(A.values)
    _L().orc_spmm(A.m, _p(ip), _p(ix), _p(v), _p(X2), k, _p(Y))
    return Y.reshape(-1) if vec else Y


def sddmm(A, G, X):
    """Values on mask(A) of G X^T: the SpMV / SpDMM VJP w.r.t. A (Table 1)."""
    G = _f64(G).reshape(A.m, -1)
    X = _f64(X).reshape(A.n, -1)
    k = G.shape[1]
    assert X.shape[1] == k
    out = np.empty(A.nnz, dtype=np.float64)
    ip, ix = _i32(A.indptr), _i32(A.indices)
    _L().orc_sddmm(A.m, _p(ip), _p(ix), _p(G), _p(X), k, _p(out))
    return out


def transpose(A):
    """(AT_indptr, AT_indices, perm) with AT.values = A.values[perm] (stable by row)."""
    ip, ix = _i32(A.indptr), _i32(A.indices)
    t_ip = np.empty(A.n + 1, dtype=np.int32)
    t_ix = np.empty(A.nnz, dtype=np.int32)
    perm = np.empty(A.nnz, dtype=np.int32)
    _L().orc_transpose(A.m, A.n, _p(ip), _p(ix), _p(t_ip), _p(t_ix), _p(perm))
    return t_ip, t_ix, perm


def spmm_t(A, G):
    """gX = A^T G: the SpMV / SpDMM VJP w.r.t. the dense operand (Table 1)."""
    G = _f64(G)
    vec = G.ndim == 1
    G2 = G.reshape(A.m, -1)
    k = G2.shape[1]
    gX = np.empty((A.n, k), dtype=np.float64)
    ip, ix, v = _i32(A.indptr), _i32(A.indices), _f64(A.values)
    _L().orc_spmm_t(A.m, A.n, _p(ip), _p(ix), _p(v), _p(G2), k, _p(gX))
    return gX.reshape(-1) if vec else gX


def spmm_mt(A, X, threads):
    """spmm on `threads` host threads (row blocks of equal entry counts); equal bit for bit
    to spmm.  Returns (Y, threads used)."""
    X2 = _f64(X).reshape(A.n, -1)
    k = X2.shape[1]
    Y = np.empty((A.m, k), dtype=np.float64)
    ip, ix, v = _i32(A.indptr), _i32(A.indices), _f64(A.values)
    used = _L().orc_spmm_mt(A.m, _p(ip), _p(ix), _p(v), _p(X2), k, _p(Y), int(threads))
    return Y, used


def sddmm_mt(A, G, X, threads):
    """sddmm on `threads` host threads; equal bit for bit to sddmm.  Returns (out, threads)."""
    G = _f64(G).reshape(A.m, -1)
    X = _f64(X).reshape(A.n, -1)
    k = G.shape[1]
    out = np.empty(A.nnz, dtype=np.float64)
    ip, ix = _i32(A.indptr), _i32(A.indices)
    used = _L().orc_sddmm_mt(A.m, _p(ip), _p(ix), _p(G), _p(X), k, _p(out), int(threads))
    return out, used


def spmm_t_mt(A, G, threads, t=None):
    """spmm_t on `threads` host threads as rows of the transpose (t = transpose(A), computed
    here if not given); equal bit for bit to spmm_t.  Returns (gX, threads used)."""
    t_ip, t_ix, perm = t if t is not None else transpose(A)
    G2 = _f64(G).reshape(A.m, -1)
    k = G2.shape[1]
    gX = np.empty((A.n, k), dtype=np.float64)
    v = _f64(A.values)
    used = _L().orc_spmm_t_mt(A.n, _p(_i32(t_ip)), _p(_i32(t_ix)), _p(_i32(perm)), _p(v), _p(G2), k, _p(gX),
                              int(threads))
    return gX, used


def spgemm_count(A, B):
    """(row_nnz int64[m], row_products int64[m], nnz_C) of the structural product."""
    assert A.n == B.m
    row_nnz = np.empty(A.m, dtype=np.int64)
    row_prod = np.empty(A.m, dtype=np.int64)
    a_ip, a_ix, b_ip, b_ix = _i32(A.indptr), _i32(A.indices), _i32(B.indptr), _i32(B.indices)
    tot = _L().orc_spgemm_count(A.m, B.n, _p(a_ip), _p(a_ix), _p(b_ip), _p(b_ix),
                                _p(row_nnz), _p(row_prod))
    return row_nnz, row_prod, int(tot)


def spgemm(A, B):
    """C = A B, all CSR (Section 3.1.2): returns (indptr int32, indices int32, values f64)."""
    row_nnz, _, tot = spgemm_count(A, B)
    c_ip = np.zeros(A.m + 1, dtype=np.int64)
    np.cumsum(row_nnz, out=c_ip[1:])
    assert c_ip[-1] < 2**31
    c_ip = c_ip.astype(np.int32)
    c_ix = np.empty(tot, dtype=np.int32)
    c_v = np.empty(tot, dtype=np.float64)
    a_ip, a_ix, b_ip, b_ix = _i32(A.indptr), _i32(A.indices), _i32(B.indptr), _i32(B.indices)
    a_v, b_v = _f64(A.values), _f64(B.values)
    _L().orc_spgemm_fill(A.m, B.n, _p(a_ip), _p(a_ix), _p(a_v), _p(b_ip), _p(b_ix), _p(b_v),
                         _p(c_ip), _p(c_ix), _p(c_v))
    return c_ip, c_ix, c_v


def spgemm_grad_a(A, B, c_indptr, c_indices, gc):
    """(V B^T) on mask(A), V given on C's pattern (Table 1, SpSpMM w.r.t. A)."""
    out = np.empty(A.nnz, dtype=np.float64)
    a_ip, a_ix, b_ip, b_ix = _i32(A.indptr), _i32(A.indices), _i32(B.indptr), _i32(B.indices)
    c_ip, c_ix, g = _i32(c_indptr), _i32(c_indices), _f64(gc)
    _L().orc_spgemm_grad_a(A.m, _p(a_ip), _p(a_ix), _p(b_ip), _p(b_ix), _p(_f64(B.values)),
                           _p(c_ip), _p(c_ix), _p(g), _p(out))
    return out


def spgemm_grad_b(A, B, c_indptr, c_indices, gc):
    """(A^T V) on mask(B), V given on C's pattern (Table 1, SpSpMM w.r.t. B)."""
    out = np.empty(B.nnz, dtype=np.float64)
    a_ip, a_ix, b_ip, b_ix = _i32(A.indptr), _i32(A.indices), _i32(B.indptr), _i32(B.indices)
    c_ip, c_ix, g = _i32(c_indptr), _i32(c_indices), _f64(gc)
    _L().orc_spgemm_grad_b(A.m, B.nnz, _p(a_ip), _p(a_ix), _p(_f64(A.values)), _p(b_ip),
                           _p(b_ix), _p(c_ip), _p(c_ix), _p(g), _p(out))
    return out


def diagonal(A):
    """The stored diagonal of A as float64 (zero where absent)."""
    rows = np.repeat(np.arange(A.m), np.diff(np.asarray(A.indptr, np.int64)))
    on = np.asarray(A.indices) == rows
    d = np.zeros(A.m)
    d[rows[on]] = np.asarray(A.values, np.float64)[on]
    return d


def tril_pattern(A):
    """(indptr, indices) of the lower triangle of A including the diagonal."""
    ip = np.asarray(A.indptr, dtype=np.int64)
    ix = np.asarray(A.indices)
    rows = np.repeat(np.arange(A.m), np.diff(ip))
    keep = ix <= rows
    counts = np.bincount(rows[keep], minlength=A.m)
    l_ip = np.zeros(A.m + 1, dtype=np.int64)
    np.cumsum(counts, out=l_ip[1:])
    return l_ip.astype(np.int32), ix[keep].astype(np.int32), keep


def ic0(A):
    """IC(0) factor values on tril(A)'s pattern: (l_indptr, l_indices, l_vals)."""
    l_ip, l_ix, _ = tril_pattern(A)
    l_v = np.empty(l_ix.size, dtype=np.float64)
    ip, ix, v = _i32(A.indptr), _i32(A.indices), _f64(A.values)
    rc = _L().orc_ic0(A.m, _p(ip), _p(ix), _p(v), _p(l_ip), _p(l_ix), _p(l_v))
    if rc != 0:
        raise ValueError("IC(0) met a non-positive pivot")
    return l_ip, l_ix, l_v


def trsv_lower(l_indptr, l_indices, l_vals, r):
    n = len(l_indptr) - 1
    y = np.empty(n)
    _L().orc_trsv_lower(n, _p(_i32(l_indptr)), _p(_i32(l_indices)), _p(_f64(l_vals)),
                        _p(_f64(r)), _p(y))
    return y


def trsv_lower_t(l_indptr, l_indices, l_vals, r):
    n = len(l_indptr) - 1
    y = np.empty(n)
    _L().orc_trsv_lower_t(n, _p(_i32(l_indptr)), _p(_i32(l_indices)), _p(_f64(l_vals)),
                          _p(_f64(r)), _p(y))
    return y


def pcg(A, b, tol=1e-8, maxit=None, pc="none", diag=None, L=None, hist=False):
    """Textbook FP64 PCG from x0 = 0 to a true relative residual <= tol.

    pc: "none" | "jacobi" | "llt" (M = L L^T, L = (indptr, indices, vals)) | "ic0"
    (M = (L L^T)^{-1}, L the IC(0) factor).  Returns (x, status, iters[, hist])."""
    n = A.m
    maxit = 10 * n if maxit is None else maxit
    kind = {"none": PC_NONE, "jacobi": PC_JACOBI, "llt": PC_LLT, "ic0": PC_IC0}[pc]
    ip, ix, v = _i32(A.indptr), _i32(A.indices), _f64(A.values)
    b = _f64(b)
    x = np.empty(n)
    d = _f64(diag) if diag is not None else None
    if kind == PC_JACOBI and d is None:
        d = diagonal(A)
    l_ip = l_ix = l_v = None
    if L is not None:
        l_ip, l_ix, l_v = _i32(L[0]), _i32(L[1]), _f64(L[2])
    it = ctypes.c_int64(0)
    h = np.zeros(maxit + 1) if hist else None
    st = _L().orc_pcg(n, _p(ip), _p(ix), _p(v), _p(b), _p(x), kind, _p(d), _p(l_ip),
                      _p(l_ix), _p(l_v), float(tol), int(maxit), ctypes.byref(it), _p(h))
    if hist:
        return x, st, it.value, h[: it.value + 1]
    return x, st, it.value


def solve_adjoint(A, x, g, tol=1e-13):
    """Sparse-solve VJP (Table 1, SpSolve): lam = A^{-T} g, grad_b = lam,
    grad_A = -(lam x^T) on mask(A).  A is taken symmetric (A^{-T} = A^{-1}, SPD)."""
    lam, st, _ = pcg(A, g, tol=tol)
    if st != 0:
        raise RuntimeError(f"adjoint CG status {STATUS_NAMES[st]}")
    ga = -sddmm(A, lam.reshape(-1, 1), np.asarray(x, np.float64).reshape(-1, 1))
    return lam, ga
