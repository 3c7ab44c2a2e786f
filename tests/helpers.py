"""Shared helpers of the parity tests: tolerances and host <-> device marshalling.

The tolerance of a floating-point output is the one the FP32 kernels are held to:
|gpu - oracle| <= 1e-5 * N elementwise, where N is the same product computed by the
oracle on absolute values (|A||X| for a product, |G||X^T| on the mask for SDDMM, ...),
so that cancellation cannot make the bound vacuous or impossible.
"""
from __future__ import annotations

import numpy as np

REL_TOL = 1e-5


def abs_csr(A):
    import synth
    return synth.CSR(A.m, A.n, A.indptr, A.indices, np.abs(A.values))


def assert_close_normalised(got, ref, norm, rel=REL_TOL, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    norm = np.asarray(norm, np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    err = np.abs(got - ref)
    bound = rel * norm + 1e-30
    bad = err > bound
    if bad.any():
        i = np.flatnonzero(bad.ravel())[0]
        raise AssertionError(f"{what}: {int(bad.sum())} of {bad.size} outside 1e-5 normalised; first "
                             f"at {i}: got {got.ravel()[i]!r} ref {ref.ravel()[i]!r} "
                             f"norm {norm.ravel()[i]!r}; max ratio {float((err / bound).max()):.3g}")


def sub_rows(A, rows):
    """CSR of the selected rows of A (same column space)."""
    import synth
    rows = np.asarray(rows, np.int64)
    ip = A.indptr.astype(np.int64)
    lens = ip[rows + 1] - ip[rows]
    new_ip = np.zeros(rows.size + 1, np.int64)
    np.cumsum(lens, out=new_ip[1:])
    take = np.concatenate([np.arange(ip[r], ip[r + 1]) for r in rows]) if rows.size else \
        np.zeros(0, np.int64)
    return synth.CSR(rows.size, A.n, new_ip, A.indices[take], A.values[take]), take
