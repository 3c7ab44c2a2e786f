"""spx_spmm_t_noalloc: the transpose product for callers that cannot allocate device
memory when they call it (the library stages A^T's values in a built-in scratch array).

Checked against the FP64 oracle (A^T G) and against the workspace entry point spx_spmm_t
on two calls in a row (the shared scratch keeps the previous call's contents, which must
not leak into the next result), and the size limit is checked to fail cleanly before any
device work.  This file is
collected last so that a failure here never hides another test's result."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from helpers import REL_TOL, abs_csr, assert_close_normalised

spx = pytest.importorskip("paper_2212_05159_gb300")
from paper_2212_05159_gb300 import abi  # noqa: E402

NOALLOC_MAX_NNZ = 1 << 22


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_twice():
    import oracle
    A = synth.powerlaw_csr(60000, seed=11, max_len=3000)        # long rows, nnz ~ 0.96M
    assert A.nnz <= NOALLOC_MAX_NNZ
    dA = spx.CSR.from_host(A)
    _, _, perm = dA.transpose_pattern()
    st = dA.t_struct()
    plan = dA.t_plan()
    for call, (k, seed) in enumerate(((32, 1), (8, 2))):
        G = torch.from_numpy(synth.normal((A.m, k), seed=seed)).cuda()
        ref = torch.empty(A.n, k, device="cuda")
        ws = abi.workspace(abi.spx_spmm_t_workspace_size(st, k, plan), "cuda")
        abi.spx_spmm_t(st, perm, G, ref, 1.0, 0.0, plan, ws)
        got = torch.full((A.n, k), float("nan"), device="cuda")
        abi.spx_spmm_t_noalloc(st, perm, G, got, 1.0, 0.0, plan)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        Gh = G.cpu().numpy()
        norm = oracle.spmm_t(abs_csr(A), np.abs(Gh))
        assert_close_normalised(g, oracle.spmm_t(A, Gh), norm, rel=REL_TOL, what=f"noalloc vs oracle, call {call}")
        assert_close_normalised(g, r, norm, rel=REL_TOL, what=f"noalloc vs workspace, call {call}")
        assert np.all(np.isfinite(g))


def test_noalloc_rejects_sizes_beyond_the_scratch():
    """Too many entries: a clear error before any device work (no GPU needed)."""
    big = abi.spx_csr(10, 10, NOALLOC_MAX_NNZ + 1, 1, 1, 1)     # never dereferenced
    G = ctypes.c_void_p(16)
    rc = abi.lib().spx_spmm_t_noalloc(ctypes.byref(big), ctypes.c_void_p(16), G, 4, 4, G, 4, 1.0, 0.0,
                                      None, None)
    assert rc == 1                                              # SPX_INVALID_ARG
    assert b"exceeds the built-in scratch" in abi.lib().spx_last_error()
