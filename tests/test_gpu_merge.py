"""Merge-path SpMM and SDDMM (spx_spmm_merge, spx_sddmm_merge) against the FP64 oracle:
power-law rows, empty rows and a hub row, rectangular matrices, the 2D Poisson stencil,
segment sizes from 1 item (every row cut, carries everywhere) to one segment for the
whole matrix, every supported width k, alpha / beta, and the transpose product through
the permutation."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import REL_TOL, abs_csr, assert_close_normalised

pytestmark = pytest.mark.gpu
spx = pytest.importorskip("paper_2212_05159_gb300")
from paper_2212_05159_gb300 import abi  # noqa: E402


def _mats():
    return {
        "powerlaw": synth.powerlaw_csr(6000, seed=5, max_len=1500),
        "ragged": synth.empty_rows_csr(900, 700, seed=2),
        "rect": synth.random_k_per_row(500, 7, seed=3, ncols=1300),
        "poisson": synth.poisson2d(24),
    }


def _items_list(A):
    tot = A.m + A.nnz
    return [1, 3, 17, 256, tot + 5]


@pytest.mark.parametrize("name", ["powerlaw", "ragged", "rect", "poisson"])
@pytest.mark.parametrize("k", [4, 8, 16, 32, 64, 128])
def test_spmm_merge_matches_oracle(name, k):
    A = _mats()[name]
    dA = spx.CSR.from_host(A)
    X = synth.normal((A.n, k), seed=k)
    Y0 = synth.normal((A.m, k), seed=k + 1)
    ref = oracle.spmm(A, X)
    norm = oracle.spmm(abs_csr(A), np.abs(X))
    Xd = torch.from_numpy(X).cuda()
    for items in _items_list(A):
        plan = dA.merge_plan(items)
        ws = abi.workspace(abi.spx_spmm_merge_workspace_size(dA.struct(), k, plan), "cuda")
        for variant in (0, 1, 2):
            Y = torch.full((A.m, k), float("nan"), device="cuda")
            abi.spx_spmm_merge(dA.struct(), Xd, Y, plan, ws, variant=variant)
            assert_close_normalised(Y.cpu().numpy(), ref, norm, what=f"{name} k={k} items={items} v={variant}")
        # alpha, beta with a prior Y
        Y = torch.from_numpy(Y0).cuda()
        abi.spx_spmm_merge(dA.struct(), Xd, Y, plan, ws, alpha=0.5, beta=-2.0)
        assert_close_normalised(Y.cpu().numpy(), 0.5 * ref - 2.0 * Y0, 0.5 * norm + 2.0 * np.abs(Y0),
                                what=f"{name} k={k} items={items} alpha/beta")


@pytest.mark.parametrize("name", ["powerlaw", "ragged", "rect"])
@pytest.mark.parametrize("k", [8, 32, 128])
def test_spmm_merge_transpose_through_permutation(name, k):
    """gX = A^T G on A^T's pattern with A's values read through the permutation."""
    A = _mats()[name]
    dA = spx.CSR.from_host(A)
    t_ip, t_ix, perm = dA.transpose_pattern()
    G = synth.normal((A.m, k), seed=7)
    ref = oracle.spmm_t(A, G)
    norm = oracle.spmm_t(abs_csr(A), np.abs(G))
    st = abi.csr_struct(A.n, A.m, t_ip, t_ix, dA.values)
    for items in (5, 200):
        plan = dA.t_merge_plan(items)
        ws = abi.workspace(abi.spx_spmm_merge_workspace_size(st, k, plan), "cuda")
        gX = torch.full((A.n, k), float("nan"), device="cuda")
        abi.spx_spmm_merge(st, torch.from_numpy(G).cuda(), gX, plan, ws, perm=perm)
        assert_close_normalised(gX.cpu().numpy(), ref, norm, what=f"{name} A^T G k={k} items={items}")


@pytest.mark.parametrize("name", ["powerlaw", "ragged", "rect", "poisson"])
@pytest.mark.parametrize("k", [4, 8, 16, 32, 64, 128])
def test_sddmm_merge_matches_oracle(name, k):
    A = _mats()[name]
    dA = spx.CSR.from_host(A)
    G = synth.normal((A.m, k), seed=k + 3)
    X = synth.normal((A.n, k), seed=k + 4)
    ref = oracle.sddmm(A, G, X)
    norm = oracle.sddmm(A, np.abs(G), np.abs(X))
    Gd, Xd = torch.from_numpy(G).cuda(), torch.from_numpy(X).cuda()
    for items in _items_list(A):
        plan = dA.merge_plan(items)
        for variant in (0, 1, 2):
            out = torch.full((A.nnz,), float("nan"), device="cuda")
            abi.spx_sddmm_merge(dA.struct(), Gd, Xd, out, plan, scale=-1.5, variant=variant)
            assert_close_normalised(out.cpu().numpy(), -1.5 * ref, 1.5 * norm,
                                    what=f"{name} k={k} items={items} v={variant}")


def test_merge_products_are_deterministic_and_handle_degenerate_shapes():
    A = synth.powerlaw_csr(5000, seed=9, max_len=2000)
    dA = spx.CSR.from_host(A)
    k = 32
    X = torch.from_numpy(synth.normal((A.n, k), seed=1)).cuda()
    plan = dA.merge_plan(64)
    ws = abi.workspace(abi.spx_spmm_merge_workspace_size(dA.struct(), k, plan), "cuda")
    outs = []
    for _ in range(3):
        Y = torch.empty(A.m, k, device="cuda")
        abi.spx_spmm_merge(dA.struct(), X, Y, plan, ws)
        outs.append(Y.cpu())
    assert all(torch.equal(outs[0], o) for o in outs[1:])
    # every row empty: Y = beta Y; one row; one column
    for B in (synth.CSR(7, 5, np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32)),
              synth.random_k_per_row(1, 3, seed=1, ncols=40),
              synth.random_k_per_row(30, 1, seed=2, ncols=1)):
        dB = spx.CSR.from_host(B)
        Xb = synth.normal((B.n, 8), seed=3)
        Yb0 = synth.normal((B.m, 8), seed=4)
        for items in (1, 4, 1000):
            pb = dB.merge_plan(items)
            wb = abi.workspace(abi.spx_spmm_merge_workspace_size(dB.struct(), 8, pb), "cuda")
            Yb = torch.from_numpy(Yb0).cuda()
            abi.spx_spmm_merge(dB.struct(), torch.from_numpy(Xb).cuda(), Yb, pb, wb, alpha=2.0, beta=0.5)
            ref = 2.0 * oracle.spmm(B, Xb) + 0.5 * Yb0
            norm = 2.0 * oracle.spmm(abs_csr(B), np.abs(Xb)) + 0.5 * np.abs(Yb0)
            assert_close_normalised(Yb.cpu().numpy(), ref, norm, rel=REL_TOL, what=f"degenerate {B.m}x{B.n} {items}")


def test_merge_entry_points_reject_bad_arguments():
    A = synth.poisson2d(8)
    dA = spx.CSR.from_host(A)
    X = torch.zeros(A.n, 12, device="cuda")
    Y = torch.zeros(A.m, 12, device="cuda")
    plan = dA.merge_plan(16)
    ws = abi.workspace(1 << 16, "cuda")
    with pytest.raises(abi.SpxError):                       # k = 12 is not a supported width
        abi.spx_spmm_merge(dA.struct(), X, Y, plan, ws)
    X8, Y8 = X[:, :8].contiguous(), Y[:, :8].contiguous()
    other = dA.merge_plan(17)                               # plan of another segment size, mislabelled
    bad = abi.spx_mergeplan(other.seg_row, other.n_segments, 16)
    with pytest.raises(abi.SpxError):
        abi.spx_spmm_merge(dA.struct(), X8, Y8, bad, ws)
    with pytest.raises(abi.SpxError):                       # workspace too small
        abi.spx_spmm_merge(dA.struct(), X8, Y8, plan, ws[:32])
    abi.spx_check_device()
