"""Both gradients of Y = A X in one pass over A^T (spx_spmm_t_sddmm) against the FP64 oracle:
gX = alpha A^T G + beta gX and gA = scale (G X^T) on A's pattern, on power-law rows (long
and medium rows of A^T), empty rows and a hub row, a rectangular matrix and the 2D Poisson
stencil, every supported width class (k = 4 .. 128), with and without the row plan of A^T,
deterministic, and the unsupported widths rejected."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import abs_csr, assert_close_normalised

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


@pytest.mark.parametrize("name", ["powerlaw", "ragged", "rect", "poisson"])
@pytest.mark.parametrize("k", [4, 12, 32, 64, 100, 128])
@pytest.mark.parametrize("use_plan,variant", [(True, 0), (False, 0), (True, 1), (True, 2), (False, 3),
                                              (True, 4), (False, 5)])
def test_fused_backward_matches_oracle(name, k, use_plan, variant):
    A = _mats()[name]
    dA = spx.CSR.from_host(A)
    t_ip, t_ix, perm = dA.transpose_pattern()
    AT = abi.csr_struct(A.n, A.m, t_ip, t_ix, dA.values)
    G = synth.normal((A.m, k), seed=k + 1)
    X = synth.normal((A.n, k), seed=k + 2)
    gX0 = synth.normal((A.n, k), seed=k + 3)
    Gd, Xd = torch.from_numpy(G).cuda(), torch.from_numpy(X).cuda()
    gX = torch.from_numpy(gX0).cuda()
    gA = torch.full((A.nnz,), float("nan"), device="cuda")
    plan = dA.t_plan() if use_plan else None
    abi.spx_spmm_t_sddmm(AT, perm, dA.values, Gd, Xd, gX, gA, alpha=0.5, beta=-1.5, scale=-2.0, plan=plan,
                         variant=variant)
    abi.spx_check_device()
    ref_x = 0.5 * oracle.spmm_t(A, G) - 1.5 * gX0
    norm_x = 0.5 * oracle.spmm_t(abs_csr(A), np.abs(G)) + 1.5 * np.abs(gX0)
    assert_close_normalised(gX.cpu().numpy(), ref_x, norm_x, what=f"{name} k={k} gX")
    ref_a = -2.0 * oracle.sddmm(A, G, X)
    norm_a = 2.0 * oracle.sddmm(A, np.abs(G), np.abs(X))
    assert_close_normalised(gA.cpu().numpy(), ref_a, norm_a, what=f"{name} k={k} gA")


def test_fused_backward_is_deterministic_and_handles_degenerate_shapes():
    A = synth.powerlaw_csr(5000, seed=9, max_len=2000)
    dA = spx.CSR.from_host(A)
    t_ip, t_ix, perm = dA.transpose_pattern()
    AT = abi.csr_struct(A.n, A.m, t_ip, t_ix, dA.values)
    k = 32
    G = torch.from_numpy(synth.normal((A.m, k), seed=1)).cuda()
    X = torch.from_numpy(synth.normal((A.n, k), seed=2)).cuda()
    outs = []
    for variant in (0, 0, 1, 2, 3, 4, 5):
        gX, gA = torch.empty(A.n, k, device="cuda"), torch.empty(A.nnz, device="cuda")
        abi.spx_spmm_t_sddmm(AT, perm, dA.values, G, X, gX, gA, plan=dA.t_plan(), variant=variant)
        outs.append((gX.cpu(), gA.cpu()))
    # the launch shapes do the same arithmetic in the same order
    assert all(torch.equal(outs[0][0], o[0]) and torch.equal(outs[0][1], o[1]) for o in outs[1:])
    # no entries: gX = beta gX; one row; one column
    for B in (synth.CSR(7, 5, np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32)),
              synth.random_k_per_row(1, 3, seed=1, ncols=40),
              synth.random_k_per_row(30, 1, seed=2, ncols=1)):
        dB = spx.CSR.from_host(B)
        bt_ip, bt_ix, bperm = dB.transpose_pattern()
        BT = abi.csr_struct(B.n, B.m, bt_ip, bt_ix, dB.values)
        Gb, Xb, gX0 = synth.normal((B.m, 8), seed=3), synth.normal((B.n, 8), seed=4), synth.normal((B.n, 8), seed=5)
        gX = torch.from_numpy(gX0).cuda()
        gA = torch.full((max(B.nnz, 1),), float("nan"), device="cuda")
        abi.spx_spmm_t_sddmm(BT, bperm, dB.values, torch.from_numpy(Gb).cuda(), torch.from_numpy(Xb).cuda(), gX,
                             gA, alpha=2.0, beta=0.5)
        assert_close_normalised(gX.cpu().numpy(), 2.0 * oracle.spmm_t(B, Gb) + 0.5 * gX0,
                                2.0 * oracle.spmm_t(abs_csr(B), np.abs(Gb)) + 0.5 * np.abs(gX0),
                                what=f"degenerate {B.m}x{B.n} gX")
        if B.nnz:
            assert_close_normalised(gA.cpu().numpy()[: B.nnz], oracle.sddmm(B, Gb, Xb),
                                    oracle.sddmm(B, np.abs(Gb), np.abs(Xb)), what=f"degenerate {B.m}x{B.n} gA")
    abi.spx_check_device()


def test_fused_backward_rejects_unsupported_widths_and_layouts():
    A = synth.poisson2d(8)
    dA = spx.CSR.from_host(A)
    t_ip, t_ix, perm = dA.transpose_pattern()
    AT = abi.csr_struct(A.n, A.m, t_ip, t_ix, dA.values)
    gA = torch.zeros(A.nnz, device="cuda")
    for k in (6, 132):
        G, X, gX = (torch.zeros(A.m, k, device="cuda") for _ in range(3))
        with pytest.raises(abi.SpxError):
            abi.spx_spmm_t_sddmm(AT, perm, dA.values, G, X, gX, gA)
    buf = torch.zeros(A.m * 8 + 1, device="cuda")
    G_bad = buf[1:].view(A.m, 8)                           # 4-byte offset: not 16-byte aligned
    X, gX = torch.zeros(A.n, 8, device="cuda"), torch.zeros(A.n, 8, device="cuda")
    with pytest.raises(abi.SpxError):
        abi.spx_spmm_t_sddmm(AT, perm, dA.values, G_bad, X, gX, gA)
    abi.spx_check_device()
