"""The network's dense layers on the tensor cores (tcgen05 + TMEM) against plain FP64 CPU
products of the same BF16-rounded operands (the BF16 products are exact in FP32, so only
the rounding of the FP32 sums differs), at the 1e-5 normalised bar of every other kernel.
The whole network on the tensor cores is checked against the oracle in test_gpu_learned."""
import numpy as np
import pytest
import torch

from helpers import assert_close_normalised

pytestmark = pytest.mark.gpu
spx = pytest.importorskip("paper_2212_05159_gb300")
from paper_2212_05159_gb300 import abi  # noqa: E402


def _bf16(t):
    return t.to(torch.bfloat16).to(torch.float32)


def _cpu(t):
    return t.detach().cpu().double()


@pytest.mark.parametrize("n", [1, 127, 300, 4096, 50003])
@pytest.mark.parametrize("K1,K2,N,mode,hin_is_x1", [
    (4, 0, 64, 1, False), (64, 64, 64, 2, False), (64, 0, 64, 0, False), (64, 0, 128, 0, False),
    (32, 16, 32, 1, False), (12, 8, 16, 1, False), (60, 68, 128, 0, False), (64, 64, 64, 3, False),
    (64, 0, 128, 4, False), (32, 0, 32, 4, False),
    # the network's residual layer (Hin is X1), on the pipelined kernel, and other pipelined shapes
    (64, 64, 64, 3, True), (64, 64, 64, 2, True), (32, 32, 32, 3, True), (96, 32, 96, 1, False),
    (32, 0, 64, 4, False), (128, 0, 128, 2, True)])
def test_tc_dense_matches_fp64_product(n, K1, K2, N, mode, hin_is_x1):
    """Y = [X1 X2] W + b (mode 0), relu of it (1), U = pre-activation and Y = Hin + relu(U)
    (2), the same Y without U (3), or the column halves of the pre-activation to Y and U (4),
    with X rounded to BF16, against the FP64 product of the rounded X and the BF16 W;
    normaliser |X||W| + |b| (+ |Hin|).  n = 50003 gives every CTA of the pipelined kernel
    several tiles (each stage, operand buffer and accumulator reused, a ragged last tile)."""
    if n == 50003 and (K1 % 32 or K2 % 32 or N % 32):
        pytest.skip("the large case is for the pipelined shapes")
    g = torch.Generator().manual_seed(n * 1000 + K1 + K2 + N + mode)
    X1 = torch.randn(n, K1, generator=g).cuda()
    X2 = torch.randn(n, K2, generator=g).cuda() if K2 else None
    W = (torch.randn(K1 + K2, N, generator=g) * 0.2).to(torch.bfloat16).cuda()
    b = torch.randn(N, generator=g).cuda()
    Hin = (X1 if hin_is_x1 else torch.randn(n, N, generator=g).cuda()) if mode in (2, 3) else None
    Y = torch.full((n, N // 2 if mode == 4 else N), float("nan"), device="cuda")
    U = torch.full((n, N // 2 if mode == 4 else N), float("nan"), device="cuda") if mode in (2, 4) else None
    abi.spx_dense_forward_tc(n, X1, K1, X2, K2, W, b, N, mode, Hin, Y, U)
    abi.spx_check_device()
    Xr = torch.cat([_cpu(_bf16(X1)), _cpu(_bf16(X2))], 1) if K2 else _cpu(_bf16(X1))
    Wd, bd = _cpu(W), _cpu(b)
    pre = Xr @ Wd + bd
    norm = (Xr.abs() @ Wd.abs() + bd.abs()).numpy()
    if mode == 0:
        ref = pre
    elif mode == 1:
        ref = torch.relu(pre)
    elif mode == 4:
        h2 = N // 2
        assert_close_normalised(U.cpu().numpy(), pre[:, h2:].numpy(), norm[:, h2:], what="tc second half")
        ref, norm = pre[:, :h2], norm[:, :h2]
    else:
        if mode == 2:
            assert_close_normalised(U.cpu().numpy(), pre.numpy(), norm, what="tc pre-activation")
        ref = _cpu(Hin) + torch.relu(pre)
        norm = norm + _cpu(Hin).abs().numpy()
    assert_close_normalised(Y.cpu().numpy(), ref.numpy(), norm, what=f"tc dense n={n} K={K1}+{K2} mode={mode}")


@pytest.mark.parametrize("n", [1, 127, 300, 4096, 50003])
@pytest.mark.parametrize("N,K1,K2,acc", [(64, 64, 64, 1), (64, 64, 0, 0), (64, 64, 0, 1), (32, 16, 16, 0),
                                         (128, 64, 0, 0), (64, 4, 0, 0), (4, 16, 0, 0), (20, 8, 12, 1),
                                         (128, 60, 68, 1), (64, 64, 64, 0), (32, 96, 32, 1), (128, 32, 0, 1)])
def test_tc_backward_data_matches_fp64_product(n, N, K1, K2, acc):
    """[dX1 dX2] (+)= G W^T on the tensor cores, G rounded to BF16, against the FP64
    product of the rounded G and the BF16 W (plus the initial dX when accumulating)."""
    if n == 50003 and (N % 32 or K1 % 32 or K2 % 32):
        pytest.skip("the large case is for the pipelined shapes")
    g = torch.Generator().manual_seed(n * 7 + N + K1 + K2 + acc)
    G = torch.randn(n, N, generator=g).cuda()
    W = (torch.randn(K1 + K2, N, generator=g) * 0.2).to(torch.bfloat16).cuda()
    d1 = torch.randn(n, K1, generator=g).cuda()
    d2 = torch.randn(n, K2, generator=g).cuda() if K2 else None
    init = torch.cat([_cpu(d1), _cpu(d2)], 1) if K2 else _cpu(d1)
    abi.spx_dense_backward_data_tc(n, G, N, W, K1, K2, d1, d2, acc)
    abi.spx_check_device()
    Gr, Wd = _cpu(_bf16(G)), _cpu(W)
    ref = Gr @ Wd.t()
    norm = Gr.abs() @ Wd.abs().t()
    if acc:
        ref = ref + init
        norm = norm + init.abs()
    got = torch.cat([d1, d2], 1) if K2 else d1
    assert_close_normalised(got.cpu().numpy(), ref.numpy(), norm.numpy(), what=f"tc dX n={n} N={N} K={K1}+{K2}")


@pytest.mark.parametrize("n", [1, 127, 300, 4096, 100003])
@pytest.mark.parametrize("K1,K2,N,with_db", [(64, 64, 64, True), (64, 0, 64, False), (4, 0, 64, True),
                                             (16, 16, 32, True), (60, 0, 16, True), (64, 64, 128, False)])
def test_tc_backward_weight_matches_fp64_product(n, K1, K2, N, with_db):
    """dW = [X1 X2]^T G on the tensor cores against an FP64 product of the BF16-rounded X and G
    (the BF16 products are exact in FP32; only the rounding of the sums differs); db against
    the FP64 column sums of the unrounded G.  n = 100003 gives every CTA several row tiles,
    so both staging buffers are reused."""
    g = torch.Generator().manual_seed(n + 3 * K1 + 5 * K2 + N)
    X1 = torch.randn(n, K1, generator=g).cuda()
    X2 = torch.randn(n, K2, generator=g).cuda() if K2 else None
    G = torch.randn(n, N, generator=g).cuda()
    K = K1 + K2
    dW = torch.full((K, N), float("nan"), device="cuda")
    db = torch.full((N,), float("nan"), device="cuda") if with_db else None
    ws = abi.workspace(abi._size("spx_dense_backward_weight_tc_workspace_size", n, K, N), "cuda")
    abi.spx_dense_backward_weight_tc(n, X1, K1, X2, K2, G, N, dW, db, ws)
    abi.spx_check_device()
    X1r, Gr = _bf16(X1).cpu().double(), _bf16(G).cpu().double()
    Xr = torch.cat([X1r, _bf16(X2).cpu().double()], 1) if K2 else X1r
    dWr = (Xr.t() @ Gr).numpy()
    norm = (Xr.abs().t() @ Gr.abs()).numpy()
    assert_close_normalised(dW.cpu().numpy(), dWr, norm, what=f"tc dW n={n} K={K1}+{K2} N={N}")
    if with_db:
        Gd = G.double()
        assert_close_normalised(db.cpu().numpy(), Gd.sum(0).cpu().numpy(), Gd.abs().sum(0).cpu().numpy(),
                                what="tc db")


def test_tc_backward_weight_is_deterministic():
    g = torch.Generator().manual_seed(9)
    n, K, N = 50000, 128, 64
    X = torch.randn(n, K, generator=g).cuda()
    G = torch.randn(n, N, generator=g).cuda()
    ws = abi.workspace(abi._size("spx_dense_backward_weight_tc_workspace_size", n, K, N), "cuda")
    outs = []
    for _ in range(3):
        dW, db = torch.empty(K, N, device="cuda"), torch.empty(N, device="cuda")
        abi.spx_dense_backward_weight_tc(n, X, K, None, 0, G, N, dW, db, ws)
        outs.append((dW.cpu(), db.cpu()))
    for dW, db in outs[1:]:
        assert torch.equal(dW, outs[0][0]) and torch.equal(db, outs[0][1])


def test_tc_backward_weight_rejects_bad_sizes():
    ws = abi.workspace(1 << 20, "cuda")
    X = torch.zeros(8, 8, device="cuda")
    Gm = torch.zeros(8, 48, device="cuda")
    dW = torch.zeros(8, 48, device="cuda")
    with pytest.raises(abi.SpxError):
        abi.spx_dense_backward_weight_tc(8, X, 8, None, 0, Gm, 48, dW, None, ws)      # N not a power of two
    with pytest.raises(abi.SpxError):
        abi.spx_dense_backward_weight_tc(8, X, 6, None, 0, Gm[:, :16], 16, dW, None, ws)  # K1 % 4


def test_tc_kernels_reject_unaligned_or_unsupported_operands():
    """The tensor-core entry points check their layout before any launch: rows that do not
    start on 16 bytes, and sizes outside the supported tiles, are argument errors."""
    n, K, N = 64, 64, 64
    buf = torch.zeros(n * K + 1, device="cuda")
    X_bad = buf[1:].view(n, K)                       # 4-byte offset: not 16-byte aligned
    X = torch.zeros(n, K, device="cuda")
    G = torch.zeros(n, N, device="cuda")
    W = torch.zeros(K, N, dtype=torch.bfloat16, device="cuda")
    Y = torch.zeros(n, N, device="cuda")
    dX = torch.zeros(n, K, device="cuda")
    with pytest.raises(abi.SpxError):
        abi.spx_dense_forward_tc(n, X_bad, K, None, 0, W, None, N, 0, None, Y, None)
    with pytest.raises(abi.SpxError):
        abi.spx_dense_forward_tc(n, X, K, None, 0, W, None, 40, 0, None, Y, None)      # N % 16
    with pytest.raises(abi.SpxError):
        abi.spx_dense_backward_data_tc(n, G, N, W, K, 0, X_bad, None, 0)
    with pytest.raises(abi.SpxError):
        abi.spx_dense_backward_data_tc(n, G, N, W, 6, 0, dX, None, 0)                 # K1 % 4
    ws = abi.workspace(abi._size("spx_dense_backward_weight_tc_workspace_size", n, K, N), "cuda")
    dW = torch.zeros(K, N, device="cuda")
    with pytest.raises(abi.SpxError):
        abi.spx_dense_backward_weight_tc(n, X_bad, K, None, 0, G, N, dW, None, ws)
    with pytest.raises(abi.SpxError):
        abi.spx_dense_backward_weight_tc(n, X, K, None, 0, G, N, dW, None, ws[:16])   # workspace too small
    abi.spx_check_device()


@pytest.mark.parametrize("n", [1, 300, 50003])
def test_tc_pipelined_kernel_equals_the_staged_kernel_bitwise(n):
    """The pipelined kernel (TMA ring, warp roles) and the stage-multiply-store kernel do the
    same arithmetic: every forward mode and the data gradient, plain and accumulating, give
    the same bits with the pipeline on and off."""
    g = torch.Generator().manual_seed(n + 17)
    H = 64
    h = torch.randn(n, H, generator=g).cuda()
    m = torch.randn(n, H, generator=g).cuda()
    W = (torch.randn(2 * H, H, generator=g) * 0.2).to(torch.bfloat16).cuda()
    Wh = (torch.randn(H, 2 * H, generator=g) * 0.2).to(torch.bfloat16).cuda()
    b = torch.randn(H, generator=g).cuda()
    G = torch.randn(n, H, generator=g).cuda()
    init1, init2 = torch.randn(n, H, generator=g).cuda(), torch.randn(n, H, generator=g).cuda()

    def run():
        out = []
        for mode in (0, 1, 2, 3):
            Y, U = torch.empty(n, H, device="cuda"), torch.empty(n, H, device="cuda")
            abi.spx_dense_forward_tc(n, h, H, m, H, W, b, H, mode, h, Y, U if mode == 2 else None)
            out += [Y.clone()] + ([U.clone()] if mode == 2 else [])
        P, Q = torch.empty(n, H, device="cuda"), torch.empty(n, H, device="cuda")
        abi.spx_dense_forward_tc(n, h, H, None, 0, Wh, None, 2 * H, 4, None, P, Q)
        out += [P, Q]
        for acc in (0, 1):
            d1, d2 = init1.clone(), init2.clone()
            abi.spx_dense_backward_data_tc(n, G, H, W, H, H, d1, d2, acc)
            out += [d1, d2]
        torch.cuda.synchronize()
        return [t.cpu() for t in out]

    try:
        abi.spx_tc_set_pipeline(True)
        on = run()
        abi.spx_tc_set_pipeline(False)
        off = run()
    finally:
        abi.spx_tc_set_pipeline(True)
    abi.spx_check_device()
    for i, (a, c) in enumerate(zip(on, off)):
        assert torch.equal(a.view(torch.int32), c.view(torch.int32)), i
