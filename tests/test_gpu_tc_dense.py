"""The network's dense layer on the tensor cores (tcgen05 + TMEM) against the FP32-activation
kernel fed the same BF16-rounded activations: only the FP32 accumulation order differs."""
import numpy as np
import pytest
import torch

from helpers import assert_close_normalised

pytestmark = pytest.mark.gpu
spx = pytest.importorskip("paper_2212_05159_gb300")
from paper_2212_05159_gb300 import abi  # noqa: E402


def _bf16(t):
    return t.to(torch.bfloat16).to(torch.float32)


@pytest.mark.parametrize("n", [1, 127, 300, 4096])
@pytest.mark.parametrize("K1,K2,N,mode", [(4, 0, 64, 1), (64, 64, 64, 2), (64, 0, 64, 0), (64, 0, 128, 0),
                                           (32, 16, 32, 1)])
def test_tc_dense_matches_fp32_kernel(n, K1, K2, N, mode):
    g = torch.Generator().manual_seed(n * 1000 + K1 + K2 + N + mode)
    X1 = torch.randn(n, K1, generator=g).cuda()
    X2 = torch.randn(n, K2, generator=g).cuda() if K2 else None
    W = (torch.randn(K1 + K2, N, generator=g) * 0.2).to(torch.bfloat16).cuda()
    b = torch.randn(N, generator=g).cuda()
    Hin = torch.randn(n, N, generator=g).cuda() if mode == 2 else None
    Y = torch.full((n, N), float("nan"), device="cuda")
    U = torch.full((n, N), float("nan"), device="cuda") if mode == 2 else None
    abi.spx_dense_forward_tc(n, X1, K1, X2, K2, W, b, N, mode, Hin, Y, U)
    abi.spx_check_device()
    Yr = torch.empty(n, N, device="cuda")
    Ur = torch.empty(n, N, device="cuda") if mode == 2 else None
    abi.spx_dense_forward(n, _bf16(X1), K1, _bf16(X2) if K2 else None, K2, W, b, N, mode, Hin, Yr, Ur)
    torch.cuda.synchronize()
    Xc = torch.cat([_bf16(X1), _bf16(X2)], 1) if K2 else _bf16(X1)
    norm = (Xc.abs().double() @ W.float().abs().double() + b.abs().double()).cpu().numpy()
    if mode == 2:
        assert_close_normalised(U.cpu().numpy(), Ur.cpu().numpy(), norm, what="tc pre-activation")
        norm = norm + Hin.abs().double().cpu().numpy()
    assert_close_normalised(Y.cpu().numpy(), Yr.cpu().numpy(), norm, what=f"tc dense n={n} K={K1}+{K2}")


def test_tc_network_forward_close_to_fp32_path():
    import synth
    from paper_2212_05159_gb300 import learned
    A, ptr, _, _ = synth.diffusion_batch(4, seed=3, side_lo=20, side_hi=40, sigma=1.0)
    net = learned.MPNN(seed=0)
    rng = np.random.default_rng(0)
    p = net.get_params()
    p["v"] = rng.normal(0, 0.3, p["v"].shape).astype(np.float32)
    net.set_params(p)
    G = learned.Graph(spx.CSR.from_host(A))
    L32, _ = net.forward(G)
    Ltc, _ = net.forward(G, tensor_cores=True)
    a, t = L32.cpu().numpy(), Ltc.cpu().numpy()
    # BF16 activations: agreement to a few BF16 ulps of the output scale
    assert np.abs(a - t).max() <= 3e-2 * np.abs(a).max()
