"""GPU parity of the optimiser step that trains the learned preconditioner's network
(spx_adam_step: Adam as Kingma and Ba define it, the paper's optimiser in Sections 4.1 and
4.5) against the FP64 oracle, step by step, and of the BF16 weight copy it refreshes.

Tolerance: the kernel rounds each float32 operation once (relative 2^-24) and receives the
bias corrections rounded once from double; one step's update carries under ten such
roundings and the moments one or two per step, so after the at most eight steps run here
every quantity stays within about 1e-6 of its absolute form (parameters: |theta0| plus the
summed |updates|; m: the recurrence over |g|; v: itself), under the 1e-5 normalised bar.
Starting from theta0 = 0 makes the parameter check a check of the updates themselves."""
import numpy as np
import pytest
import torch

from helpers import assert_close_normalised
from oracle import adam as oadam
from oracle import mpnn as ompnn

pytestmark = pytest.mark.gpu
spx = pytest.importorskip("paper_2212_05159_gb300")
from paper_2212_05159_gb300 import abi  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _f32(x):
    return float(np.float32(x))


def _grads(count, steps, seed):
    """Gradients of changing scale (1e-6 .. 1e2), with exact zeros and sign flips mixed in."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(steps):
        g = rng.normal(0, 1, count) * np.exp(rng.uniform(np.log(1e-6), np.log(1e2), count))
        g[rng.random(count) < 0.02] = 0.0
        if t % 3 == 2:
            g = -g
        out.append(g.astype(np.float32))
    return out


@pytest.mark.parametrize("count,lr,b1,b2,eps,zero_start,steps", [
    (10007, 1e-3, 0.9, 0.999, 1e-8, False, 8),
    (10007, 1e-3, 0.9, 0.999, 1e-8, True, 8),
    (1, 0.05, 0.8, 0.99, 1e-3, False, 5),
    (333333, 3e-3, 0.9, 0.999, 1e-8, True, 4),
])
def test_adam_steps_match_oracle(count, lr, b1, b2, eps, zero_start, steps):
    lr, b1, b2, eps = _f32(lr), _f32(b1), _f32(b2), _f32(eps)     # the values the kernel receives
    rng = np.random.default_rng(count)
    theta0 = np.zeros(count, np.float32) if zero_start else rng.uniform(-1, 1, count).astype(np.float32)
    grads = _grads(count, steps, seed=count + 1)
    ref = oadam.adam(theta0, grads, lr, b1, b2, eps)
    mag = oadam.adam(theta0, grads, lr, b1, b2, eps, absolute=True)
    p, m, v = dev(theta0), torch.zeros(count, device="cuda"), torch.zeros(count, device="cuda")
    p16 = torch.empty(count, dtype=torch.bfloat16, device="cuda")
    for t, g in enumerate(grads, start=1):
        abi.spx_adam_step(p, dev(g), m, v, t, lr, b1, b2, eps, p16)
        assert_close_normalised(host(p), ref[t - 1][0], mag[t - 1][0], what=f"theta after step {t}")
        assert_close_normalised(host(m), ref[t - 1][1], mag[t - 1][1], what=f"m after step {t}")
        assert_close_normalised(host(v), ref[t - 1][2], ref[t - 1][2], what=f"v after step {t}")
        want16 = ompnn.bf16_round(torch.from_numpy(host(p).astype(np.float64)))
        assert torch.equal(p16.cpu().to(torch.float64), want16), f"BF16 copy after step {t}"


def test_to_bf16_rounds_to_nearest_even():
    rng = np.random.default_rng(11)
    ties = 1.0 + (2 * np.arange(40) + 1) * 2.0 ** -8          # halfway between two BF16 values
    x = np.concatenate([rng.normal(0, 1, 70001), rng.normal(0, 1e-30, 500), rng.normal(0, 1e30, 500),
                        ties, -ties, [0.0, -0.0, 1.0, 2.0 ** -126, 3.0e38]]).astype(np.float32)
    dst = torch.empty(x.size, dtype=torch.bfloat16, device="cuda")
    abi.spx_to_bf16(dev(x), dst)
    want = ompnn.bf16_round(torch.from_numpy(x.astype(np.float64)))
    assert torch.equal(dst.cpu().to(torch.float64), want)


def test_adam_rejects_bad_arguments():
    p = torch.zeros(4, device="cuda")
    with pytest.raises(abi.SpxError):
        abi.spx_adam_step(p, p.clone(), p.clone(), p.clone(), 0, 1e-3)      # step numbers start at 1
    empty = torch.zeros(0, device="cuda")
    abi.spx_adam_step(empty, empty, empty, empty, 1, 1e-3)                 # nothing to do
