"""Pins of the Adam oracle (Kingma and Ba, Algorithm 1; the paper's optimiser in Sections
4.1 and 4.5) against things other than itself: torch.optim.Adam in float64 (an independent
implementation of the same definition), the closed form of a constant gradient (every step
moves exactly lr sign(g) when eps = 0), the first step's closed form with eps, and the
invariance of the eps = 0 trajectory to a positive scaling of all gradients."""
import numpy as np
import torch

from oracle import adam as oadam


def _grads(n, steps, seed):
    rng = np.random.default_rng(seed)
    return [rng.normal(0, 1, n) * rng.uniform(0.1, 10) for _ in range(steps)]


def test_matches_torch_adam_in_float64():
    rng = np.random.default_rng(0)
    theta0 = rng.uniform(-1, 1, 257)
    grads = _grads(257, 12, seed=1)
    for lr, b1, b2, eps in [(1e-3, 0.9, 0.999, 1e-8), (0.05, 0.8, 0.99, 1e-3)]:
        got = oadam.adam(theta0, grads, lr, b1, b2, eps)
        mags = oadam.adam(theta0, grads, lr, b1, b2, eps, absolute=True)
        p = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
        opt = torch.optim.Adam([p], lr=lr, betas=(b1, b2), eps=eps)
        for t, g in enumerate(grads):
            p.grad = torch.tensor(g, dtype=torch.float64)
            opt.step()
            st = opt.state[p]
            # torch forms m by interpolation (another rounding order): compare at the scale of
            # each quantity's absolute form
            assert np.all(np.abs(got[t][0] - p.detach().numpy()) <= 1e-13 * mags[t][0])
            assert np.all(np.abs(got[t][1] - st["exp_avg"].numpy()) <= 1e-13 * mags[t][1])
            np.testing.assert_allclose(got[t][2], st["exp_avg_sq"].numpy(), rtol=1e-13, atol=0)


def test_constant_gradient_moves_lr_sign_g_per_step():
    """m_t = (1 - beta1^t) g and v_t = (1 - beta2^t) g^2, so with eps = 0 each bias-corrected
    step is lr g / |g|: theta_t = theta0 - t lr sign(g)."""
    rng = np.random.default_rng(2)
    theta0 = rng.uniform(-1, 1, 64)
    g = rng.normal(0, 1, 64) * np.exp(rng.uniform(-5, 5, 64))
    lr = 0.01
    out = oadam.adam(theta0, [g] * 9, lr, 0.9, 0.999, eps=0.0)
    for t, (theta, m, v) in enumerate(out, start=1):
        np.testing.assert_allclose(theta, theta0 - t * lr * np.sign(g), rtol=0, atol=1e-14)
        np.testing.assert_allclose(m, (1 - 0.9 ** t) * g, rtol=1e-14)
        np.testing.assert_allclose(v, (1 - 0.999 ** t) * g * g, rtol=1e-12)


def test_first_step_closed_form_with_eps():
    """At t = 1 the bias corrections undo (1 - beta): the update is lr g / (|g| + eps)."""
    g = np.array([1e-9, -3e-8, 2.0, -0.5, 0.0])
    theta0 = np.array([0.1, 0.2, -0.3, 0.4, 0.5])
    lr, eps = 0.02, 1e-8
    (theta, _, _), = oadam.adam(theta0, [g], lr, 0.9, 0.999, eps)
    np.testing.assert_allclose(theta, theta0 - lr * g / (np.abs(g) + eps), rtol=1e-14, atol=1e-18)


def test_eps_free_trajectory_is_invariant_to_gradient_scale():
    rng = np.random.default_rng(4)
    theta0 = rng.uniform(-1, 1, 50)
    grads = _grads(50, 7, seed=5)
    a = oadam.adam(theta0, grads, 3e-3, 0.9, 0.999, eps=0.0)
    b = oadam.adam(theta0, [1024.0 * g for g in grads], 3e-3, 0.9, 0.999, eps=0.0)
    for (ta, _, _), (tb, _, _) in zip(a, b):
        np.testing.assert_allclose(ta, tb, rtol=1e-14, atol=1e-16)


def test_absolute_form_bounds_the_values():
    rng = np.random.default_rng(6)
    theta0 = rng.uniform(-1, 1, 100)
    grads = _grads(100, 6, seed=7)
    vals = oadam.adam(theta0, grads, 1e-2)
    mags = oadam.adam(theta0, grads, 1e-2, absolute=True)
    for (th, m, v), (tha, ma, va) in zip(vals, mags):
        assert np.all(np.abs(th) <= tha) and np.all(np.abs(m) <= ma) and np.array_equal(v, va)
