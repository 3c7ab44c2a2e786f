"""Adam, the optimiser the paper trains its examples with (Section 4.1's entry-wise Jacobi
weights, Section 4.5's GCN), as Kingma and Ba define it (ICLR 2015, Algorithm 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Per step t = 1, 2, ... with gradient g_t: the moment estimates m_t = beta1 m_{t-1} +
(1 - beta1) g_t and v_t = beta2 v_{t-1} + (1 - beta2) g_t^2 (both zero at t = 0), their
bias-corrected forms m_t / (1 - beta1^t) and v_t / (1 - beta2^t), and the update
theta_t = theta_{t-1} - lr * mhat_t / (sqrt(vhat_t) + eps), element by element.  Float64
throughout; the hyperparameters are taken as given (a caller matching a float32 kernel
passes the float32 values the kernel receives).  Plain numpy, one step at a time.
"""
from __future__ import annotations

import numpy as np


def adam(theta0, grads, lr, beta1=0.9, beta2=0.999, eps=1e-8, absolute=False):
    """Run len(grads) Adam steps from theta0 (moments zero) and return the list of
    (theta_t, m_t, v_t) after each step, float64.

    absolute=True returns instead the magnitudes that bound each quantity's rounding:
    theta_t -> |theta0| + sum of |update_s| (s <= t), m_t -> the same recurrence over |g|,
    v_t unchanged (it is a sum of nonnegative terms)."""
    theta = np.asarray(theta0, dtype=np.float64).copy()
    mag = np.abs(theta)
    m = np.zeros_like(theta)
    m_abs = np.zeros_like(theta)
    v = np.zeros_like(theta)
    out = []
    for t, g in enumerate(grads, start=1):
        g = np.asarray(g, dtype=np.float64)
        m = beta1 * m + (1.0 - beta1) * g
        m_abs = beta1 * m_abs + (1.0 - beta1) * np.abs(g)
        v = beta2 * v + (1.0 - beta2) * g * g
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        update = lr * mhat / (np.sqrt(vhat) + eps)
        theta = theta - update
        mag = mag + np.abs(update)
        out.append((mag.copy(), m_abs.copy(), v.copy()) if absolute else (theta.copy(), m.copy(), v.copy()))
    return out
