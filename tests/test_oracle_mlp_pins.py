"""Pins of the network oracle (oracle/mlp.py) against independent facts."""
import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp as M


def test_gelu_is_z_times_normal_cdf():
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(M.gelu(z), z * norm.cdf(z), rtol=1e-13, atol=1e-15)


def test_gelu_grad_matches_finite_differences():
    z = np.linspace(-5, 5, 41)
    fd = (M.gelu(z + 1e-6) - M.gelu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(M.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)
    assert abs(M.gelu_grad(0.0) - 0.5) < 1e-15


def test_bf16_rounding_is_round_to_nearest_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> ties to even (1); 1 + 3*2^-8 -> 1 + 2^-6
    assert M.bf16(1.0 + 2.0 ** -8) == 1.0
    assert M.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    v = np.random.default_rng(0).standard_normal(1000)
    r = M.bf16(v)
    assert np.all(np.abs(r - v) <= np.abs(v) * 2.0 ** -8 + 1e-300)


@pytest.mark.parametrize("widths", [[8, 16, 8], [16, 24, 24, 8]])
def test_backprop_matches_finite_differences(widths):
    """Exact-arithmetic mode: the analytic gradient equals central differences."""
    rng = np.random.default_rng(1)
    n = sum(widths[l] * widths[l + 1] + widths[l + 1] for l in range(len(widths) - 1))
    p = rng.standard_normal(n) * 0.3
    x = rng.standard_normal((5, widths[0]))
    t = rng.standard_normal((5, widths[-1]))
    _, g = M.loss_and_grads(p, widths, x, t, bf16_ops=False)
    fd = np.zeros(n)
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1e-6
        fd[j] = (M.loss_and_grads(p + e, widths, x, t, False)[0]
                 - M.loss_and_grads(p - e, widths, x, t, False)[0]) / 2e-6
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_adam_first_step_moves_by_lr_times_sign():
    """With zero moments, the bias-corrected first step is lr * sign(g) (|g| >> eps)."""
    g = np.array([3.0, -0.5, 1e-2, -7.0])
    p, m, v = M.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 1e-3)
    np.testing.assert_allclose(p, -1e-3 * np.sign(g), rtol=1e-6)
