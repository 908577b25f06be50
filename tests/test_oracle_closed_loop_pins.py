"""Pins of the oracle's closed-loop parts (oracle/nmpc.py plant_step and
closed_loop, Sec. 5.3's receding-horizon use) and of the network oracle's
Adam update (oracle/mlp.py adam_step) against closed forms.

* plant_step with k1 = 0 is the linear recursion w <- (I + tau k0 Lap) w +
  tau b0 B u1, tau = dt / n_sub.  On the Dirichlet FD Laplacian's sine
  eigenvectors (closed-form eigenvalues) every mode evolves by a scalar
  geometric recursion, so the result after n_sub sub-steps has a closed form
  that never calls the oracle's Laplacian.
* closed_loop with k1 = 0 applies, at each step, the first control of the
  linear-quadratic problem posed from the current plant state, which the
  textbook Riccati recursion gives independently of the Jacobi iteration.
* Adam (Kingma & Ba, ICLR 2015, Algorithm 1): with a constant gradient g the
  bias-corrected moments are exactly g and g^2, so every step moves by
  lr g / (|g| + eps); a two-step case with different gradients, derived by
  hand, depends on beta2 and on both bias corrections.
"""
import copy

import numpy as np
import pytest

from oracle import mlp as M
from oracle import nmpc as O
from paper_2004_02484_gb300 import workloads as wl


def _sine_basis_1d(m):
    """Orthonormal sine eigenvectors of the M-cell Dirichlet FD Laplacian and
    their eigenvalues -4/dx^2 sin^2(j pi dx / 2), j = 1..M, dx = 1/(M+1)."""
    dx = 1.0 / (m + 1)
    xs = np.arange(1, m + 1) * dx
    V = np.stack([np.sin(j * np.pi * xs) for j in range(1, m + 1)], axis=1)
    V /= np.linalg.norm(V, axis=0)[None, :]
    lam = np.array([-(4.0 / dx ** 2) * np.sin(j * np.pi * dx / 2) ** 2 for j in range(1, m + 1)])
    return V, lam


def _linear_plant_closed_form(inst, w0, u1, dt, n_sub):
    """n_sub explicit-Euler sub-steps of w' = k0 Lap w + b0 B u1 in the sine
    eigenbasis: c <- (1 + tau k0 lam) c + tau s, s = V^T b0 B u1."""
    V, lam = _sine_basis_1d(inst.mx)
    tau = dt / n_sub
    src = np.zeros(inst.mx)
    for a, cell in enumerate(inst.act):
        src[cell] += inst.act_gain * u1[a]
    c, s = V.T @ w0, V.T @ src
    g = 1.0 + tau * inst.k0 * lam
    # geometric series: c_n = g^n c_0 + tau s (g^n - 1) / (g - 1)
    cn = g ** n_sub * c + tau * s * (g ** n_sub - 1.0) / (g - 1.0)
    return V @ cn


@pytest.mark.parametrize("n_sub", [1, 3, 7])
def test_plant_step_of_a_sine_mode_is_the_scalar_recursion(n_sub):
    inst = wl.tiny1d(m=12, horizon=3, n_u=2, k1=0.0)
    p = O.Problem(inst)
    V, lam = _sine_basis_1d(inst.mx)
    mode = 3
    w0 = V[:, mode - 1].copy()
    dt = 2.5e-3
    w = O.plant_step(p, w0, np.zeros(p.nu), dt, n_sub).ravel()
    expect = (1.0 + (dt / n_sub) * inst.k0 * lam[mode - 1]) ** n_sub * w0
    np.testing.assert_allclose(w, expect, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("n_sub", [1, 4])
def test_plant_step_with_sources_matches_the_eigenbasis_closed_form(n_sub):
    inst = wl.tiny1d(m=10, horizon=3, n_u=2, k1=0.0, seed=5)
    p = O.Problem(inst)
    u1 = np.array([0.7, -1.3])
    dt = 1.7e-3
    w = O.plant_step(p, inst.x0, u1, dt, n_sub).ravel()
    expect = _linear_plant_closed_form(inst, np.asarray(inst.x0), u1, dt, n_sub)
    np.testing.assert_allclose(w, expect, rtol=1e-12, atol=1e-13)


def test_plant_step_nonlinear_single_substep_is_one_explicit_euler_step():
    # k1 != 0, one sub-step: w1 - w0 = dt (div(k(w) grad w) + b0 B u), with the
    # flux form written out face by face (k at the face mean, zero ring)
    inst = wl.tiny1d(m=9, horizon=2, n_u=1, k1=0.5, seed=9)
    p = O.Problem(inst)
    u1 = np.array([0.4])
    dt = 1e-3
    w0 = np.asarray(inst.x0, dtype=np.float64)
    w1 = O.plant_step(p, w0, u1, dt, 1).ravel()
    wb = np.concatenate([[0.0], w0, [0.0]])
    dx = 1.0 / (inst.mx + 1)
    kf = inst.k0 * (1.0 + inst.k1 * 0.5 * (wb[1:] + wb[:-1]))   # faces j-1/2 .. M+1/2
    flux = kf * (wb[1:] - wb[:-1]) / dx
    rate = (flux[1:] - flux[:-1]) / dx
    rate[inst.act[0]] += inst.act_gain * u1[0]
    np.testing.assert_allclose(w1, w0 + dt * rate, rtol=1e-12, atol=1e-14)


def test_closed_loop_applies_the_first_lq_control_and_the_linear_plant():
    inst = wl.tiny1d(m=8, horizon=4, n_u=1, k1=0.0, seed=13)
    steps, n_sub = 3, 2
    U1, W, its = O.closed_loop(inst, steps, n_sub, tol=1e-11)
    assert U1.shape == (steps, 1) and W.shape == (steps + 1, inst.mx)
    for k in range(steps):
        cur = copy.copy(inst)
        cur.x0 = W[k].copy()
        u_lq = O.riccati_lq(O.Problem(cur))
        # the control applied at step k is the first stage's (not a later one)
        np.testing.assert_allclose(U1[k], u_lq[0], rtol=1e-7, atol=1e-9)
        assert np.abs(u_lq[0] - u_lq[1]).max() > 1e-3 * np.abs(u_lq[0]).max()
        # the plant advances by one stage length h in n_sub sub-steps
        expect = _linear_plant_closed_form(inst, W[k], U1[k], inst.h, n_sub)
        np.testing.assert_allclose(W[k + 1], expect, rtol=1e-12, atol=1e-13)


def test_adam_constant_gradient_moves_lr_per_step():
    g = np.array([3.0, -0.5, 2e-2, -7.0])
    lr, eps = 1e-3, 1e-8
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 6):
        p, m, v = M.adam_step(p, g, m, v, t, lr, eps=eps)
        np.testing.assert_allclose(p, -t * lr * g / (np.abs(g) + eps), rtol=1e-12)


def test_adam_two_steps_hand_derived():
    """g1 = 1, g2 = -2, beta1 = 0.9, beta2 = 0.999, lr = 1, eps = 0:
    m1 = 0.1, v1 = 0.001 -> step 1 moves by -1;
    m2 = 0.09 - 0.2 = -0.11, v2 = 0.000999 + 0.004 = 0.004999,
    m2^ = -0.11 / 0.19, v2^ = 0.004999 / 0.001999 -> p2 = -1 + (11/19) / sqrt(4999/1999)."""
    p, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    p, m, v = M.adam_step(p, np.array([1.0]), m, v, 1, 1.0, eps=0.0)
    np.testing.assert_allclose(p, [-1.0], rtol=1e-14)
    p, m, v = M.adam_step(p, np.array([-2.0]), m, v, 2, 1.0, eps=0.0)
    np.testing.assert_allclose(m, [-0.11], rtol=1e-13)
    np.testing.assert_allclose(v, [0.004999], rtol=1e-13)
    np.testing.assert_allclose(p, [-1.0 + (11.0 / 19.0) / np.sqrt(4999.0 / 1999.0)], rtol=1e-13)
