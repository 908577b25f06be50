"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against the mathematics the paper fixes: the
Lagrangian whose gradient the KKT map must be (eq. 6 -> eq. 9), finite-
difference Jacobians, closed-form Laplacian eigenpairs, the conservative flux
form of the heat equation, Newton vs. a dense LU of eq. 10, the textbook
Riccati/LQ solution of the linear case, brute-force optimality of the root,
Lemma 1's textbook Jacobi iteration on matrices assembled by finite
differences, Lemma 4's nilpotency and Lemma 3's convergence factor.
"""
import os

import numpy as np
import pytest

from oracle import nmpc as O
from paper_2004_02484_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _perturbed(p, seed=0, sx=0.1, su=1.0, sl=0.01):
    rng = np.random.default_rng(seed)
    X, U, L = p.cold_start()
    return (X + sx * rng.standard_normal(X.shape), U + su * rng.standard_normal(U.shape),
            L + sl * rng.standard_normal(L.shape))


def _fd_grad(fun, s, eps):
    g = np.zeros_like(s)
    for j in range(len(s)):
        e = np.zeros_like(s)
        e[j] = eps
        g[j] = (fun(s + e) - fun(s - e)) / (2 * eps)
    return g


# ---------------------------------------------------------------------------
# Input generator
# ---------------------------------------------------------------------------
def test_splitmix64_published_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    for seed, idx, val in rows:
        out = wl.splitmix64(int(seed), int(idx) + 1)
        assert int(out[int(idx)]) == int(val, 16)


def test_workloads_deterministic_and_shaped():
    a, b = wl.heat2d_single(), wl.heat2d_single()
    assert np.array_equal(a.x0, b.x0) and np.array_equal(a.ref, b.ref)
    assert a.ng == 4096 and a.n_u == 8 and a.horizon == 50
    # 2 x 4 actuator grid at x in {1/8, 3/8, 5/8, 7/8}, y in {1/4, 3/4}; 0-based
    # cell j sits at (j+1)/65: 1/8 -> 7.125 -> 7, 3/8 -> 23, 5/8 -> 40, 7/8 -> 56,
    # 1/4 -> 15.25 -> 15, 3/4 -> 47.75 -> 48
    assert sorted(a.act.tolist()) == sorted(iy * 64 + ix for iy in (15, 48) for ix in (7, 23, 40, 56))
    c1 = wl.heat1d_single()
    assert c1.act.tolist() == [7, 24] and c1.ng == 32
    assert 0.0 <= c1.x0.min() and c1.x0.max() < 1.0
    batch = wl.heat1d_ragged_batch(64)
    ms = [i.mx for i in batch]
    assert min(ms) >= 32 and max(ms) <= 256
    assert all(10 <= i.horizon <= 60 and 1 <= i.n_u <= 4 for i in batch)
    assert all(1e-3 <= i.r <= 1e-1 for i in batch)


# ---------------------------------------------------------------------------
# Model (Sec. 2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [1, 2])
def test_laplacian_closed_form_eigenpairs(dim):
    """sin modes are eigenvectors of the Dirichlet FD Laplacian with eigenvalue
    -(4/dx^2) sin^2(m pi dx / 2) (per axis)."""
    inst = wl.tiny1d(m=17) if dim == 1 else wl.tiny2d(mx=9, my=7)
    p = O.Problem(inst)
    xs = np.arange(1, p.mx + 1) * p.dx
    ys = np.arange(1, p.my + 1) * p.dy
    for m, n in [(1, 1), (3, 2), (p.mx, 1)]:
        if dim == 1:
            v = np.sin(m * np.pi * xs)[None, :]
            lam = -(4 / p.dx ** 2) * np.sin(m * np.pi * p.dx / 2) ** 2
        else:
            n = min(n, p.my)
            v = np.outer(np.sin(n * np.pi * ys), np.sin(m * np.pi * xs))
            lam = (-(4 / p.dx ** 2) * np.sin(m * np.pi * p.dx / 2) ** 2
                   - (4 / p.dy ** 2) * np.sin(n * np.pi * p.dy / 2) ** 2)
        np.testing.assert_allclose(p.lap(v), lam * v, rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("dim", [1, 2])
def test_kirchhoff_equals_flux_form(dim):
    """Lap Phi(w) equals the conservative flux difference with face
    conductivity k((w_j + w_m)/2), written out face by face."""
    inst = wl.tiny1d(m=11) if dim == 1 else wl.tiny2d(mx=7, my=5)
    p = O.Problem(inst)
    w = np.random.default_rng(1).uniform(-0.5, 1.5, p.shape)
    k = lambda a, b: p.k0 * (1 + p.k1 * 0.5 * (a + b))
    wp = np.pad(w, 1)  # Dirichlet-zero ring
    flux = np.zeros_like(w)
    for iy in range(p.my):
        for ix in range(p.mx):
            c = wp[iy + 1, ix + 1]
            acc = 0.0
            for (dy, dx, h2) in ([(0, 1, p.dx ** 2), (0, -1, p.dx ** 2)] +
                                 ([(1, 0, p.dy ** 2), (-1, 0, p.dy ** 2)] if dim == 2 else [])):
                nb = wp[iy + 1 + dy, ix + 1 + dx]
                acc += k(c, nb) * (nb - c) / h2
            flux[iy, ix] = acc
    np.testing.assert_allclose(p.lap(p.phi(w)), flux, rtol=1e-12, atol=1e-10)


# ---------------------------------------------------------------------------
# KKT map (Sec. 3.2, eq. 9)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mk", [lambda: wl.tiny1d(m=8, horizon=4, n_u=2),
                                lambda: wl.tiny2d(mx=5, my=4, horizon=3)])
def test_kkt_is_gradient_of_lagrangian(mk):
    """K1 = dL/dlambda, K2 = dL/du, K3 = dL/dx for the Lagrangian of eq. 6."""
    p = O.Problem(mk())
    X, U, L = _perturbed(p)
    S = O.pack(p, X, U, L)
    g = _fd_grad(lambda s: O.lagrangian(p, *O.unpack(p, s)), S, 1e-6)
    gX, gU, gL = O.unpack(p, g)
    K1, K2, K3 = O.kkt(p, X, U, L)
    scale = max(np.abs(K1).max(), np.abs(K3).max())
    np.testing.assert_allclose(K1, gL, atol=1e-7 * max(1, scale))
    np.testing.assert_allclose(K3, gX, atol=1e-7 * max(1, scale))
    np.testing.assert_allclose(K2, gU, atol=1e-9)


def test_kkt_regularization_term():
    p = O.Problem(wl.tiny1d())
    X, U, L = _perturbed(p)
    ut = U + 0.3
    a = O.kkt(p, X, U, L, u_tilde=ut)[1]
    b = O.kkt(p, X, U, L)[1]
    np.testing.assert_allclose(a - b, p.gamma * (U - ut), rtol=1e-12)


@pytest.mark.parametrize("mk", [lambda: wl.tiny1d(m=7, horizon=3, n_u=2),
                                lambda: wl.tiny2d(mx=4, my=4, horizon=3)])
def test_stage_blocks_and_couplings_match_fd(mk):
    """D_i (exact Jacobian) and the constant M_L / M_U couplings of eq. 10
    against a central-difference Jacobian of the whole KKT map."""
    p = O.Problem(mk())
    X, U, L = _perturbed(p, 2)
    S = O.pack(p, X, U, L)
    Kf = lambda s: O.pack_kkt(p, *O.kkt(p, *O.unpack(p, s)))
    n = len(S)
    J = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1e-6
        J[:, j] = (Kf(S + e) - Kf(S - e)) / 2e-6
    A = O.dense_kkt_matrix(p, X, U, L, with_gamma=False)
    np.testing.assert_allclose(A, J, atol=1e-7 * np.abs(A).max())


# ---------------------------------------------------------------------------
# Newton (Sec. 3.3) and the root
# ---------------------------------------------------------------------------
def test_block_elimination_equals_dense_lu():
    p = O.Problem(wl.tiny2d(mx=4, my=3, horizon=4))
    X, U, L = _perturbed(p, 3)
    S1 = O.newton_step(p, X, U, L, use_dense_lu=False)
    S2 = O.newton_step(p, X, U, L, use_dense_lu=True)
    for a, b in zip(S1, S2):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12)


def test_newton_converges_quadratically_on_heat1d_single():
    p = O.Problem(wl.heat1d_single())
    _, hist = O.newton_solve(p, tol=1e-14)
    assert hist[-1] <= 1e-14 and len(hist) <= 8
    # quadratic: each residual below C * previous^2 once in the local regime
    for a, b in zip(hist[1:-1], hist[2:]):
        assert b <= 10.0 * a * a / hist[1] + 1e-15


@pytest.mark.parametrize("dim", [1, 2])
def test_linear_case_matches_riccati(dim):
    """k1 = 0 makes the NLP an LQ problem: the KKT root's controls equal the
    textbook Riccati/LQ solution, and one Newton step from anywhere is exact."""
    inst = (wl.tiny1d(m=9, horizon=5, n_u=2, k1=0.0) if dim == 1
            else wl.tiny2d(mx=5, my=4, horizon=4, k1=0.0))
    p = O.Problem(inst)
    U_lq = O.riccati_lq(p)
    X, U, L = _perturbed(p, 4)
    X1, U1, L1 = O.newton_step(p, X, U, L)
    assert O.kkt_norms(*O.kkt(p, X1, U1, L1))[0] < 1e-12
    np.testing.assert_allclose(U1, U_lq, rtol=1e-7, atol=1e-9 * np.abs(U_lq).max())


def test_root_is_a_local_minimum_of_the_nlp():
    """Brute force on eq. 6: at the KKT root the reduced cost J(U) (states by
    simulation) is stationary and grows along random directions."""
    p = O.Problem(wl.tiny1d(m=8, horizon=4, n_u=2, h=1e-3))
    (X, U, L), hist = O.newton_solve(p)
    assert hist[-1] < 1e-13
    J0 = O.nlp_cost(p, U)
    g = _fd_grad(lambda u: O.nlp_cost(p, u.reshape(U.shape)), U.ravel(), 1e-4)
    assert np.abs(g).max() < 1e-9
    rng = np.random.default_rng(5)
    for _ in range(5):
        d = rng.standard_normal(U.shape)
        assert O.nlp_cost(p, U + 0.05 * d) > J0
    # the root's states are the simulated trajectory
    Xs = O.simulate_backward_euler(p, U)
    np.testing.assert_allclose(X.reshape(p.N, -1), Xs, atol=1e-12)


# ---------------------------------------------------------------------------
# Lower layer (Sec. 4.3) against textbook Jacobi on FD-assembled matrices
# ---------------------------------------------------------------------------
def _fd_Fx(p, x, u):
    """F_x = h grad_x f - I assembled column by column from f by central differences."""
    n = p.ng
    F = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1e-6
        fp = p.f((x.ravel() + e).reshape(p.shape), u).ravel()
        fm = p.f((x.ravel() - e).reshape(p.shape), u).ravel()
        F[:, j] = (fp - fm) / 2e-6
    return p.h * F - np.eye(n)


@pytest.mark.parametrize("n_lo", [1, 2, 3])
def test_P_inverse_is_textbook_jacobi(n_lo):
    """apply_P_inv = n_lo textbook Jacobi sweeps (Lemma 1) on F_x, then on F_x^T
    with right-hand side b5 - A_xx v5, using matrices from finite differences."""
    p = O.Problem(wl.tiny2d(mx=5, my=4, horizon=2))
    X, U, L = _perturbed(p, 6)
    c = O.StageCoeffs(p, X, U, L)
    i = 1
    Fx = _fd_Fx(p, X[i], U[i])
    rng = np.random.default_rng(7)
    b4 = rng.standard_normal(p.shape)
    b5 = rng.standard_normal(p.shape)
    v4, v5 = O.apply_P_inv(c, np.stack([b4, b4]), np.stack([b5, b5]), n_lo)

    def textbook(A, b, k):
        D = np.diag(np.diag(A))
        LU = A - D
        v = np.zeros_like(b)
        for _ in range(k):
            v = np.linalg.solve(D, b - LU @ v)
        return v
    # A_xx = d K3_i / d x_i by central differences of the KKT map (itself pinned
    # to the Lagrangian gradient above)
    Axx = np.zeros((p.ng, p.ng))
    for j in range(p.ng):
        Xp, Xm = X.copy(), X.copy()
        Xp[i].flat[j] += 1e-6
        Xm[i].flat[j] -= 1e-6
        Axx[:, j] = (O.kkt(p, Xp, U, L)[2][i].ravel() - O.kkt(p, Xm, U, L)[2][i].ravel()) / 2e-6
    w5 = textbook(Fx, b4.ravel(), n_lo)
    w4 = textbook(Fx.T, b5.ravel() - Axx @ w5, n_lo)
    np.testing.assert_allclose(v5[i].ravel(), w5, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(v4[i].ravel(), w4, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("mk", [lambda: wl.tiny1d(m=9, horizon=3, n_u=2),
                                lambda: wl.tiny2d(mx=5, my=5, horizon=3)])
def test_lower_layer_converges_to_exact_stage_solve(mk):
    """Stage-decoupling invariant: with many inner iterations the lower layer
    equals a dense solve of each D_i (eq. 17 block, with gamma)."""
    p = O.Problem(mk())
    X, U, L = _perturbed(p, 8)
    Xa, Ua, La, _ = O.jacobi_iteration(p, X, U, L, n_lo=80, n_u_it=80)
    Xb, Ub, Lb, _ = O.jacobi_iteration(p, X, U, L, exact_inner=True)
    for a, b in zip((Xa, Ua, La), (Xb, Ub, Lb)):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-11)


def test_stage_update_depends_only_on_neighbours():
    """Eq. 15: stage i's update reads x_{i-1}, s_i, lambda_{i+1} of iterate k only."""
    p = O.Problem(wl.tiny1d(m=8, horizon=6, n_u=2))
    X, U, L = _perturbed(p, 9)
    base = O.jacobi_iteration(p, X, U, L)
    i = 3
    X2, U2, L2 = X.copy(), U.copy(), L.copy()
    for j in range(p.N):
        if j not in (i - 1, i, i + 1):
            X2[j] += 1.0
            U2[j] += 1.0
            L2[j] += 1.0
    U2[i - 1] += 1.0; L2[i - 1] += 1.0   # only x_{i-1} may matter from stage i-1
    X2[i + 1] += 1.0; U2[i + 1] += 1.0   # only lambda_{i+1} may matter from stage i+1
    pert = O.jacobi_iteration(p, X2, U2, L2)
    for a, b in zip(base[:3], pert[:3]):
        np.testing.assert_array_equal(a[i], b[i])


# ---------------------------------------------------------------------------
# Upper layer (Sec. 4.2): convergence theory on tiny instances
# ---------------------------------------------------------------------------
def _iteration_blocks(p, S, with_gamma=True):
    X, U, L = S
    D = O.dense_stage_blocks(p, X, U, L, with_gamma)
    ML, MU = O.coupling_blocks(p)
    n = D[0].shape[0]
    Dm = np.zeros((p.N * n, p.N * n))
    LU = np.zeros_like(Dm)
    for i in range(p.N):
        Dm[i * n:(i + 1) * n, i * n:(i + 1) * n] = D[i]
        if i > 0:
            LU[i * n:(i + 1) * n, (i - 1) * n:i * n] = ML
        if i < p.N - 1:
            LU[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = MU
    return Dm, LU, n


def test_lemma4_split_is_nilpotent():
    """rho(Dbar^{-1}(L+U)) = 0 (Lemma 4): the matrix is nilpotent, so a power of
    it vanishes (checked by the power, which avoids unstable eigenvalues)."""
    p = O.Problem(wl.tiny1d(m=6, horizon=4, n_u=2))
    (S, _) = O.newton_solve(p)
    Dm, LU, n = _iteration_blocks(p, S)
    # remove h * Dtilde: the h grad_u f and h (grad_u f)^T blocks
    Dbar = Dm.copy()
    ng, nu = p.ng, p.nu
    for i in range(p.N):
        o = i * n
        Dbar[o:o + ng, o + ng:o + ng + nu] = 0.0
        Dbar[o + ng:o + ng + nu, o + ng + nu:o + n] = 0.0
    G = np.linalg.solve(Dbar, LU)
    Gk = np.linalg.matrix_power(G, 2 * p.N)
    assert np.abs(Gk).max() < 1e-10 * max(1.0, np.abs(G).max())
    # with the full D the iteration matrix is not nilpotent
    G2 = np.linalg.solve(Dm, LU)
    assert np.abs(np.linalg.matrix_power(G2, 2 * p.N)).max() > 1e-12


def _observed_rate(hist):
    h = np.array(hist)
    k = len(h)
    a, b = int(0.5 * k), int(0.8 * k)
    return (h[b] / h[a]) ** (1.0 / (b - a))


def test_lemma3_observed_rate_is_the_spectral_radius():
    """Thm 1 / Lemma 3 with a fixed regularization reference u~ = u*: the
    exact-inner Jacobi iteration converges with factor rho((D*)^{-1}(L+U))."""
    p = O.Problem(wl.tiny1d(m=6, horizon=4, n_u=2, h=2e-3))
    (S, _) = O.newton_solve(p)
    Dm, LU, _ = _iteration_blocks(p, S)
    rho = np.abs(np.linalg.eigvals(np.linalg.solve(Dm, LU))).max()
    assert rho < 1.0
    (_, info) = O.solve_jacobi(p, tol=1e-13, exact_inner=True, record=True, max_iter=3000,
                               u_tilde=S[1])
    assert info["converged"]
    assert abs(_observed_rate(info["hist"]) - rho) < 0.03


def test_proximal_reference_changes_the_iteration_matrix():
    """With u~ = u^k (Remark 1) the gamma term of K vanishes, so the linearized
    map is (D*)^{-1}(gamma E_u - (L+U)), E_u selecting the u entries."""
    p = O.Problem(wl.tiny1d(m=6, horizon=4, n_u=2, h=2e-3))
    (S, _) = O.newton_solve(p)
    Dm, LU, n = _iteration_blocks(p, S)
    Eu = np.zeros(Dm.shape[0])
    for i in range(p.N):
        Eu[i * n + p.ng:i * n + p.ng + p.nu] = 1.0
    rho = np.abs(np.linalg.eigvals(np.linalg.solve(Dm, p.gamma * np.diag(Eu) - LU))).max()
    (_, info) = O.solve_jacobi(p, tol=1e-13, exact_inner=True, record=True, max_iter=3000)
    assert info["converged"]
    assert abs(_observed_rate(info["hist"]) - rho) < 0.03


def test_theorem2_short_horizon_gives_convergence():
    """Thm 2(i): with gamma > 0 fixed, rho((D*)^{-1}(L+U)) -> 0 as T -> 0."""
    rhos = []
    for h in (4e-3, 1e-3, 2.5e-4):
        inst = wl.tiny1d(m=6, horizon=4, n_u=2, h=h, gamma=1e-4)
        p = O.Problem(inst)
        (S, _) = O.newton_solve(p)
        Dm, LU, _ = _iteration_blocks(p, S)
        rhos.append(np.abs(np.linalg.eigvals(np.linalg.solve(Dm, LU))).max())
    assert rhos[0] > rhos[1] > rhos[2]
    assert rhos[-1] < 0.5


# ---------------------------------------------------------------------------
# The double-layer Jacobi iteration reaches the Newton root
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mk", [wl.heat1d_single,
                                lambda: wl.tiny2d(mx=8, my=8, horizon=6, h=2e-4)])
def test_double_layer_jacobi_reaches_newton_root(mk):
    p = O.Problem(mk())
    (Sn, hist) = O.newton_solve(p)
    assert hist[-1] < 1e-13
    (Sj, info) = O.solve_jacobi(p, tol=1e-13, max_iter=5000)
    assert info["converged"]
    for a, b in zip(Sj, Sn):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-6 * max(1.0, np.abs(b).max()))
    np.testing.assert_allclose(Sj[1], Sn[1], atol=1e-9 * np.abs(Sn[1]).max() / 1e-3)
