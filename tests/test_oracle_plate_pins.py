"""Pins of the pinned-actuator oracle (oracle/plate.py): the paper's copper
plate (Sec. 5.1, Tables 1-2) and the 1D heat workload with pinned actuators.

* The zero-Neumann Laplacian with mirrored fictitious points (eq. 3) has the
  cosine modes as eigenvectors with the closed-form eigenvalues
  -4/dp^2 sin^2(k pi dp / 2), and annihilates constants.
* The KKT map (eq. 9) is the gradient of the Lagrangian of eq. 8 (barrier and
  radiation included): central finite differences.
* The stage blocks (eq. 17) and the couplings of eq. 10 are the finite-
  difference Jacobian of K.
* The root from Newton is a minimum of the reduced NLP (states simulated by
  backward Euler): the finite-difference gradient of the cost in U vanishes
  and perturbations raise it.
* The fraction-to-the-boundary step (eq. 11) leaves exactly 0.5% of the
  binding bound's slack, and never crosses a bound.
* The lower layer with many sweeps equals the dense stage solve.
* The Gauss-Seidel sweeps with exact stage solves are their matrix
  definitions (eqs. 18, 20).
* The SGS convergence factor (Sec. 5.4, Theorem 2) falls with gamma > 0 and
  with a shorter horizon (dense iteration matrices at the root).
* Evidence for the reading of the heat workloads' actuators as heat
  sources: with the actuator cells pinned instead (the plate's model), the
  linearised double-layer iteration at the root of the 1D heat workload has
  spectral radius >= 0.99 for every gamma tried (above 1 for some) and the
  solve from the cold start diverges, while the heat-source model's factor
  is about 0.91.
"""
import numpy as np
import pytest

from oracle import nmpc as O
from oracle import plate as P
from paper_2004_02484_gb300 import workloads as wl


def small_plate(tau=100.0, m=7, N=4, shape="slope", seed=None):
    inst = wl.plate_instance(m=m, horizon=N, T=20.0, shape=shape, act_idx=(1, 4), tau=tau)
    if seed is not None:
        rng = np.random.default_rng(seed)
        inst.x0 = inst.x0 + 20.0 * rng.standard_normal(inst.x0.shape)
    return inst


def _perturbed(p, seed, sx=20.0, su=30.0, sl=1e-3):
    rng = np.random.default_rng(seed)
    X, U, L = p.cold_start()
    return (X + sx * rng.standard_normal(X.shape), U + su * rng.uniform(-1, 1, U.shape),
            L + sl * rng.standard_normal(L.shape))


def test_neumann_laplacian_cosine_eigenpairs_and_constants():
    for m in (7, 13):
        inst = wl.plate_instance(m=m, horizon=2, act_idx=(1, 4) if m < 13 else (1, 4, 8, 11))
        p = P.PinnedProblem(inst)
        dp = 1.0 / (m - 1)
        xs = np.arange(m) * dp
        assert np.allclose(p.L @ np.ones(m * m), 0.0, atol=1e-9)
        for kx, ky in ((1, 0), (2, 3), (m - 1, 1)):
            v = np.outer(np.cos(ky * np.pi * xs), np.cos(kx * np.pi * xs)).reshape(-1)
            lam = -(4 / dp ** 2) * (np.sin(kx * np.pi * dp / 2) ** 2 + np.sin(ky * np.pi * dp / 2) ** 2)
            np.testing.assert_allclose(p.L @ v, lam * v, rtol=1e-10, atol=1e-8)


def test_plate_parameters_follow_tables_1_and_2():
    inst = wl.plate_instance()
    assert inst.ns == 153 and len(inst.act) == 16 and inst.h == 5.0 and inst.horizon == 20
    rc = 8960.0 * 386.0
    assert inst.k0 == pytest.approx(400.0 / rc) and inst.beta == pytest.approx(2.0 / (rc * 0.01))
    assert inst.gamma_r == pytest.approx(2 * 0.5 * 5.67e-8 / (rc * 0.01))
    assert (inst.u_lo, inst.u_hi, inst.tau, inst.gamma, inst.r) == (300.0, 700.0, 100.0, 0.5, 0.1)


@pytest.mark.parametrize("mk", [lambda: small_plate(), lambda: wl.pinned_heat1d(m=8, horizon=3, h=1e-3)])
def test_kkt_is_the_gradient_of_the_lagrangian(mk):
    p = P.PinnedProblem(mk())
    X, U, L = _perturbed(p, 1) if p.tau > 0 else _perturbed(p, 1, 0.1, 0.3, 0.01)
    K1, K2, K3 = P.kkt(p, X, U, L)
    eps = 1e-5 * max(1.0, np.abs(X).max())
    for i in (0, p.N - 1):
        for j in range(0, p.ns, max(1, p.ns // 6)):
            # the Lagrangian is linear in lambda: a unit step is exact (a tiny
            # one would drown in the cancellation of a large cost)
            E = np.zeros_like(L); E[i, j] = 1.0
            fd = (P.lagrangian(p, X, U, L + E) - P.lagrangian(p, X, U, L - E)) / 2.0
            assert fd == pytest.approx(K1[i, j], rel=1e-6, abs=1e-6 * np.abs(K1).max())
            E = np.zeros_like(X); E[i, j] = eps
            fd = (P.lagrangian(p, X + E, U, L) - P.lagrangian(p, X - E, U, L)) / (2 * eps)
            assert fd == pytest.approx(K3[i, j], rel=1e-5, abs=1e-6 * np.abs(K3).max())
        for a in range(p.nu):
            E = np.zeros_like(U); E[i, a] = eps
            fd = (P.lagrangian(p, X, U + E, L) - P.lagrangian(p, X, U - E, L)) / (2 * eps)
            assert fd == pytest.approx(K2[i, a], rel=1e-5, abs=1e-6 * np.abs(K2).max())


def test_stage_blocks_and_couplings_are_the_jacobian_of_K():
    p = P.PinnedProblem(small_plate(m=5, N=3))
    X, U, L = _perturbed(p, 2)
    A = P.kkt_matrix(p, X, U, L, with_gamma=False)
    S = P.pack(p, X, U, L)

    def Kp(S_):
        K = P.kkt(p, *P.unpack(p, S_))
        return np.concatenate([np.concatenate([K[0][i], K[1][i], K[2][i]]) for i in range(p.N)])
    J = np.zeros_like(A)
    for c in range(len(S)):
        e = np.zeros_like(S)
        e[c] = 1e-4 * max(1.0, abs(S[c]))
        J[:, c] = (Kp(S + e) - Kp(S - e)) / (2 * e[c])
    np.testing.assert_allclose(A, J, rtol=1e-5, atol=1e-7 * np.abs(A).max())


@pytest.fixture(scope="module")
def plate_root():
    p = P.PinnedProblem(small_plate(seed=3))
    (X, U, L), hist = P.newton_solve(p, tol=1e-9)
    assert hist[-1] <= 1e-9
    return p, X, U, L


def test_newton_root_minimises_the_reduced_nlp(plate_root):
    p, X, U, L = plate_root
    assert np.all(U > p.u_lo) and np.all(U < p.u_hi)
    np.testing.assert_allclose(P.simulate(p, U), X, rtol=1e-9, atol=1e-7)
    J0 = P.reduced_cost(p, U)
    rng = np.random.default_rng(4)
    g = np.zeros_like(U)
    for i in range(p.N):
        for a in range(p.nu):
            E = np.zeros_like(U); E[i, a] = 1e-3
            g[i, a] = (P.reduced_cost(p, U + E) - P.reduced_cost(p, U - E)) / 2e-3
    # the gradient of the reduced cost vanishes at the root (relative to its
    # size at the cold start)
    g0 = np.zeros_like(U)
    Uc = p.cold_start()[1]
    for i in range(p.N):
        for a in range(p.nu):
            E = np.zeros_like(U); E[i, a] = 1e-3
            g0[i, a] = (P.reduced_cost(p, Uc + E) - P.reduced_cost(p, Uc - E)) / 2e-3
    assert np.abs(g).max() <= 1e-5 * np.abs(g0).max()
    for _ in range(5):
        assert P.reduced_cost(p, U + 0.5 * rng.standard_normal(U.shape)) > J0


def test_fraction_to_the_boundary_leaves_half_a_percent():
    p = P.PinnedProblem(small_plate())
    U = np.full((p.N, p.nu), 650.0)
    dU = np.zeros_like(U)
    dU[1, 2] = -200.0          # would push u to 850 > 700
    dU[0, 0] = 600.0           # would push u to 50 < 300
    a = P.alpha_max(p, U, dU)
    Un = U - a * dU
    G_lo, G_hi = Un - p.u_lo, p.u_hi - Un
    assert np.all(G_lo >= 0.005 * (U - p.u_lo) - 1e-12) and np.all(G_hi >= 0.005 * (p.u_hi - U) - 1e-12)
    # the binding component keeps exactly 0.5% of its slack
    assert min(G_lo[0, 0] / (U[0, 0] - p.u_lo), G_hi[1, 2] / (p.u_hi - U[1, 2])) == pytest.approx(0.005)
    assert P.alpha_max(p, U, np.zeros_like(U)) == 1.0


def test_lower_layer_with_many_sweeps_is_the_dense_stage_solve(plate_root):
    p, X, U, L = plate_root
    Xp, Up, Lp = _perturbed(p, 5, 2.0, 5.0, 1e-4)
    Xp, Up, Lp = X + (Xp - p.cold_start()[0]) * 0.1, U + 0.1 * (Up - p.cold_start()[1]), L
    K1, K2, K3 = P.kkt(p, Xp, Up, Lp)
    for i in (0, p.N - 1):
        D = P.stage_block(p, Xp, Up, Lp, i)
        d = np.linalg.solve(D, np.concatenate([K1[i], K2[i], K3[i]]))
        low = P.StageLower(p, Xp, Up, Lp, i, n_lo=60, n_u_it=60)
        dx, du, dl = low.solve(K1[i], K3[i], K2[i])
        np.testing.assert_allclose(dx, d[:p.ns], rtol=1e-8, atol=1e-10 * np.abs(d).max())
        np.testing.assert_allclose(du, d[p.ns:p.ns + p.nu], rtol=1e-8, atol=1e-10 * np.abs(d).max())
        np.testing.assert_allclose(dl, d[p.ns + p.nu:], rtol=1e-8, atol=1e-12 + 1e-8 * np.abs(d).max())


@pytest.mark.parametrize("variant", ["jacobi", "fgs", "sgs", "redblack"])
def test_sweeps_with_exact_stage_solves_are_their_matrix_definitions(variant):
    p = P.PinnedProblem(small_plate(m=5, N=4, tau=0.0))
    X, U, L = _perturbed(p, 6)
    A = P.kkt_matrix(p, X, U, L, with_gamma=True)
    n = 2 * p.ns + p.nu
    D = np.zeros_like(A)
    for i in range(p.N):
        D[i * n:(i + 1) * n, i * n:(i + 1) * n] = A[i * n:(i + 1) * n, i * n:(i + 1) * n]
    Lo, Up = np.tril(A - D), np.triu(A - D)
    K = P.kkt(p, X, U, L)
    Kp = np.concatenate([np.concatenate([K[0][i], K[1][i], K[2][i]]) for i in range(p.N)])
    if variant == "jacobi":
        d = np.linalg.solve(D, Kp)
    elif variant == "fgs":
        d = np.linalg.solve(D + Lo, Kp)
    elif variant == "sgs":
        d = np.linalg.solve(D + Lo, Kp - Up @ np.linalg.solve(D + Up, Kp))
    else:
        Lrb = np.zeros_like(A)
        for i in range(1, p.N, 2):
            for j in (i - 1, i + 1):
                if 0 <= j < p.N:
                    Lrb[i * n:(i + 1) * n, j * n:(j + 1) * n] = (Lo + Up)[i * n:(i + 1) * n, j * n:(j + 1) * n]
        d = np.linalg.solve(D + Lrb, Kp)
    Xe, Ue, Le = P.unpack(p, P.pack(p, X, U, L) - d)
    Xg, Ug, Lg, _, a = P.iteration(p, X, U, L, variant, exact_inner=True)
    assert a == 1.0
    for g, e in ((Xg, Xe), (Ug, Ue), (Lg, Le)):
        np.testing.assert_allclose(g, e, rtol=1e-9, atol=1e-9 * np.abs(e).max())


@pytest.mark.parametrize("variant", ["jacobi", "sgs", "redblack"])
def test_plate_iterations_reach_the_newton_root(plate_root, variant):
    p, X, U, L = plate_root
    (Xv, Uv, Lv), info = P.solve(p, variant, tol=1e-7, max_iter=3000)
    assert info["converged"], info["res_inf"]
    assert np.abs(Uv - U).max() <= 1e-5 * np.abs(U).max()
    assert all(0.0 < a <= 1.0 for a in info["alphas"])


def _radius(p, X, U, L):
    """Spectral radius of the linearised double-layer iteration at the root
    with u~ = u^k: I - D^{-1} A (D: stage blocks with gamma, A: the full KKT
    matrix without it), exact stage solves."""
    A = P.kkt_matrix(p, X, U, L, with_gamma=False)
    n = 2 * p.ns + p.nu
    D = np.zeros_like(A)
    Ag = P.kkt_matrix(p, X, U, L, with_gamma=True)
    for i in range(p.N):
        D[i * n:(i + 1) * n, i * n:(i + 1) * n] = Ag[i * n:(i + 1) * n, i * n:(i + 1) * n]
    return float(np.abs(np.linalg.eigvals(np.eye(len(A)) - np.linalg.solve(D, A))).max())


def test_pinned_actuators_stall_the_1d_heat_workload_while_heat_sources_converge():
    """The reading recorded for the heat workloads: with the actuator cells
    pinned to the inputs (the plate's model) and no bounds, the linearised
    double-layer iteration at the root of the 1D heat workload has spectral
    radius >= 0.99 for every gamma/h from 1e-3 to 1e4 (above 1 for some), and
    the iteration from the cold start with the workload's gamma = h R
    diverges; with the actuators as heat sources (the reading the build uses)
    the factor is about 0.91 and the solve converges."""
    inst = wl.pinned_heat1d()
    base = P.PinnedProblem(inst)
    (X, U, L), hist = P.newton_solve(base, S0=base.cold_start(0.0), tol=1e-10)
    assert hist[-1] <= 1e-10
    radii = []
    for ratio in (1e-3, 1e-1, 1.0, 10.0, 100.0, 1e4):
        inst.gamma = ratio * inst.h
        radii.append(_radius(P.PinnedProblem(inst), X, U, L))
    assert min(radii) >= 0.99 and max(radii) > 1.0, radii
    inst.gamma = inst.h * inst.r
    p = P.PinnedProblem(inst)
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)
        _, info = P.solve(p, "jacobi", S0=p.cold_start(0.0), tol=1e-6, max_iter=200)
    assert not info["converged"]
    # the heat-source reading of the same workload
    hp = O.Problem(wl.heat1d_single())
    (Xh, Uh, Lh), hh = O.newton_solve(hp, tol=1e-12)
    Ah = O.dense_kkt_matrix(hp, Xh, Uh, Lh, with_gamma=False)
    Dh = np.zeros_like(Ah)
    blocks = O.dense_stage_blocks(hp, Xh, Uh, Lh)
    n = blocks[0].shape[0]
    for i, B in enumerate(blocks):
        Dh[i * n:(i + 1) * n, i * n:(i + 1) * n] = B
    rh = float(np.abs(np.linalg.eigvals(np.eye(len(Ah)) - np.linalg.solve(Dh, Ah))).max())
    assert rh < 0.95
    assert O.solve_jacobi(hp, tol=1e-6)[1]["converged"]


def _sgs_factor(p, X, U, L):
    """rho((D + L)^{-1} U (D + U)^{-1} L) of the KKT matrix at (X, U, L) with
    the regularization in D (the linearization of Theorem 1, u~ = u*)."""
    A = P.kkt_matrix(p, X, U, L, with_gamma=True)
    n = 2 * p.ns + p.nu
    D = np.zeros_like(A)
    for i in range(p.N):
        D[i * n:(i + 1) * n, i * n:(i + 1) * n] = A[i * n:(i + 1) * n, i * n:(i + 1) * n]
    R = A - D
    Lo, Up = np.tril(R), np.triu(R)
    M = np.linalg.solve(D + Lo, Up) @ np.linalg.solve(D + Up, Lo)
    return float(np.abs(np.linalg.eigvals(M)).max())


def test_sgs_factor_falls_with_regularization_and_a_short_horizon():
    """Sec. 5.4 and Theorem 2: the SGS convergence factor at the root of the
    plate problem (7 x 7 grid, N = 20, Table 2's tau) is smaller with gamma =
    0.5 than without regularization, and smaller for T = 20 s than for
    T = 100 s; with either remedy it is well below 1."""
    rho = {}
    for T in (20.0, 100.0):
        for g in (0.0, 0.5):
            inst = wl.plate_instance(m=7, horizon=20, T=T, act_idx=(1, 4), gamma=g)
            p = P.PinnedProblem(inst)
            (X, U, L), hist = P.newton_solve(p, tol=1e-9)
            assert hist[-1] <= 1e-9
            rho[T, g] = _sgs_factor(p, X, U, L)
    assert rho[100.0, 0.5] < 0.8 * rho[100.0, 0.0]
    assert rho[20.0, 0.0] < 0.5 * rho[100.0, 0.0] and rho[20.0, 0.5] < rho[100.0, 0.5]
    assert max(rho[20.0, 0.0], rho[20.0, 0.5], rho[100.0, 0.5]) < 0.7
