"""Pins of the second-order-in-time oracle (oracle/wave.py): a damped string /
membrane with a cubic term, state x = (W, dW/dt) (eq. 5), the lower layer's
F_x solves by the elimination of v6 (eq. 25).

* The Laplacian: sine modes (zero Dirichlet) and cosine modes (mirrored
  zero Neumann) are eigenvectors with eigenvalues -4/dp^2 sin^2(k pi dp / 2).
* The KKT map (eq. 9) is the gradient of the Lagrangian of eq. 8:
  central finite differences.
* The stage blocks and the couplings of eq. 10 are the finite-difference
  Jacobian of K.
* The v6 elimination solves F_x exactly when E is solved exactly, and its
  transposed form solves F_x^T: against a dense solve of h grad_x f - I.
* The lower layer with many sweeps equals the dense stage solve.
* The Newton root minimises the reduced NLP (states simulated by backward
  Euler): the finite-difference gradient in U vanishes, perturbations raise
  the cost.
* With kappa = 0 the problem is linear-quadratic: one Newton step from any
  start lands on the root.
* The Gauss-Seidel sweeps with exact stage solves are their matrix
  definitions (eqs. 18, 20); with N = 1 the Jacobi iteration with exact
  stage solves is Newton.
* Theorem 3: the red-black ordering's iteration matrix (consistently ordered)
  has spectral radius rho_J^2 at the root.
* The iterations reach the Newton root.
"""
import numpy as np
import pytest

from oracle import wave as Wv
from paper_2004_02484_gb300 import workloads as wl


def small(dim=1, m=6, N=3, seed=0, **kw):
    return wl.wave_instance(dim=dim, m=m, horizon=N, T=0.01 * N, seed=seed, **kw)


def _perturbed(p, seed, sx=0.1, su=0.5, sl=0.05):
    rng = np.random.default_rng(seed)
    X, U, L = p.cold_start()
    return (X + sx * rng.standard_normal(X.shape), U + su * rng.standard_normal(U.shape),
            L + sl * rng.standard_normal(L.shape))


def _Kvec(p, X, U, L):
    K = Wv.kkt(p, X, U, L)
    return np.concatenate([np.concatenate([K[0][i], K[1][i], K[2][i]]) for i in range(p.N)])


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_laplacian_eigenpairs(bc):
    for dim, m in ((1, 9), (2, 7)):
        p = Wv.WaveProblem(small(dim=dim, m=m, bc=bc))
        if bc == "dirichlet":
            dp = 1.0 / (m + 1)
            xs = np.arange(1, m + 1) * dp
            mode = lambda k: np.sin(k * np.pi * xs)
            ks = (1, 2, m)
        else:
            dp = 1.0 / (m - 1)
            xs = np.arange(m) * dp
            mode = lambda k: np.cos(k * np.pi * xs)
            ks = (0, 1, m - 1)
        lam1 = lambda k: -(4 / dp ** 2) * np.sin(k * np.pi * dp / 2) ** 2
        for kx in ks:
            for ky in (ks if dim == 2 else (None,)):
                if dim == 1:
                    v, lam = mode(kx), lam1(kx)
                else:
                    v = np.outer(mode(ky), mode(kx)).reshape(-1)
                    lam = lam1(kx) + lam1(ky)
                np.testing.assert_allclose(p.L @ v, lam * v, rtol=1e-10, atol=1e-8 * max(1, abs(lam)))


@pytest.mark.parametrize("dim,bc,a", [(1, "dirichlet", 1.0), (2, "dirichlet", 1.0),
                                      (1, "neumann", 1.0), (1, "dirichlet", 2.5)])
def test_kkt_is_the_gradient_of_the_lagrangian(dim, bc, a):
    p = Wv.WaveProblem(small(dim=dim, m=6 if dim == 1 else 4, N=3, bc=bc, a=a))
    X, U, L = _perturbed(p, 1)
    K1, K2, K3 = Wv.kkt(p, X, U, L)
    eps = 1e-5
    for i in range(p.N):
        for j in range(p.nx):
            E = np.zeros_like(L); E[i, j] = 1.0   # linear in lambda: a unit step is exact
            fd = (Wv.lagrangian(p, X, U, L + E) - Wv.lagrangian(p, X, U, L - E)) / 2.0
            assert fd == pytest.approx(K1[i, j], rel=1e-7, abs=1e-9)
            E = np.zeros_like(X); E[i, j] = eps
            fd = (Wv.lagrangian(p, X + E, U, L) - Wv.lagrangian(p, X - E, U, L)) / (2 * eps)
            assert fd == pytest.approx(K3[i, j], rel=1e-5, abs=1e-8)
        for a in range(p.nu):
            E = np.zeros_like(U); E[i, a] = eps
            fd = (Wv.lagrangian(p, X, U + E, L) - Wv.lagrangian(p, X, U - E, L)) / (2 * eps)
            assert fd == pytest.approx(K2[i, a], rel=1e-5, abs=1e-8)


@pytest.mark.parametrize("dim,a", [(1, 1.0), (2, 1.0), (1, 2.5)])
def test_stage_blocks_and_couplings_are_the_jacobian_of_K(dim, a):
    p = Wv.WaveProblem(small(dim=dim, m=5 if dim == 1 else 3, N=3, a=a))
    X, U, L = _perturbed(p, 2)
    A = Wv.kkt_matrix(p, X, U, L, with_gamma=False)
    S = Wv.pack(p, X, U, L)
    J = np.zeros_like(A)
    for c in range(len(S)):
        e = np.zeros_like(S)
        e[c] = 1e-5
        J[:, c] = (_Kvec(p, *Wv.unpack(p, S + e)) - _Kvec(p, *Wv.unpack(p, S - e))) / 2e-5
    np.testing.assert_allclose(A, J, rtol=1e-6, atol=1e-8 * np.abs(A).max())


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_v6_elimination_solves_Fx_and_its_transpose(bc):
    p = Wv.WaveProblem(small(dim=2, m=5, N=2, bc=bc))
    X, U, L = _perturbed(p, 3)
    low = Wv.StageLower(p, X, U, L, 0, n_lo=200, n_u_it=1)
    Fx = p.h * p.fx(X[0], U[0]) - np.eye(p.nx)
    # the paper's block form of F_x
    n = p.ng
    np.testing.assert_allclose(Fx[:n, :n], -np.eye(n))
    np.testing.assert_allclose(Fx[:n, n:], p.h * np.eye(n))
    b = np.random.default_rng(4).standard_normal(p.nx)
    np.testing.assert_allclose(low.fx_solve(b), np.linalg.solve(Fx, b), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(low.fxT_solve(b), np.linalg.solve(Fx.T, b), rtol=1e-10, atol=1e-12)
    if bc == "neumann":   # a non-symmetric Laplacian: E and E^T differ
        assert np.abs(low.E - low.E.T).max() > 1e-3


def test_lower_layer_with_many_sweeps_is_the_dense_stage_solve():
    p = Wv.WaveProblem(small(dim=2, m=5, N=3))
    X, U, L = _perturbed(p, 5)
    K1, K2, K3 = Wv.kkt(p, X, U, L)
    for i in (0, p.N - 1):
        D = Wv.stage_block(p, X, U, L, i)
        d = np.linalg.solve(D, np.concatenate([K1[i], K2[i], K3[i]]))
        dx, du, dl = Wv.StageLower(p, X, U, L, i, n_lo=200, n_u_it=200).solve(K1[i], K3[i], K2[i])
        tol = 1e-9 * np.abs(d).max()
        np.testing.assert_allclose(dx, d[:p.nx], atol=tol)
        np.testing.assert_allclose(du, d[p.nx:p.nx + p.nu], atol=tol)
        np.testing.assert_allclose(dl, d[p.nx + p.nu:], atol=tol)


@pytest.fixture(scope="module")
def wave_root():
    p = Wv.WaveProblem(small(dim=1, m=8, N=4, seed=3))
    (X, U, L), hist = Wv.newton_solve(p, tol=1e-12)
    assert hist[-1] <= 1e-12
    # quadratic convergence over the last steps
    assert hist[-1] <= 1e-3 * hist[-2] or hist[-2] <= 1e-9
    return p, X, U, L


def test_newton_root_minimises_the_reduced_nlp(wave_root):
    p, X, U, L = wave_root
    np.testing.assert_allclose(Wv.simulate(p, U), X, rtol=1e-9, atol=1e-11)
    J0 = Wv.reduced_cost(p, U)
    g, g0 = np.zeros_like(U), np.zeros_like(U)
    Uc = p.cold_start()[1]
    for i in range(p.N):
        for a in range(p.nu):
            E = np.zeros_like(U); E[i, a] = 1e-4
            g[i, a] = (Wv.reduced_cost(p, U + E) - Wv.reduced_cost(p, U - E)) / 2e-4
            g0[i, a] = (Wv.reduced_cost(p, Uc + E) - Wv.reduced_cost(p, Uc - E)) / 2e-4
    assert np.abs(g).max() <= 1e-6 * np.abs(g0).max()
    rng = np.random.default_rng(4)
    for _ in range(5):
        assert Wv.reduced_cost(p, U + 0.05 * rng.standard_normal(U.shape)) > J0


def test_linear_quadratic_case_is_solved_by_one_newton_step():
    p = Wv.WaveProblem(small(dim=1, m=7, N=4, kappa=0.0))
    X, U, L = _perturbed(p, 6, 0.3, 2.0, 0.3)
    (Xn, Un, Ln), hist = Wv.newton_solve(p, S0=(X, U, L), tol=0.0, max_iter=2)
    assert hist[0] > 1e-2 and hist[1] <= 1e-11


@pytest.mark.parametrize("variant", ["jacobi", "fgs", "bgs", "sgs", "redblack"])
def test_sweeps_with_exact_stage_solves_are_their_matrix_definitions(variant):
    p = Wv.WaveProblem(small(dim=1, m=5, N=4))
    X, U, L = _perturbed(p, 7)
    A = Wv.kkt_matrix(p, X, U, L, with_gamma=True)
    n = 2 * p.nx + p.nu
    D = np.zeros_like(A)
    for i in range(p.N):
        D[i * n:(i + 1) * n, i * n:(i + 1) * n] = A[i * n:(i + 1) * n, i * n:(i + 1) * n]
    Lo, Up = np.tril(A - D), np.triu(A - D)
    Kp = _Kvec(p, X, U, L)
    if variant == "jacobi":
        d = np.linalg.solve(D, Kp)
    elif variant == "fgs":
        d = np.linalg.solve(D + Lo, Kp)
    elif variant == "bgs":
        d = np.linalg.solve(D + Up, Kp)
    elif variant == "sgs":
        d = np.linalg.solve(D + Lo, Kp - Up @ np.linalg.solve(D + Up, Kp))
    else:
        Lrb = np.zeros_like(A)
        for i in range(1, p.N, 2):
            for j in (i - 1, i + 1):
                if 0 <= j < p.N:
                    Lrb[i * n:(i + 1) * n, j * n:(j + 1) * n] = (Lo + Up)[i * n:(i + 1) * n, j * n:(j + 1) * n]
        d = np.linalg.solve(D + Lrb, Kp)
    Xe, Ue, Le = Wv.unpack(p, Wv.pack(p, X, U, L) - d)
    Xg, Ug, Lg, _ = Wv.iteration(p, X, U, L, variant, exact_inner=True)
    for g_, e in ((Xg, Xe), (Ug, Ue), (Lg, Le)):
        np.testing.assert_allclose(g_, e, rtol=1e-9, atol=1e-10 * np.abs(e).max())


def test_single_stage_jacobi_with_exact_stage_solve_is_newton():
    p = Wv.WaveProblem(small(dim=1, m=6, N=1))
    X, U, L = _perturbed(p, 8)
    Kp = _Kvec(p, X, U, L)
    d = np.linalg.solve(Wv.kkt_matrix(p, X, U, L, with_gamma=True), Kp)
    Xe, Ue, Le = Wv.unpack(p, Wv.pack(p, X, U, L) - d)
    Xg, Ug, Lg, _ = Wv.iteration(p, X, U, L, "jacobi", exact_inner=True)
    np.testing.assert_allclose(Xg, Xe, atol=1e-12)
    np.testing.assert_allclose(Ug, Ue, atol=1e-12)
    np.testing.assert_allclose(Lg, Le, atol=1e-12)


def test_theorem_3_red_black_radius_is_the_jacobi_radius_squared(wave_root):
    """The linearization of Theorem 1 (u~ fixed at u*, so gamma sits in the
    matrix): the KKT matrix is block tridiagonal, hence consistently ordered,
    and the red-black splitting's radius is rho_J^2."""
    p, X, U, L = wave_root
    A = Wv.kkt_matrix(p, X, U, L, with_gamma=True)
    n = 2 * p.nx + p.nu
    D = np.zeros_like(A)
    for i in range(p.N):
        D[i * n:(i + 1) * n, i * n:(i + 1) * n] = A[i * n:(i + 1) * n, i * n:(i + 1) * n]
    R = A - D
    Lrb = np.zeros_like(A)
    for i in range(1, p.N, 2):
        for j in (i - 1, i + 1):
            if 0 <= j < p.N:
                Lrb[i * n:(i + 1) * n, j * n:(j + 1) * n] = R[i * n:(i + 1) * n, j * n:(j + 1) * n]
    rho = lambda M: float(np.abs(np.linalg.eigvals(M)).max())
    rj = rho(np.linalg.solve(D, R))
    assert 0.05 < rj < 1.0
    assert rho(np.linalg.solve(D + Lrb, R - Lrb)) == pytest.approx(rj ** 2, rel=1e-7)
    assert rho(np.linalg.solve(D + np.tril(R), np.triu(R))) == pytest.approx(rj ** 2, rel=1e-7)


@pytest.mark.parametrize("variant", ["jacobi", "redblack", "sgs"])
def test_iterations_reach_the_newton_root(wave_root, variant):
    p, X, U, L = wave_root
    (Xv, Uv, Lv), info = Wv.solve(p, variant, tol=1e-11, max_iter=3000)
    assert info["converged"], info["res_inf"]
    # ||K||_inf <= 1e-11 bounds the distance to the root by ||A^-1|| 1e-11
    np.testing.assert_allclose(Uv, U, rtol=0, atol=1e-6 * np.abs(U).max())
    np.testing.assert_allclose(Xv, X, rtol=0, atol=1e-6 * np.abs(X).max())


def test_plant_converges_to_the_standing_wave_at_first_order():
    """With b = kappa = 0 and no input, a discrete eigenmode v of L (L v = mu
    v) released at rest oscillates as cos(omega t) v, omega^2 = -c mu / a.
    The plant's symplectic Euler steps converge to it at first order (the
    error halves with twice the sub-steps) and never grow in amplitude."""
    inst = small(dim=1, m=15, N=2, b=0.0, kappa=0.0)
    p = Wv.WaveProblem(inst)
    xs = np.arange(1, p.m + 1) / (p.m + 1)
    v = np.sin(np.pi * xs)
    mu = -(4 * (p.m + 1) ** 2) * np.sin(np.pi / (2 * (p.m + 1))) ** 2
    omega = np.sqrt(-p.c * mu / p.a)
    t = 1.3 * 2 * np.pi / omega          # 1.3 periods
    x0 = np.concatenate([v, np.zeros(p.ng)])
    exact = np.cos(omega * t) * v
    errs = []
    for n_sub in (200, 400, 800):
        x = Wv.plant_step(p, x0, np.zeros(p.nu), t, n_sub)
        errs.append(np.abs(x[:p.ng] - exact).max())
        assert np.abs(x[:p.ng]).max() <= 1.01  # no growth
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2, errs


def test_plant_damping_and_forces():
    """Damping b > 0 makes the energy a/2 |V|^2 - c/2 W.L W fall step by step
    (no input, kappa = 0); a constant force on an actuator cell accelerates
    that cell first (its V grows by tau gain u / a in the first sub-step)."""
    inst = small(dim=1, m=15, N=2, b=2.0, kappa=0.0)
    p = Wv.WaveProblem(inst)
    rng = np.random.default_rng(1)
    x = np.concatenate([0.1 * rng.standard_normal(p.ng), np.zeros(p.ng)])
    energy = lambda y: 0.5 * p.a * y[p.ng:] @ y[p.ng:] - 0.5 * p.c * y[:p.ng] @ (p.L @ y[:p.ng])
    e = [energy(x)]
    for _ in range(20):
        x = Wv.plant_step(p, x, np.zeros(p.nu), 1e-3, 1)
        e.append(energy(x))
    assert all(e[k + 1] < e[k] for k in range(len(e) - 1))
    x1 = Wv.plant_step(p, np.zeros(2 * p.ng), np.array([1.0] + [0.0] * (p.nu - 1)), 1e-4, 1)
    V = x1[p.ng:]
    assert V[p.act[0]] == pytest.approx(1e-4 * p.gain / p.a)
    assert np.abs(np.delete(V, p.act[0])).max() == 0.0
