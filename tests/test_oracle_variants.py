"""Pins of the oracle's Jacobi-type variants (Sec. 4.2, eqs. 18-20).

* With exact stage solves, one oracle sweep equals its matrix definition
  written with dense matrices assembled from the KKT matrix of eq. 10:
  FGS S - (D + L)^{-1} K (eq. 18), BGS S - (D + U)^{-1} K, SGS
  S - (D + L)^{-1}(K - U (D + U)^{-1} K) (eq. 20), red-black S - (D + L_rb)^{-1} K
  with L_rb the couplings of odd stages to even ones.
* Theorem 3: the KKT matrix is block tridiagonal, hence consistently ordered,
  so rho((D* + L)^{-1} U) = rho((D* + U)^{-1} L) = rho(D*^{-1}(L + U))^2, and
  the same holds for the red-black order; the oracle's sweeps then converge
  at that factor (Lemma 3), checked near the root with u~ fixed at u*.
* With the lower layer (inexact stage solves) every variant reaches the
  Newton root, and the Gauss-Seidel variants need about half the Jacobi
  iterations.
"""
import numpy as np
import pytest

from oracle import nmpc as O
from paper_2004_02484_gb300 import workloads as wl


def _perturbed(p, seed=0, sx=0.05, su=0.5, sl=0.01):
    rng = np.random.default_rng(seed)
    X, U, L = p.cold_start()
    return (X + sx * rng.standard_normal(X.shape), U + su * rng.standard_normal(U.shape),
            L + sl * rng.standard_normal(L.shape))


def _blocks(p, X, U, L):
    """Dense D (block diagonal), L (lower couplings), U (upper couplings) of
    the iteration matrix (gamma in the u-blocks) and the packed K."""
    A = O.dense_kkt_matrix(p, X, U, L, with_gamma=True)
    n = 2 * p.ng + p.nu
    D = np.zeros_like(A)
    for i in range(p.N):
        D[i * n:(i + 1) * n, i * n:(i + 1) * n] = A[i * n:(i + 1) * n, i * n:(i + 1) * n]
    Lo = np.tril(A - D)
    Up = np.triu(A - D)
    return D, Lo, Up, n


def _rb_lower(p, A_off, n):
    """Couplings of odd (0-based) stages to even ones: the block rows visited
    second take the already updated even neighbours."""
    M = np.zeros_like(A_off)
    for i in range(1, p.N, 2):
        for j in (i - 1, i + 1):
            if 0 <= j < p.N:
                M[i * n:(i + 1) * n, j * n:(j + 1) * n] = A_off[i * n:(i + 1) * n, j * n:(j + 1) * n]
    return M


MKS = [lambda: wl.tiny1d(m=6, horizon=5, n_u=1, seed=3),
       lambda: wl.tiny2d(mx=4, my=3, horizon=4, seed=4)]


@pytest.mark.parametrize("mk", MKS)
@pytest.mark.parametrize("variant", ["fgs", "bgs", "sgs", "redblack"])
def test_sweep_with_exact_stage_solves_is_its_matrix_definition(mk, variant):
    p = O.Problem(mk())
    X, U, L = _perturbed(p, 1)
    D, Lo, Up, n = _blocks(p, X, U, L)
    K = O.pack_kkt(p, *O.kkt(p, X, U, L))
    if variant == "fgs":
        d = np.linalg.solve(D + Lo, K)
    elif variant == "bgs":
        d = np.linalg.solve(D + Up, K)
    elif variant == "sgs":
        d = np.linalg.solve(D + Lo, K - Up @ np.linalg.solve(D + Up, K))
    else:
        d = np.linalg.solve(D + _rb_lower(p, Lo + Up, n), K)
    expect = O.unpack(p, O.pack(p, X, U, L) - 0.8 * d)
    got = O.variant_iteration(p, X, U, L, variant, alpha=0.8, exact_inner=True)[:3]
    for g, e in zip(got, expect):
        np.testing.assert_allclose(g, e, rtol=1e-9, atol=1e-12)


def _root(p):
    (X, U, L), hist = O.newton_solve(p, tol=1e-13)
    assert hist[-1] <= 1e-13
    return X, U, L


@pytest.mark.parametrize("mk", MKS)
def test_theorem3_gauss_seidel_factor_is_jacobi_squared(mk):
    p = O.Problem(mk())
    X, U, L = _root(p)
    D, Lo, Up, n = _blocks(p, X, U, L)
    rho = lambda M: float(np.abs(np.linalg.eigvals(M)).max())
    rj = rho(np.linalg.solve(D, Lo + Up))
    assert 0.05 < rj < 1.0
    Lrb = _rb_lower(p, Lo + Up, n)
    for M, Rst in ((D + Lo, Up), (D + Up, Lo), (D + Lrb, Lo + Up - Lrb)):
        np.testing.assert_allclose(rho(np.linalg.solve(M, Rst)), rj ** 2, rtol=1e-7)


@pytest.mark.parametrize("variant", ["fgs", "bgs", "redblack"])
def test_theorem3_observed_rate_of_the_oracle_sweeps(variant):
    """Near the root, with u~ fixed at u* (the linearization of Theorem 1),
    the error of the oracle's sweeps decays by rho_J^2 per iteration."""
    p = O.Problem(wl.tiny1d(m=6, horizon=5, n_u=1, seed=3))
    Xs, Us, Ls = _root(p)
    D, Lo, Up, n = _blocks(p, Xs, Us, Ls)
    rj = float(np.abs(np.linalg.eigvals(np.linalg.solve(D, Lo + Up))).max())
    rng = np.random.default_rng(5)
    X, U, L = (Xs + 1e-4 * rng.standard_normal(Xs.shape), Us + 1e-4 * rng.standard_normal(Us.shape),
               Ls + 1e-6 * rng.standard_normal(Ls.shape))
    errs = []
    for _ in range(66):
        X, U, L, _ = O.variant_iteration(p, X, U, L, variant, exact_inner=True, u_tilde=Us)
        errs.append(np.abs(O.pack(p, X, U, L) - O.pack(p, Xs, Us, Ls)).max())
    # the leading eigenvalues are complex, so single ratios oscillate: the
    # geometric mean over 60 sweeps (errors 1e-5 .. 1e-12, above round-off)
    rate = (errs[65] / errs[5]) ** (1.0 / 60)
    assert abs(rate - rj ** 2) <= 0.04 * rj ** 2, (rate, rj ** 2)
    # Jacobi on the same start decays by rho_J only
    X, U, L = (Xs + 1e-4 * rng.standard_normal(Xs.shape), Us + 1e-4 * rng.standard_normal(Us.shape),
               Ls + 1e-6 * rng.standard_normal(Ls.shape))
    e0 = None
    for k in range(66):
        X, U, L, _ = O.jacobi_iteration(p, X, U, L, exact_inner=True, u_tilde=Us)
        if k == 5:
            e0 = np.abs(O.pack(p, X, U, L) - O.pack(p, Xs, Us, Ls)).max()
    rate_j = (np.abs(O.pack(p, X, U, L) - O.pack(p, Xs, Us, Ls)).max() / e0) ** (1.0 / 60)
    assert abs(rate_j - rj) <= 0.04 * rj, (rate_j, rj)


@pytest.mark.parametrize("variant", ["fgs", "bgs", "sgs", "redblack"])
def test_variants_reach_the_newton_root_in_about_half_the_jacobi_iterations(variant):
    p = O.Problem(wl.heat1d(16, 12, 2, 0.01, seed=2))
    Xs, Us, Ls = _root(p)
    _, ij = O.solve_variant(p, "jacobi", tol=1e-11)
    (X, U, L), iv = O.solve_variant(p, variant, tol=1e-11)
    assert iv["converged"] and ij["converged"]
    # ||A^{-1}|| ~ 1e6 on this instance: a 1e-11 residual pins U to ~1e-5
    assert np.abs(U - Us).max() <= 1e-5 * np.abs(Us).max()
    assert iv["iters"] <= 0.65 * ij["iters"], (iv["iters"], ij["iters"])


def test_jacobi_through_the_variant_entry_is_eq15():
    p = O.Problem(wl.tiny2d())
    X, U, L = _perturbed(p, 2)
    a = O.variant_iteration(p, X, U, L, "jacobi")
    b = O.jacobi_iteration(p, X, U, L)
    for g, e in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(g, e)
