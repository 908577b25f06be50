"""The C oracle (oracle/nmpc_oracle.c) against the numpy oracle (oracle/nmpc.py).

Both compute the same double-layer Jacobi iteration (eq. 15 with the lower
layer of eqs. 21-24 and the u-iteration of Sec. 5.2) in float64; the numpy
oracle is pinned to the paper's mathematics by tests/test_oracle_pins.py.
The C oracle is checked element by element against it on 1D and 2D
instances (several inner counts, stage counts and actuator layouts), through
complete solves (the same iteration count, the same iterate) and through the
closed-loop plant.  Tolerances: one iteration 1e-12 relative (the two differ
only in summation order); a complete solve 1e-10.
"""
import numpy as np
import pytest

from oracle import c_oracle as C
from oracle import nmpc as O
from paper_2004_02484_gb300 import workloads as wl


CASES = [
    lambda: wl.tiny1d(m=8, horizon=4, n_u=1),
    lambda: wl.heat1d(37, 9, 3, 0.02, seed=4),
    lambda: wl.tiny2d(),
    lambda: wl.heat2d(20, 18, 6, 2, 2, seed=5),
    lambda: wl.heat2d(33, 9, 5, 3, 1, seed=6, k1=0.0),
]


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def _start(p, seed):
    rng = np.random.default_rng(seed)
    X, U, L = p.cold_start()
    return (X + 0.05 * rng.standard_normal(X.shape), U + 0.5 * rng.standard_normal(U.shape),
            L + 0.01 * rng.standard_normal(L.shape))


@pytest.mark.parametrize("mk", CASES)
@pytest.mark.parametrize("n_lo,n_u_it", [(1, 1), (2, 2), (3, 1), (2, 3)])
def test_one_iteration_matches_numpy_oracle(mk, n_lo, n_u_it):
    inst = mk()
    po, pc = O.Problem(inst), C.Problem(inst)
    X, U, L = _start(po, 1)
    Xo, Uo, Lo, no = O.jacobi_iteration(po, X, U, L, n_lo=n_lo, n_u_it=n_u_it, alpha=0.7)
    Xc, Uc, Lc, nc = C.jacobi_iteration(pc, X, U, L, n_lo=n_lo, n_u_it=n_u_it, alpha=0.7)
    assert _rel(Xc, Xo) <= 1e-12 and _rel(Lc, Lo) <= 1e-12 and _rel(Uc, Uo) <= 1e-12
    assert abs(nc[0] - no[0]) <= 1e-12 * no[0] and abs(nc[1] - no[1]) <= 1e-12 * no[1]


@pytest.mark.parametrize("mk", CASES)
def test_kkt_norms_match(mk):
    inst = mk()
    po, pc = O.Problem(inst), C.Problem(inst)
    X, U, L = _start(po, 2)
    no = O.kkt_norms(*O.kkt(po, X, U, L))
    nc = C.kkt_norms(pc, X, U, L)
    assert abs(nc[0] - no[0]) <= 1e-13 * no[0] and abs(nc[1] - no[1]) <= 1e-12 * no[1]


@pytest.mark.parametrize("mk", [CASES[0], CASES[2], CASES[3]])
def test_complete_solve_matches_numpy_oracle(mk):
    inst = mk()
    (Xo, Uo, Lo), io = O.solve_jacobi(O.Problem(inst), tol=1e-10)
    (Xc, Uc, Lc), ic = C.solve_jacobi(C.Problem(inst), tol=1e-10)
    assert ic["converged"] and ic["iters"] == io["iters"]
    assert _rel(Uc, Uo) <= 1e-10 and _rel(Xc, Xo) <= 1e-10 and _rel(Lc, Lo) <= 1e-10


def test_nan_start_is_reported_diverged():
    inst = wl.tiny1d()
    p = C.Problem(inst)
    X, U, L = p.cold_start()
    X[1, 0, 3] = np.nan
    _, info = C.solve_jacobi(p, S0=(X, U, L), tol=1e-8)
    assert info["diverged"] and not info["converged"] and info["iters"] == 0


def test_max_iter_returns_the_last_iterate():
    inst = wl.tiny2d()
    (_, Uo, _), io = O.solve_jacobi(O.Problem(inst), tol=1e-14, max_iter=3)
    (_, Uc, _), ic = C.solve_jacobi(C.Problem(inst), tol=1e-14, max_iter=3)
    assert io["iters"] == ic["iters"] == 3 and not ic["converged"]
    assert _rel(Uc, Uo) <= 1e-12


@pytest.mark.parametrize("n_sub", [1, 3])
def test_plant_step_matches(n_sub):
    inst = wl.heat2d(20, 18, 6, 2, 2, seed=8)
    po, pc = O.Problem(inst), C.Problem(inst)
    u1 = np.array([0.3, -0.2, 0.5, 0.1])
    wo = O.plant_step(po, inst.x0, u1, 3e-5, n_sub).ravel()
    wc = C.plant_step(pc, inst.x0, u1, 3e-5, n_sub)
    assert _rel(wc, wo) <= 1e-14


def test_closed_loop_matches():
    inst = wl.heat1d(24, 6, 2, 0.01, seed=9)
    Uo, Wo, io = O.closed_loop(inst, 3, 2, tol=1e-10)
    Uc, Wc, ic = C.closed_loop(inst, 3, 2, tol=1e-10)
    assert io == ic
    assert _rel(Uc, Uo) <= 1e-9 and _rel(Wc, Wo) <= 1e-12
