"""GPU parity of the pinned-actuator solver (include/nmpc_plate.h) against the
oracle (oracle/plate.py, pinned by tests/test_oracle_plate_pins.py): the
paper's copper plate (Sec. 5.1, Tables 1-2) with input bounds, the log
barrier (eq. 8) and the fraction-to-the-boundary step (eq. 11).

Everything is float64 on both sides, so one iteration agrees to a few ulps
of the largest term (1e-11 relative, scaled by each field's maximum), twelve
to 1e-10, and a solve follows the oracle's iterate sequence: the same
iteration count and controls within 1e-9 relative.
"""
import numpy as np
import pytest

from oracle import plate as P
from paper_2004_02484_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def GP():
    from paper_2004_02484_gb300 import build as b
    b.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2004_02484_gb300 import plate as GP
    return GP


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _start(p, seed):
    """A perturbed cold start: states +- 15 K on the plate (0.05 on the unit
    1D problem), inputs spread inside the bounds, small multipliers."""
    rng = np.random.default_rng(seed)
    X, U, L = p.cold_start()
    if p.tau > 0:
        X = X + 15.0 * rng.standard_normal(X.shape)
        U = rng.uniform(p.u_lo + 20.0, p.u_hi - 20.0, U.shape)
    else:
        X = X + 0.05 * rng.standard_normal(X.shape)
        U = U + 0.3 * rng.standard_normal(U.shape)
    L = L + 1e-3 * rng.standard_normal(L.shape)
    return X, U, L


def _first_cut(p, variant):
    """The first iterate of the oracle's cold-started solve whose step the
    fraction-to-the-boundary rule shortens (alpha < 1)."""
    X, U, L = p.cold_start()
    for _ in range(200):
        _, _, _, _, a = P.iteration(p, X, U, L, variant)
        if a < 1.0:
            return X, U, L
        X, U, L, _, _ = P.iteration(p, X, U, L, variant)
    raise AssertionError("no shortened step")


CASES = {
    "plate_7x7_N4": lambda: [wl.plate_instance(m=7, horizon=4, T=20.0, act_idx=(1, 4))],
    "plate_13x13_N20": lambda: [wl.plate_instance()],
    "plate_batch_3": lambda: wl.plate_batch(3, m=9, horizon=6, act_idx=(1, 4, 7)),
    "pinned_1d_dirichlet": lambda: [wl.pinned_heat1d(m=16, horizon=5, h=1e-3, r=1.0)],
}


def _gpu_iter(GP, insts, states, n_iter, **opts):
    s = GP.PlateSolver(insts, **opts)
    pk = lambda A: np.concatenate([a.reshape(-1) for a in A])
    x, u, lam = _t(pk([st[0] for st in states])), _t(pk([st[1] for st in states])), \
        _t(pk([st[2] for st in states]))
    (xo, uo, lo), out = s.iterate(x, u, lam, n_iter)
    res = (xo.cpu().numpy(), uo.cpu().numpy(), lo.cpu().numpy())
    s.close()
    outs, ox, ou = [], 0, 0
    for inst in insts:
        ns, nu, N = inst.ns, len(inst.act), inst.horizon
        outs.append((res[0][ox:ox + N * ns].reshape(N, ns), res[1][ou:ou + N * nu].reshape(N, nu),
                     res[2][ox:ox + N * ns].reshape(N, ns)))
        ox += N * ns
        ou += N * nu
    return outs, out


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("variant,oracle_variant", [(0, "jacobi"), (1, "redblack")])
@pytest.mark.parametrize("n_iter,rtol", [(1, 1e-11), (12, 1e-10)])
def test_iterations_match_the_oracle(GP, case, variant, oracle_variant, n_iter, rtol):
    insts = CASES[case]()
    probs = [P.PinnedProblem(i) for i in insts]
    states = [_start(p, 10 + b) for b, p in enumerate(probs)]
    gpu, out = _gpu_iter(GP, insts, states, n_iter, variant=variant)
    for b, p in enumerate(probs):
        X, U, L = states[b]
        for _ in range(n_iter):
            X, U, L, nm, a = P.iteration(p, X, U, L, oracle_variant)
        for g, o in zip(gpu[b], (X, U, L)):
            err = np.abs(g - o).max() / max(np.abs(o).max(), 1e-300)
            assert err <= rtol, (b, err)
        assert abs(out[b, 0] - nm[0]) <= 1e-11 * nm[0]
        assert abs(out[b, 2] - a) <= 1e-12


@pytest.mark.parametrize("case", ["plate_7x7_N4", "plate_13x13_N20"])
@pytest.mark.parametrize("variant,oracle_variant", [(0, "jacobi"), (1, "redblack")])
def test_fraction_to_the_boundary_step_matches(GP, case, variant, oracle_variant):
    """From the first iterate whose step the bounds shorten (alpha < 1): the
    GPU's alpha and next iterate equal the oracle's, inside the bounds."""
    insts = CASES[case]()
    p = P.PinnedProblem(insts[0])
    st = _first_cut(p, oracle_variant)
    X, U, L, _, a_or = P.iteration(p, *st, oracle_variant)
    assert a_or < 1.0
    gpu, out = _gpu_iter(GP, insts, [st], 1, variant=variant)
    assert abs(out[0, 2] - a_or) <= 1e-12
    for g, o in zip(gpu[0], (X, U, L)):
        assert np.abs(g - o).max() <= 1e-11 * np.abs(o).max()
    assert np.all(gpu[0][1] > p.u_lo) and np.all(gpu[0][1] < p.u_hi)


@pytest.mark.parametrize("case", ["plate_7x7_N4", "plate_13x13_N20", "plate_batch_3",
                                  "pinned_1d_dirichlet"])
@pytest.mark.parametrize("variant,oracle_variant", [(0, "jacobi"), (1, "redblack")])
def test_solve_follows_the_oracle_iterates(GP, case, variant, oracle_variant):
    import torch
    insts = CASES[case]()
    s = GP.PlateSolver(insts, tol=1e-6, variant=variant, max_iter=3000)
    rc, st = s.solve()
    torch.cuda.synchronize()
    u = s.u.cpu().numpy()
    s.close()
    assert rc == 0
    ou = 0
    for b, inst in enumerate(insts):
        p = P.PinnedProblem(inst)
        (X, U, L), info = P.solve(p, oracle_variant, tol=1e-6, max_iter=3000)
        assert info["converged"]
        assert st[b].iters == info["iters"], (b, st[b].iters, info["iters"])
        nu, N = len(inst.act), inst.horizon
        ug = u[ou:ou + N * nu].reshape(N, nu)
        assert np.abs(ug - U).max() <= 1e-9 * np.abs(U).max()
        assert np.all(ug > p.u_lo) and np.all(ug < p.u_hi)
        ou += N * nu


def test_redblack_needs_fewer_iterations_on_the_paper_plate(GP):
    import torch
    insts = [wl.plate_instance()]
    its = []
    for variant in (0, 1):
        s = GP.PlateSolver(insts, tol=1e-6, variant=variant)
        rc, st = s.solve()
        torch.cuda.synchronize()
        s.close()
        assert rc == 0
        its.append(st[0].iters)
    assert its[1] < its[0], its


def test_closed_loop_matches_the_oracle(GP):
    """The receding-horizon use (Sec. 5.3) on a 9x9 plate, 3 periods, each
    solve to 1e-9 from the previous solution shifted by one stage: the GPU
    loop and the oracle's apply the same first-stage inputs and their plants
    reach the same state."""
    import copy
    import torch
    inst = wl.plate_instance(m=9, horizon=6, T=30.0, act_idx=(1, 4, 7))
    steps, nu = 3, 9
    s = GP.PlateSolver([inst], tol=1e-9, max_iter=20000)
    w = _t(inst.x0)
    u_hist = torch.zeros(steps * nu, dtype=torch.float64, device="cuda")
    rc, iters, res = s.closed_loop(w, steps, 1, u_hist)
    torch.cuda.synchronize()
    s.close()
    assert rc == 0 and np.all(res <= 1e-9)
    uh = u_hist.cpu().numpy().reshape(steps, nu)
    x = np.asarray(inst.x0, dtype=np.float64).copy()
    S = None
    for t in range(steps):
        cur = copy.copy(inst)
        cur.x0 = x.copy()
        p = P.PinnedProblem(cur)
        (X, U, L), info = P.solve(p, "jacobi", S0=S, tol=1e-9, max_iter=20000)
        assert info["converged"]
        assert abs(int(iters[t, 0]) - info["iters"]) <= 1, (t, iters[t, 0], info["iters"])
        assert np.abs(uh[t] - U[0]).max() <= 1e-7 * np.abs(U[0]).max()
        x = P.plant_step(p, x, U[0], p.h, 1)
        S = tuple(np.vstack([A[1:], A[-1:]]) for A in (X, U, L))
    assert np.abs(w.cpu().numpy() - x).max() <= 1e-7 * np.abs(x).max()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("variant,oracle_variant", [(0, "jacobi"), (1, "redblack")])
def test_mixed_iteration_matches_the_oracle(GP, case, variant, oracle_variant):
    """Float32 lower layer (NMPC_MIXED): one iteration's change agrees with the
    oracle's float64 change to 1e-4 of its size; the norms come from the
    float64 residual (1e-11)."""
    insts = CASES[case]()
    probs = [P.PinnedProblem(i) for i in insts]
    states = [_start(p, 30 + b) for b, p in enumerate(probs)]
    gpu, out = _gpu_iter(GP, insts, states, 1, variant=variant, precision=1)
    for b, p in enumerate(probs):
        X0, U0, L0 = states[b]
        X, U, L, nm, a = P.iteration(p, X0, U0, L0, oracle_variant)
        for g, o, i in zip(gpu[b], (X, U, L), (X0, U0, L0)):
            assert np.abs((g - i) - (o - i)).max() <= 1e-4 * np.abs(o - i).max(), b
        assert abs(out[b, 0] - nm[0]) <= 1e-11 * nm[0]
        assert abs(out[b, 2] - a) <= 1e-4


@pytest.mark.parametrize("variant", [0, 1])
def test_mixed_solve_reaches_the_float64_root(GP, variant):
    """NMPC_MIXED solves stop on the float64 residual and land on the float64
    root: controls within 1e-7 (relative) of the oracle's solve, about the
    same iteration count as the float64 GPU solve."""
    import torch
    insts = CASES["plate_batch_3"]() + CASES["plate_13x13_N20"]()
    its, us = {}, {}
    for prec in (0, 1):
        s = GP.PlateSolver(insts, tol=1e-6, variant=variant, precision=prec, max_iter=3000)
        rc, st = s.solve()
        torch.cuda.synchronize()
        assert rc == 0 and all(x.res_inf <= 1e-6 for x in st)
        its[prec] = [x.iters for x in st]
        us[prec] = s.u.cpu().numpy()
        s.close()
    ou = 0
    for b, inst in enumerate(insts):
        p = P.PinnedProblem(inst)
        (X, U, L), info = P.solve(p, "redblack" if variant else "jacobi", tol=1e-6, max_iter=3000)
        nu, N = len(inst.act), inst.horizon
        ug = us[1][ou:ou + N * nu].reshape(N, nu)
        assert np.abs(ug - U).max() <= 1e-7 * np.abs(U).max()
        assert abs(its[1][b] - its[0][b]) <= max(2, 0.05 * its[0][b]), (its[0][b], its[1][b])
        ou += N * nu
