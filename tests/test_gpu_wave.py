"""GPU parity of the second-order-in-time solver (include/nmpc_wave.h)
against the oracle (oracle/wave.py, pinned by tests/test_oracle_wave_pins.py):
a damped nonlinear string / membrane, state (W, dW/dt) (eq. 5), F_x and
F_x^T solved by eliminating v6 (eq. 25).

Both sides are float64: one iteration agrees to 1e-11 of each field's
largest entry, twelve to 1e-10, and a solve follows the oracle's iterate
sequence (the same iteration count, controls within 1e-9 relative).
"""
import numpy as np
import pytest

from oracle import wave as Wv
from paper_2004_02484_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def GW():
    from paper_2004_02484_gb300 import build as b
    b.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2004_02484_gb300 import wave as GW
    return GW


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _start(p, seed):
    rng = np.random.default_rng(seed)
    X, U, L = p.cold_start()
    return (X + 0.05 * rng.standard_normal(X.shape), U + 0.5 * rng.standard_normal(U.shape),
            L + 0.01 * rng.standard_normal(L.shape))


CASES = {
    "string_m64_N20": lambda: [wl.wave_instance()],
    "membrane_16x16_N10": lambda: [wl.wave_instance(dim=2, m=16, horizon=10)],
    "string_neumann_m33_N8": lambda: [wl.wave_instance(m=33, horizon=8, T=0.024, bc="neumann")],
    "membrane_32x32_N4": lambda: [wl.wave_instance(dim=2, m=32, horizon=4, T=0.012, n_act=3)],
    "ragged_batch_4": lambda: [wl.wave_instance(m=40, horizon=7, T=0.021, seed=1),
                               wl.wave_instance(dim=2, m=9, horizon=1, T=0.003, seed=2),
                               wl.wave_instance(dim=2, m=12, horizon=6, bc="neumann", seed=3, a=2.0),
                               wl.wave_instance(m=5, horizon=3, T=0.009, seed=4, n_act=1)],
}


def _gpu_iter(GW, insts, states, n_iter, **opts):
    s = GW.WaveSolver(insts, **opts)
    pk = lambda A: np.concatenate([a.reshape(-1) for a in A])
    x, u, lam = _t(pk([st[0] for st in states])), _t(pk([st[1] for st in states])), \
        _t(pk([st[2] for st in states]))
    (xo, uo, lo), out = s.iterate(x, u, lam, n_iter)
    res = (xo.cpu().numpy(), uo.cpu().numpy(), lo.cpu().numpy())
    s.close()
    outs, ox, ou = [], 0, 0
    for inst in insts:
        nx, nu, N = 2 * inst.ng, len(inst.act), inst.horizon
        outs.append((res[0][ox:ox + N * nx].reshape(N, nx), res[1][ou:ou + N * nu].reshape(N, nu),
                     res[2][ox:ox + N * nx].reshape(N, nx)))
        ox += N * nx
        ou += N * nu
    return outs, out


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("variant,oracle_variant", [(0, "jacobi"), (1, "redblack")])
@pytest.mark.parametrize("n_iter,rtol", [(1, 1e-11), (12, 1e-10)])
def test_iterations_match_the_oracle(GW, case, variant, oracle_variant, n_iter, rtol):
    insts = CASES[case]()
    probs = [Wv.WaveProblem(i) for i in insts]
    states = [_start(p, 20 + b) for b, p in enumerate(probs)]
    gpu, out = _gpu_iter(GW, insts, states, n_iter, variant=variant)
    for b, p in enumerate(probs):
        X, U, L = states[b]
        for _ in range(n_iter):
            X, U, L, nm = Wv.iteration(p, X, U, L, oracle_variant)
        for g, o in zip(gpu[b], (X, U, L)):
            err = np.abs(g - o).max() / max(np.abs(o).max(), 1e-300)
            assert err <= rtol, (b, err)
        assert abs(out[b, 0] - nm[0]) <= 1e-11 * nm[0]
        assert abs(out[b, 1] - nm[1]) <= 1e-10 * nm[1]
        assert out[b, 2] == 1.0


@pytest.mark.parametrize("n_lo,n_u_it", [(1, 0), (1, 1), (3, 2), (4, 3)])
def test_inner_iteration_counts_match_the_oracle(GW, n_lo, n_u_it):
    insts = CASES["ragged_batch_4"]()
    probs = [Wv.WaveProblem(i) for i in insts]
    states = [_start(p, 40 + b) for b, p in enumerate(probs)]
    gpu, _ = _gpu_iter(GW, insts, states, 3, n_lo=n_lo, n_u_it=n_u_it)
    for b, p in enumerate(probs):
        X, U, L = states[b]
        for _ in range(3):
            X, U, L, _ = Wv.iteration(p, X, U, L, "jacobi", n_lo=n_lo, n_u_it=n_u_it)
        for g, o in zip(gpu[b], (X, U, L)):
            assert np.abs(g - o).max() <= 1e-10 * np.abs(o).max()


@pytest.mark.parametrize("case", ["string_m64_N20", "membrane_16x16_N10", "ragged_batch_4"])
@pytest.mark.parametrize("variant,oracle_variant", [(0, "jacobi"), (1, "redblack")])
def test_solve_follows_the_oracle_iterates(GW, case, variant, oracle_variant):
    import torch
    insts = CASES[case]()
    s = GW.WaveSolver(insts, tol=1e-8, variant=variant, max_iter=3000)
    rc, st = s.solve()
    torch.cuda.synchronize()
    u = s.u.cpu().numpy()
    x, _, _ = s.state()
    x = x.cpu().numpy()
    s.close()
    assert rc == 0
    ou = ox = 0
    for b, inst in enumerate(insts):
        p = Wv.WaveProblem(inst)
        (X, U, L), info = Wv.solve(p, oracle_variant, tol=1e-8, max_iter=3000)
        assert info["converged"]
        assert st[b].iters == info["iters"], (b, st[b].iters, info["iters"])
        nu, nx, N = len(inst.act), 2 * inst.ng, inst.horizon
        ug = u[ou:ou + N * nu].reshape(N, nu)
        assert np.abs(ug - U).max() <= 1e-9 * np.abs(U).max()
        xg = x[ox:ox + N * nx].reshape(N, nx)
        assert np.abs(xg - X).max() <= 1e-9 * np.abs(X).max()
        assert st[b].res_inf <= 1e-8
        ou += N * nu
        ox += N * nx


def test_redblack_needs_fewer_iterations(GW):
    import torch
    insts = [wl.wave_instance(), wl.wave_instance(dim=2, m=16, horizon=10)]
    its = []
    for variant in (0, 1):
        s = GW.WaveSolver(insts, tol=1e-8, variant=variant)
        rc, st = s.solve()
        torch.cuda.synchronize()
        s.close()
        assert rc == 0
        its.append([x.iters for x in st])
    assert all(r < 0.7 * j for j, r in zip(*its)), its


def test_warm_and_shifted_starts_use_the_returned_state(GW):
    """A warm restart from a converged state stops at once; a shifted one
    starts from the state moved by one stage (checked through one
    iteration against the oracle from that shifted state)."""
    import torch
    inst = wl.wave_instance(m=24, horizon=6, T=0.018)
    p = Wv.WaveProblem(inst)
    s = GW.WaveSolver([inst], tol=1e-9)
    rc, st = s.solve()
    assert rc == 0
    x, u, lam = (t.cpu().numpy().reshape(inst.horizon, -1) for t in s.state())
    rc, st = s.solve(init=1)
    assert rc == 0 and st[0].iters == 0
    S = tuple(np.vstack([A[1:], A[-1:]]) for A in (x, u, lam))
    s.close()
    s = GW.WaveSolver([inst], tol=0.0, max_iter=1)
    s.solve()
    # the handle now holds one iterate from cold; iterate from the shifted
    # state directly and compare with the oracle
    (xo, uo, lo), out = s.iterate(_t(S[0].reshape(-1)), _t(S[1].reshape(-1)), _t(S[2].reshape(-1)), 1)
    torch.cuda.synchronize()
    s.close()
    X, U, L, nm = Wv.iteration(p, *S, "jacobi")
    assert np.abs(uo.cpu().numpy().reshape(U.shape) - U).max() <= 1e-11 * np.abs(U).max()
    assert out[0, 0] == pytest.approx(nm[0], rel=1e-11)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("variant,oracle_variant", [(0, "jacobi"), (1, "redblack")])
def test_mixed_iteration_matches_the_oracle(GW, case, variant, oracle_variant):
    """Float32 lower layer (NMPC_MIXED): one iteration's change agrees with the
    oracle's float64 change to 1e-4 of its size; the norms come from the
    float64 residual (1e-11)."""
    insts = CASES[case]()
    probs = [Wv.WaveProblem(i) for i in insts]
    states = [_start(p, 60 + b) for b, p in enumerate(probs)]
    gpu, out = _gpu_iter(GW, insts, states, 1, variant=variant, precision=1)
    for b, p in enumerate(probs):
        X0, U0, L0 = states[b]
        X, U, L, nm = Wv.iteration(p, X0, U0, L0, oracle_variant)
        for g, o, i in zip(gpu[b], (X, U, L), (X0, U0, L0)):
            assert np.abs((g - i) - (o - i)).max() <= 1e-4 * np.abs(o - i).max(), b
        assert abs(out[b, 0] - nm[0]) <= 1e-11 * nm[0]


@pytest.mark.parametrize("variant", [0, 1])
def test_mixed_solve_reaches_the_float64_root(GW, variant):
    """NMPC_MIXED solves to 1e-9 stop on the float64 residual and land on the
    float64 root: controls within 1e-6 (relative) of the oracle's solve to
    the same tolerance, about the same iteration count as float64."""
    import torch
    insts = CASES["ragged_batch_4"]() + CASES["string_m64_N20"]()
    its, us = {}, {}
    for prec in (0, 1):
        s = GW.WaveSolver(insts, tol=1e-9, variant=variant, precision=prec, max_iter=5000)
        rc, st = s.solve()
        torch.cuda.synchronize()
        assert rc == 0 and all(x.res_inf <= 1e-9 for x in st)
        its[prec] = [x.iters for x in st]
        us[prec] = s.u.cpu().numpy()
        s.close()
    ou = 0
    for b, inst in enumerate(insts):
        p = Wv.WaveProblem(inst)
        (X, U, L), info = Wv.solve(p, "redblack" if variant else "jacobi", tol=1e-9, max_iter=5000)
        nu, N = len(inst.act), inst.horizon
        ug = us[1][ou:ou + N * nu].reshape(N, nu)
        assert np.abs(ug - U).max() <= 1e-6 * np.abs(U).max()
        assert abs(its[1][b] - its[0][b]) <= max(2, 0.05 * its[0][b]), (its[0][b], its[1][b])
        ou += N * nu


def test_closed_loop_matches_the_oracle(GW):
    """The receding-horizon use (Sec. 5.3) on a 24-point string, 4 periods,
    each solve to 1e-9 from the previous solution shifted by one stage, the
    plant 4 symplectic Euler steps per period: the GPU loop and the oracle's
    apply the same first-stage inputs and their plants reach the same state."""
    import torch
    inst = wl.wave_instance(m=24, horizon=6, T=0.018)
    steps, nu = 4, len(inst.act)
    s = GW.WaveSolver([inst], tol=1e-9, max_iter=20000)
    x = _t(inst.x0)
    u_hist = torch.zeros(steps * nu, dtype=torch.float64, device="cuda")
    rc, iters, res = s.closed_loop(x, steps, 4, u_hist)
    torch.cuda.synchronize()
    s.close()
    assert rc == 0 and np.all(res <= 1e-9)
    us, its, xf = Wv.closed_loop(inst, steps, 4, tol=1e-9)
    for t in range(steps):
        assert abs(int(iters[t, 0]) - int(its[t])) <= 1, (t, iters[t, 0], its[t])
    uh = u_hist.cpu().numpy().reshape(steps, nu)
    assert np.abs(uh - us).max() <= 1e-7 * np.abs(us).max()
    assert np.abs(x.cpu().numpy() - xf).max() <= 1e-8 * np.abs(xf).max()


def test_plant_step_matches_the_oracle(GW):
    """One plant call on a membrane (Neumann edges, 3 x 3 point forces) from a
    solved state: the same symplectic Euler sub-steps as the oracle's."""
    import torch
    inst = wl.wave_instance(dim=2, m=12, horizon=4, T=0.012, n_act=3, bc="neumann", seed=5)
    p = Wv.WaveProblem(inst)
    s = GW.WaveSolver([inst], tol=1e-8)
    rc, st = s.solve()
    assert rc == 0
    u1 = s.u.cpu().numpy().reshape(inst.horizon, -1)[0]
    x = _t(inst.x0)
    s.plant_step(x, 0.01, 7)
    torch.cuda.synchronize()
    s.close()
    xo = Wv.plant_step(p, inst.x0, u1, 0.01, 7)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-12 * max(1.0, np.abs(xo).max())
