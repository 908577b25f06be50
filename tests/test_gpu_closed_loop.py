"""Closed loop (receding horizon) on the GPU against the oracle's closed loop.

Each step the GPU solves from the shifted previous solution and the oracle
from the cold start; both stop at ||K||_inf <= 1e-10 in float64, so the
first-stage controls agree to the root's conditioning (~1e-10 / (h r) in the
u-row, relative 1e-6 here), and the explicit-Euler plant trajectories agree
to the same level.  Compared: u_1 per step and the plant state after the
last step, relative 1e-5.
"""
import numpy as np
import pytest

from oracle import nmpc as O
from paper_2004_02484_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2004_02484_gb300 import build as b
    b.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2004_02484_gb300 import nmpc as G
    return G


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("precision", [0, 1])
def test_closed_loop_matches_oracle(G, precision):
    import torch
    insts = [wl.heat2d(20, 18, 8, 2, 2, seed=51), wl.heat1d(40, 10, 3, 0.02, seed=52)]
    steps, n_sub = 6, 2
    s = G.Solver(insts, tol=1e-10, precision=precision, max_iter=20000)
    w = _t(G.pack_fields(insts, "x0"))
    nu_tot = sum(len(i.act) for i in insts)
    u_hist = torch.zeros(steps * nu_tot, dtype=torch.float64, device="cuda")
    rc, iters, res = G.nmpc_closed_loop(s.h, w, s.ref, steps, n_sub, len(insts), u_hist)
    torch.cuda.synchronize()
    assert rc == G.NMPC_OK and np.all(res <= 1e-10)
    uh = u_hist.cpu().numpy().reshape(steps, nu_tot)
    wg = w.cpu().numpy()
    o_u, o_w = 0, 0
    for inst in insts:
        U1, W, its = O.closed_loop(inst, steps, n_sub, tol=1e-10)
        nu, ng = len(inst.act), inst.mx * inst.my
        gu = uh[:, o_u:o_u + nu]
        assert np.abs(gu - U1).max() <= 1e-5 * np.abs(U1).max()
        gw = wg[o_w:o_w + ng]
        assert np.abs(gw - W[-1]).max() <= 1e-5 * np.abs(W[-1]).max()
        o_u += nu
        o_w += ng
    # the shifted warm start needs fewer iterations than the first, cold solve
    assert iters[1:].mean() < iters[0].mean()
    s.close()


def test_plant_step_matches_oracle_at_full_size(G):
    """One explicit-Euler plant step of the 64-instance 256x256 workload's first
    two instances (the kernel is the same at any batch size)."""
    import torch
    insts = wl.heat2d_large_batch(n=2)
    s = G.Solver(insts, tol=1e-3, precision=1, max_iter=3)
    s.solve()
    x, u, lam = s.state()
    w = s.x0.clone()
    G.nmpc_plant_step(s.h, w, 0.0, 2)
    torch.cuda.synchronize()
    wg = w.cpu().numpy()
    ug = u.cpu().numpy()
    o_w, o_u = 0, 0
    for inst in insts:
        p = O.Problem(inst)
        ng, nu, N = inst.mx * inst.my, len(inst.act), inst.horizon
        wo = O.plant_step(p, inst.x0, ug[o_u:o_u + nu], inst.h, 2).ravel()
        assert np.abs(wg[o_w:o_w + ng] - wo).max() <= 1e-12 * max(1.0, np.abs(wo).max())
        o_w += ng
        o_u += N * nu
    s.close()


@pytest.mark.parametrize("n_sub", [1, 2])
def test_graph_closed_loop_equals_host_driven_loop(G, n_sub):
    """The closed loop captured as one graph (nested WHILE nodes over steps and
    over chunks of iterations) performs the same operations as the loop driven
    from the host: identical controls, plant state, iterations and residuals."""
    import torch
    insts = [wl.heat2d(20, 18, 8, 2, 2, seed=61), wl.heat1d(40, 10, 3, 0.02, seed=62)]
    steps = 4
    out = []
    for use_graph in (1, 0):
        s = G.Solver(insts, tol=1e-8, precision=1, max_iter=5000, use_graph=use_graph)
        w = _t(G.pack_fields(insts, "x0"))
        nu_tot = sum(len(i.act) for i in insts)
        u_hist = torch.zeros(steps * nu_tot, dtype=torch.float64, device="cuda")
        rc, iters, res = G.nmpc_closed_loop(s.h, w, s.ref, steps, n_sub, len(insts), u_hist)
        torch.cuda.synchronize()
        out.append((rc, iters.copy(), res.copy(), u_hist.cpu().numpy(), w.cpu().numpy()))
        s.close()
    a, b = out
    assert a[0] == b[0] == G.NMPC_OK
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])
    assert np.array_equal(a[3], b[3])
    assert np.array_equal(a[4], b[4])


def test_pool_and_start_state_match_their_definitions(G):
    """nmpc_pool_avg is the f x f block mean; nmpc_start_state writes the cold
    start (x_i = x0, u = 0, lambda = 0) and the receding-horizon shift (stage i
    takes stage i + 1, the last repeated) of the handle's state."""
    import torch
    from paper_2004_02484_gb300 import mlp as GM
    insts = [wl.heat2d(32, 24, 5, 2, 2, seed=71), wl.heat2d(32, 24, 5, 2, 2, seed=72)]
    s = G.Solver(insts, tol=1e-6, precision=1, max_iter=2000)
    B, ng = 2, 32 * 24
    f = torch.empty((B, (32 // 4) * (24 // 4)), dtype=torch.float32, device="cuda")
    GM.nmpc_pool_avg(s.x0, f, B, 32, 24, 4)
    x0 = s.x0.cpu().numpy().reshape(B, 24, 32)
    want = x0.reshape(B, 6, 4, 8, 4).mean(axis=(2, 4)).reshape(B, -1)
    assert np.abs(f.cpu().numpy() - want).max() <= 1e-6 * np.abs(want).max()
    x = torch.empty(s.n_s, dtype=torch.float64, device="cuda")
    lam = torch.empty_like(x)
    u = torch.empty(s.n_u, dtype=torch.float64, device="cuda")
    G.nmpc_start_state(s.h, G.NMPC_INIT_COLD, s.x0, x, u, lam)
    assert np.array_equal(x.cpu().numpy().reshape(B, 5, ng), np.repeat(x0.reshape(B, 1, ng), 5, 1))
    assert not u.cpu().numpy().any() and not lam.cpu().numpy().any()
    s.solve()
    xs, us, ls = s.state()
    G.nmpc_start_state(s.h, G.NMPC_INIT_SHIFT, None, x, u, lam)
    X, L, U = (a.cpu().numpy() for a in (xs, ls, us))
    for arr, got, per in ((X, x, ng), (L, lam, ng), (U, u, 4)):
        a = arr.reshape(B, 5, per)
        want = np.concatenate([a[:, 1:], a[:, -1:]], axis=1)
        assert np.array_equal(got.cpu().numpy().reshape(B, 5, per), want)
    s.close()


def test_learned_closed_loop_keeps_the_better_start_and_converges(G):
    """The learned closed loop (network on pooled inputs, per-instance choice
    of the start with the smaller float64 residual) solves every step to the
    tolerance, and every chosen start's residual is the smaller one."""
    import torch
    from paper_2004_02484_gb300 import warmstart as WS
    train = wl.heat2d_large_batch(n=4, base_seed=7000, m=32, horizon=10)
    X, U = WS.closed_loop_data(train, 4, 2)
    lcs = WS.LearnedControlStart(train[0], pool=4, max_batch=16)
    losses = lcs.fit(X, U, steps=200, batch=16)
    assert losses[-1] < losses[0]
    test = wl.heat2d_large_batch(n=2, base_seed=5000, m=32, horizon=10)
    s = G.Solver(test, tol=1e-6, precision=1, max_iter=4000)
    w = s.x0.clone()
    out = WS.closed_loop_learned(s, lcs, w, 3, 2, rule="residual", decode="rollout")
    x, u, lam = s.state()
    r = G.nmpc_residual(s.h, w, s.ref, x, u, lam, 2)  # the last step's solution, plant moved on
    chosen = out["learned"].astype(bool)
    best = np.where(chosen, out["res_learned"], out["res_plain"])
    assert np.all(best <= np.minimum(out["res_learned"], out["res_plain"]))
    assert out["iters"].shape == (3, 2) and np.all(out["iters"] > 0)
    s.close()


@pytest.mark.parametrize("precision,rtol", [(0, 1e-12), (1, 2e-6)])
def test_rollout_matches_its_definition(G, precision, rtol):
    """nmpc_rollout: explicit-Euler state trajectory of u from x0 and the
    costate recursion lambda_i = lambda_{i+1} + h (q (x_i - ref) + Phi'(x_i)
    Lap lambda_{i+1}) from lambda_{N+1} = h qf (x_N - ref), written out here
    with the oracle's model terms, on a ragged 2D + 1D batch: to float64
    rounding on an FP64 handle, to float32 rounding accumulated over the
    stages (relative 2e-6 of each field's scale) on a MIXED one."""
    import torch
    insts = [wl.heat2d(20, 18, 7, 3, 3, seed=81), wl.heat1d(40, 11, 2, 0.02, seed=82)]
    s = G.Solver(insts, tol=1e-6, precision=precision, max_iter=2000)
    rng = np.random.default_rng(83)
    u = _t(rng.normal(0.0, 0.3, s.n_u))
    x = torch.empty(s.n_s, dtype=torch.float64, device="cuda")
    lam = torch.empty_like(x)
    G.nmpc_rollout(s.h, s.x0, s.ref, u, x, lam)
    torch.cuda.synchronize()
    Us = G.split_stages(insts, u.cpu().numpy(), "nu")
    Xs = G.split_stages(insts, x.cpu().numpy(), "ng")
    Ls = G.split_stages(insts, lam.cpu().numpy(), "ng")
    for inst, Ub, Xb, Lb in zip(insts, Us, Xs, Ls):
        p = O.Problem(inst)
        X = np.empty((p.N,) + p.shape)
        prev = p.x0
        for i in range(p.N):
            X[i] = prev + p.h * p.f(prev, Ub[i])
            prev = X[i]
        L = np.empty_like(X)
        nxt = p.h * p.qf * (X[-1] - p.ref)
        for i in range(p.N - 1, -1, -1):
            L[i] = nxt + p.h * (p.q * (X[i] - p.ref) + p.dphi(X[i]) * p.lap(nxt))
            nxt = L[i]
        sx = np.abs(X).max()
        sl = np.abs(L).max()
        assert np.abs(Xb.reshape(X.shape) - X).max() <= rtol * sx
        assert np.abs(Lb.reshape(L.shape) - L).max() <= rtol * sl
    s.close()


@pytest.mark.parametrize("strips", [2, 1])
def test_learned_closed_loop_graph_equals_host_driven_loops(G, strips):
    """The learned closed loop as one CUDA graph (network kernels captured into
    the step body, rollout, solve, plant) gives the host-driven C loop's and
    the Python-driven loop's iterations and plant states, on the cluster path
    (strips 2) and on the strip path (strips 1)."""
    import torch
    from paper_2004_02484_gb300 import warmstart as WS
    train = wl.heat2d_large_batch(n=4, base_seed=7000, m=32, horizon=10)
    X, U = WS.closed_loop_data(train, 4, 2)
    lcs = WS.LearnedControlStart(train[0], pool=4, max_batch=16)
    lcs.fit(X, U, steps=100, batch=16)
    test = wl.heat2d_large_batch(n=2, base_seed=5000, m=32, horizon=10)
    out = []
    for use_graph in (1, 0):
        s = G.Solver(test, tol=1e-6, precision=1, max_iter=4000, use_graph=use_graph, strips=strips)
        w = s.x0.clone()
        rc, iters, res = WS.closed_loop_learned_graph(s, lcs, w, 3, 2)
        torch.cuda.synchronize()
        assert rc == G.NMPC_OK and np.all(res <= 1e-6)
        out.append((iters, w.cpu().numpy()))
        s.close()
    s = G.Solver(test, tol=1e-6, precision=1, max_iter=4000, strips=strips)
    w = s.x0.clone()
    py = WS.closed_loop_learned(s, lcs, w, 3, 2, rule="always", decode="rollout")
    torch.cuda.synchronize()
    out.append((py["iters"], w.cpu().numpy()))
    s.close()
    for it, wf in out[1:]:
        assert np.array_equal(it, out[0][0])
        assert np.array_equal(wf, out[0][1])


def test_fused_rollout_matches_the_float64_rollout(G):
    """nmpc_rollout_fused (one launch, float32 arithmetic) gives the float64
    rollout's trajectories to float32 accuracy (relative 1e-5 of each field's
    scale), on a ragged 2D + 1D batch."""
    import torch
    insts = [wl.heat2d(20, 18, 7, 3, 3, seed=81), wl.heat1d(40, 11, 2, 0.02, seed=82),
             wl.heat2d(64, 64, 12, 4, 2, seed=84)]
    s = G.Solver(insts, tol=1e-6, precision=0, max_iter=2000)  # nmpc_rollout in float64
    rng = np.random.default_rng(85)
    u = _t(rng.normal(0.0, 0.3, s.n_u))
    x, lam = (torch.empty(s.n_s, dtype=torch.float64, device="cuda") for _ in range(2))
    xf, lf = torch.empty_like(x), torch.empty_like(x)
    G.nmpc_rollout(s.h, s.x0, s.ref, u, x, lam)
    G.nmpc_rollout_fused(s.h, s.x0, s.ref, u, xf, lf)
    torch.cuda.synchronize()
    s.close()
    for a, b_, per in ((x, xf, "ng"), (lam, lf, "ng")):
        A = G.split_stages(insts, a.cpu().numpy(), per)
        Bf = G.split_stages(insts, b_.cpu().numpy(), per)
        for ai, bi in zip(A, Bf):
            assert np.abs(ai - bi).max() <= 1e-5 * np.abs(ai).max()
