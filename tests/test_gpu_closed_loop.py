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
