"""Parity at the benchmarked sizes, on sampled outputs the oracle computes one
instance at a time.

* The 1024-instance ragged 1D batch (line path, mixed precision): every
  instance converges; the float64 KKT residual (eq. 9) of a seeded sample of
  32 returned states, recomputed by the oracle, is <= tol; for 4 of them the
  oracle's own solve gives controls within the float32-path bound 1e-3.
* The 64-instance 256x256, N=100 batch (strip path, mixed precision) in the
  bench's launch configuration, Jacobi and red-black upper layers: the C
  oracle (pinned element-wise to the numpy oracle) recomputes the float64
  residual of 3 sampled instances' returned states.
* A closed loop on the strip path (2 instances of 64x64, N = 10): per-step
  applied controls and the final plant state against the oracle's closed
  loop, for both upper-layer variants.
"""
import numpy as np
import pytest

from oracle import c_oracle as C
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


def _solve_states(G, insts, **opts):
    import torch
    s = G.Solver(insts, **opts)
    rc, st = s.solve()
    torch.cuda.synchronize()
    x, u, lam = (t.cpu().numpy() for t in s.state())
    stats = [(st[b].status, st[b].iters, st[b].res_inf) for b in range(len(insts))]
    s.close()
    return rc, stats, (G.split_stages(insts, x, "ng"), G.split_stages(insts, u, "nu"),
                       G.split_stages(insts, lam, "ng"))


def test_ragged_1024_line_path_sampled_against_the_oracle(G):
    insts = wl.heat1d_ragged_batch(1024)
    rc, stats, (xs, us, ls) = _solve_states(G, insts, tol=1e-6, precision=G.NMPC_MIXED,
                                            max_iter=6000)
    assert rc == G.NMPC_OK
    assert all(st[0] == G.NMPC_STATUS_CONVERGED and st[2] <= 1e-6 for st in stats)
    sample = np.random.default_rng(2024).choice(len(insts), 32, replace=False)
    for b in sample:
        p = O.Problem(insts[b])
        K = O.kkt(p, xs[b].reshape((p.N,) + p.shape), us[b], ls[b].reshape((p.N,) + p.shape))
        assert O.kkt_norms(*K)[0] <= 1e-6, b
    for b in sample[:4]:
        (_, U, _), info = C.solve_jacobi(C.Problem(insts[b]), tol=1e-6)
        assert info["converged"]
        assert np.abs(us[b] - U).max() <= 1e-3 * np.abs(U).max(), b


@pytest.mark.parametrize("variant", [0, 1])
def test_bench_batch_256_strip_path_sampled_against_the_oracle(G, variant):
    insts = wl.heat2d_large_batch(64)
    rc, stats, (xs, us, ls) = _solve_states(G, insts, tol=1e-6, precision=G.NMPC_MIXED,
                                            max_iter=4000, variant=variant)
    assert rc == G.NMPC_OK
    assert all(st[0] == G.NMPC_STATUS_CONVERGED and st[2] <= 1e-6 for st in stats)
    C.set_threads(0)
    for b in (0, 31, 63):
        p = C.Problem(insts[b])
        r = C.kkt_norms(p, xs[b], us[b], ls[b])[0]
        assert r <= 1e-6, (b, r)


@pytest.mark.parametrize("variant", [0, 1])
def test_strip_path_closed_loop_matches_the_oracle(G, variant):
    import torch
    insts = [wl.heat2d(64, 64, 10, 2, 2, seed=61), wl.heat2d(64, 64, 10, 2, 2, seed=62)]
    steps, n_sub = 4, 2
    s = G.Solver(insts, tol=1e-9, precision=G.NMPC_MIXED, max_iter=20000, strips=1,
                 strip_rows=16, variant=variant)
    assert G.nmpc_strip_plan(s.h)["instances"] == 2
    w = _t(G.pack_fields(insts, "x0"))
    nu_tot = sum(len(i.act) for i in insts)
    u_hist = torch.zeros(steps * nu_tot, dtype=torch.float64, device="cuda")
    rc, iters, res = G.nmpc_closed_loop(s.h, w, s.ref, steps, n_sub, len(insts), u_hist)
    torch.cuda.synchronize()
    s.close()
    assert rc == G.NMPC_OK and np.all(res <= 1e-9)
    uh = u_hist.cpu().numpy().reshape(steps, nu_tot)
    wg = w.cpu().numpy()
    o_u, o_w = 0, 0
    for inst in insts:
        U1, W, _ = C.closed_loop(inst, steps, n_sub, tol=1e-11)
        nu, ng = len(inst.act), inst.mx * inst.my
        assert np.abs(uh[:, o_u:o_u + nu] - U1).max() <= 1e-4 * np.abs(U1).max()
        assert np.abs(wg[o_w:o_w + ng] - W[-1]).max() <= 1e-5 * np.abs(W[-1]).max()
        o_u += nu
        o_w += ng
