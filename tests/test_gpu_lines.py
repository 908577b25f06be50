"""Line path (k_line: one warp per 1D stage, cells in registers) against the
FP64 oracle and against the cluster path.

The line kernel evaluates the cluster path's 1D formulas (split or float64
residual, n_u_it + 1 applications of P^{-1} with n_lo sweeps each) with the
stage's cells spread over a warp, 1, 2, 4 or 8 per lane.  The cases cover
every cells-per-lane class and its ragged ends (M = 1, 31, 32, 33, 64, 65,
127, 128, 129, 200, 255, 256), actuators at the line's ends and on lane
boundaries, two actuators on one cell, and a 1D batch mixed with a 2D
instance on the cluster path in one handle.  Bars: the mixed update Delta s
to float32 accuracy (1e-4 of |Delta s|, as for the other float32 paths), the
float64 residual entry point to 1e-12, solves to ||K||_inf <= 1e-6 in float64.
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
    from paper_2004_02484_gb300 import nmpc as G
    import torch
    torch.cuda.set_device(0)
    return G


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _lines_batch():
    """One instance per cells-per-lane class and ragged end; actuators at the
    ends, on lane boundaries (cells 7/8 for 8 cells per lane, 31/32) and two
    on one cell."""
    out = []
    for i, (m, n, nu) in enumerate([(1, 3, 1), (31, 4, 2), (32, 3, 2), (33, 5, 3), (64, 2, 2),
                                    (65, 4, 4), (127, 3, 3), (128, 2, 2), (129, 3, 2),
                                    (200, 4, 4), (255, 2, 3), (256, 3, 4)]):
        inst = wl.heat1d(m, n, nu, 10.0 ** (-3 + 0.2 * i), seed=4000 + i)
        out.append(inst)
    out[3].act = np.asarray([0, 32, 32], dtype=np.int32)       # two on cell 32 (lane 16 / 2 cells)
    out[6].act = np.asarray([3, 4, 126], dtype=np.int32)       # lane boundary for 4 cells per lane
    out[9].act = np.asarray([7, 8, 199, 100], dtype=np.int32)  # lane boundary, last cell
    out[11].act = np.asarray([0, 255, 128, 127], dtype=np.int32)
    return out


def _rand_state(insts, seed, sx=0.05, su=0.5, sl=1e-4):
    rng = np.random.default_rng(seed)
    Xs, Us, Ls = [], [], []
    for inst in insts:
        X, U, L = O.Problem(inst).cold_start()
        Xs.append(X + sx * rng.standard_normal(X.shape))
        Us.append(U + su * rng.standard_normal(U.shape))
        Ls.append(L + sl * rng.standard_normal(L.shape))
    pk = lambda A: np.concatenate([a.reshape(-1) for a in A])
    return (pk(Xs), pk(Us), pk(Ls)), (Xs, Us, Ls)


def _iterate(G, insts, state, n_iter, **opts):
    import torch
    h = G.nmpc_setup(insts, **opts)
    plan = G.nmpc_line_plan(h)
    x0 = _t(G.pack_fields(insts, "x0"))
    ref = _t(G.pack_fields(insts, "ref"))
    xi, ui, li = (_t(a) for a in state)
    xo, uo, lo = torch.empty_like(xi), torch.empty_like(ui), torch.empty_like(li)
    res = G.nmpc_iterate(h, x0, ref, xi, ui, li, xo, uo, lo, n_iter, len(insts))
    torch.cuda.synchronize()
    G.nmpc_destroy(h)
    return (xo.cpu().numpy(), uo.cpu().numpy(), lo.cpu().numpy()), res, plan


def _oracle(insts, lists, n_iter, **kw):
    out, norms = [], []
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        X, U, L = lists[0][b], lists[1][b], lists[2][b]
        nm = None
        for _ in range(n_iter):
            X, U, L, nm = O.jacobi_iteration(p, X, U, L, **kw)
        out.append((X.reshape(p.N, -1), U, L.reshape(p.N, -1)))
        norms.append(nm)
    return out, norms


def _split(G, insts, x, u, lam):
    return (G.split_stages(insts, x, "ng"), G.split_stages(insts, u, "nu"),
            G.split_stages(insts, lam, "ng"))


@pytest.mark.parametrize("n_lo,n_u_it", [(1, 1), (2, 1), (2, 2), (3, 2)])
def test_line_iterate_matches_oracle(G, n_lo, n_u_it):
    """One mixed iteration from a perturbed state: the update Delta s agrees
    with the oracle's to 1e-4 of its size, the split residual norm to 1e-5."""
    insts = _lines_batch()
    state, lists = _rand_state(insts, 51)
    gpu, res, plan = _iterate(G, insts, state, 1, precision=G.NMPC_MIXED, n_lo=n_lo,
                              n_u_it=n_u_it)
    assert plan["instances"] == len(insts)
    assert plan["lines"] == sum(i.horizon for i in insts)
    ora, norms = _oracle(insts, lists, 1, n_lo=n_lo, n_u_it=n_u_it)
    gx, gu, gl = _split(G, insts, *gpu)
    for b in range(len(insts)):
        X, U, L = ora[b]
        for g, o, i in ((gx[b], X, lists[0][b]), (gl[b], L, lists[2][b]), (gu[b], U, lists[1][b])):
            i = i.reshape(o.shape)
            d_or = o - i
            err = np.abs((g - i) - d_or).max() / max(np.abs(d_or).max(), 1e-300)
            assert err <= 1e-4, (b, insts[b].mx, err)
        assert abs(res[b, 0] - norms[b][0]) <= 1e-5 * norms[b][0], b


def test_line_iterates_equal_cluster_iterates(G):
    """Three mixed iterations on the line path and on the cluster path
    (lines = 2) from the same state: the same formulas in float32, so the
    iterates agree to float32 rounding of the update (1e-4 of |Delta s|)."""
    insts = _lines_batch()
    state, lists = _rand_state(insts, 52)
    a, ra, pa = _iterate(G, insts, state, 3, precision=G.NMPC_MIXED)
    c, rc, pc = _iterate(G, insts, state, 3, precision=G.NMPC_MIXED, lines=2)
    assert pa["instances"] == len(insts) and pc["instances"] == 0
    for ga, gc, s0 in zip(a, c, state):
        d = np.abs(gc - s0).max()
        assert np.abs(ga - gc).max() <= 1e-4 * d
    assert np.allclose(ra[:, 0], rc[:, 0], rtol=1e-5)


def test_line_residual_entry_point_matches_oracle(G):
    """The float64 residual (one-shot, residual only) on the line path."""
    import torch
    insts = _lines_batch()
    state, lists = _rand_state(insts, 53)
    h = G.nmpc_setup(insts, precision=G.NMPC_MIXED)
    assert G.nmpc_line_plan(h)["instances"] == len(insts)
    x0 = _t(G.pack_fields(insts, "x0"))
    ref = _t(G.pack_fields(insts, "ref"))
    r = G.nmpc_residual(h, x0, ref, *(_t(v) for v in state), len(insts))
    torch.cuda.synchronize()
    G.nmpc_destroy(h)
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        K = O.kkt(p, lists[0][b].reshape((p.N,) + p.shape), lists[1][b],
                  lists[2][b].reshape((p.N,) + p.shape))
        inf, two = O.kkt_norms(*K)
        assert abs(r[b, 0] - inf) <= 1e-12 * inf
        assert abs(r[b, 1] - two) <= 1e-10 * two


def test_line_solve_reaches_the_oracle_residual(G):
    """Solves of the ragged batch cases and a 2D instance (cluster path) in one
    handle: the float64 residual of every returned state, recomputed by the
    oracle, is <= 1e-6; controls agree with the cluster path's solve to the
    float32 bar (1e-3 relative)."""
    import torch
    insts = _lines_batch() + [wl.heat2d(24, 20, 3, 2, 2, seed=77)]
    out = {}
    for lines in (0, 2):
        s = G.Solver(insts, tol=1e-6, precision=G.NMPC_MIXED, max_iter=8000, lines=lines)
        assert G.nmpc_line_plan(s.h)["instances"] == (len(insts) - 1 if lines == 0 else 0)
        rc, st = s.solve()
        torch.cuda.synchronize()
        assert rc == G.NMPC_OK
        x, u, lam = (t.cpu().numpy() for t in s.state())
        out[lines] = ([st[b].iters for b in range(len(insts))], u)
        s.close()
        xs, us, ls = _split(G, insts, x, u, lam)
        for b, inst in enumerate(insts):
            p = O.Problem(inst)
            K = O.kkt(p, xs[b].reshape((p.N,) + p.shape), us[b].reshape(p.N, p.nu),
                      ls[b].reshape((p.N,) + p.shape))
            assert O.kkt_norms(*K)[0] <= 1e-6, (lines, b)
    ul, uc = out[0][1], out[2][1]
    assert np.abs(ul - uc).max() <= 1e-3 * np.abs(uc).max()
    # same method, same rounding class: iteration counts within a few
    assert np.abs(np.array(out[0][0]) - np.array(out[2][0])).max() <= 3


def test_line_ragged_batch_solve(G):
    """64 instances of the ragged 1D batch: every instance converges on the
    line path, and the oracle's float64 residual of sampled returned states is
    <= 1e-6."""
    import torch
    insts = wl.heat1d_ragged_batch(64)
    s = G.Solver(insts, tol=1e-6, precision=G.NMPC_MIXED, max_iter=8000)
    assert G.nmpc_line_plan(s.h)["instances"] == 64
    rc, st = s.solve()
    torch.cuda.synchronize()
    assert rc == G.NMPC_OK
    assert all(st[b].res_inf <= 1e-6 for b in range(64))
    x, u, lam = (t.cpu().numpy() for t in s.state())
    s.close()
    xs, us, ls = _split(G, insts, x, u, lam)
    for b in (0, 17, 40, 63):
        p = O.Problem(insts[b])
        K = O.kkt(p, xs[b].reshape((p.N,) + p.shape), us[b].reshape(p.N, p.nu),
                  ls[b].reshape((p.N,) + p.shape))
        assert O.kkt_norms(*K)[0] <= 1e-6, b


def test_fp64_handles_keep_1d_on_the_cluster_path(G):
    h = G.nmpc_setup(_lines_batch()[:3], precision=G.NMPC_FP64)
    assert G.nmpc_line_plan(h)["instances"] == 0
    G.nmpc_destroy(h)


def test_line_mixed_solve_reaches_a_tight_tolerance(G):
    """Mixed precision at tol = 1e-9 on the line path (float32 lower layer,
    float64 residual once the split residual's bound can no longer show the
    level): every instance converges and the oracle's float64 residual of the
    returned state is <= 1e-9."""
    import torch
    insts = _lines_batch()
    s = G.Solver(insts, tol=1e-9, precision=G.NMPC_MIXED, max_iter=8000)
    rc, st = s.solve()
    torch.cuda.synchronize()
    assert rc == G.NMPC_OK
    x, u, lam = (t.cpu().numpy() for t in s.state())
    s.close()
    xs, us, ls = _split(G, insts, x, u, lam)
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        K = O.kkt(p, xs[b].reshape((p.N,) + p.shape), us[b].reshape(p.N, p.nu),
                  ls[b].reshape((p.N,) + p.shape))
        assert O.kkt_norms(*K)[0] <= 1.0001e-9, b
