"""Strip path (k_patch + k_strip) against the FP64 oracle.

The strip kernel computes each strip of 32 - 2E own columns from a region
extended by E = 2 n_lo - 1 cells (one warp walking down the rows with every
pass pipelined; in mixed precision with n_lo <= 2 and even grid widths two
columns per lane: 64 - 4 n_lo own columns of a 64-column region, packed
float32 pairs), and k_patch the actuators' controls v3 from patches around
them, so the path evaluates the same formulas as the oracle in a different
order: FP64 iterates agree to a few ulps of the largest term (relative
1e-10), the mixed path's update Delta s to float32 accuracy (relative 1e-4 of
|Delta s|).  The cases put actuators on strip corners and edges, use ragged
strips (grids that are not multiples of the strip), and mix strip-path
instances with a 1D instance (line path in mixed precision, cluster path in
FP64) in one handle.
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


def _with_act(inst, rows_cols):
    """Actuators at explicit (row, column) cells."""
    inst.act = np.asarray([r * inst.mx + c for r, c in rows_cols], dtype=np.int64)
    return inst


def _batch(far=True):
    """70x20 (strips of 26 columns for n_lo = 2: 26, 26, 18; rows of 8, 8, 4
    with strip_rows 8), 30x26 (a full and a ragged strip), and a 1D instance
    (cluster path).  With `far` the 2D actuators are more than 4 cells apart
    (Manhattan)."""
    a = wl.heat2d(70, 20, 4, 3, 2, seed=91)
    cells = [(7, 63), (10, 66), (0, 0), (19, 69), (12, 30), (8, 5)] if far else \
        [(7, 63), (8, 64), (0, 0), (19, 69), (12, 30), (12, 31)]
    a = _with_act(a, cells)
    b = _with_act(wl.heat2d(30, 26, 3, 2, 2, seed=92), [(8, 8), (8, 21), (17, 0), (25, 29)])
    c = wl.heat1d(40, 5, 2, 0.02, seed=93)
    return [a, b, c]


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
    plan = G.nmpc_strip_plan(h)
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


@pytest.mark.parametrize("n_lo,n_u_it", [(1, 1), (2, 1), (2, 2), (3, 1), (3, 3), (4, 1), (1, 3)])
def test_strip_iterates_fp64_match_oracle(G, n_lo, n_u_it):
    insts = _batch(far=True)
    state, lists = _rand_state(insts, 94)
    gpu, res, plan = _iterate(G, insts, state, 2, precision=G.NMPC_FP64, strips=1, strip_rows=8,
                              n_lo=n_lo, n_u_it=n_u_it)
    tx = 32 - 2 * (2 * n_lo - 1)
    assert plan["instances"] == 2 and plan["strip_x"] == tx and plan["strip_y"] == 8
    assert plan["strips"] == 4 * -(-70 // tx) * 3 + 3 * -(-30 // tx) * 4
    ora, norms = _oracle(insts, lists, 2, n_lo=n_lo, n_u_it=n_u_it)
    gx, gu, gl = _split(G, insts, *gpu)
    for b in range(len(insts)):
        for g, o in zip((gx[b], gu[b], gl[b]), ora[b]):
            err = np.abs(g - o).max() / max(np.abs(o).max(), 1e-300)
            assert err <= 1e-10, (b, err)
        assert abs(res[b, 0] - norms[b][0]) <= 1e-11 * norms[b][0]
        assert abs(res[b, 1] - norms[b][1]) <= 1e-9 * norms[b][1]


def test_strip_actuators_close_together_with_one_u_iteration(G):
    """Neighbouring and adjacent actuators are fine for n_u_it = 1 (each
    control starts from zero); with n_u_it = 2 the instance goes to the
    cluster path and still matches."""
    insts = _batch(far=False)
    state, lists = _rand_state(insts, 95)
    for n_u_it, on_strips in ((1, 2), (2, 1)):
        gpu, _, plan = _iterate(G, insts, state, 2, precision=G.NMPC_FP64, strips=1, strip_rows=8,
                                n_u_it=n_u_it)
        assert plan["instances"] == on_strips
        ora, _ = _oracle(insts, lists, 2, n_u_it=n_u_it)
        gx, gu, gl = _split(G, insts, *gpu)
        for b in range(len(insts)):
            for g, o in zip((gx[b], gu[b], gl[b]), ora[b]):
                err = np.abs(g - o).max() / max(np.abs(o).max(), 1e-300)
                assert err <= 1e-10, (n_u_it, b, err)


def _check_mixed_update(G, insts, state, lists, gpu, res, n_lo=2):
    ora, norms = _oracle(insts, lists, 1, n_lo=n_lo)
    gx, gu, gl = _split(G, insts, *gpu)
    for b in range(len(insts)):
        X, U, L = ora[b]
        for g, o, i in ((gx[b], X, lists[0][b]), (gl[b], L, lists[2][b]), (gu[b], U, lists[1][b])):
            i = i.reshape(o.shape)
            d_or = o - i
            err = np.abs((g - i) - d_or).max() / max(np.abs(d_or).max(), 1e-300)
            assert err <= 1e-4, (b, err)
        assert abs(res[b, 0] - norms[b][0]) <= 1e-5 * norms[b][0]


@pytest.mark.parametrize("strip_cols,strip_x", [(0, 56), (1, 26)])
@pytest.mark.parametrize("strip_rows", [3, 8, 16])
def test_strip_iterate_mixed_matches_oracle(G, strip_rows, strip_cols, strip_x):
    """Float32 lower layer with the split residual, two columns per lane
    (strips of 56 own columns) or one (26): the update Delta s agrees with
    the oracle's to 1e-4 of its size, the split residual norm to 1e-5."""
    insts = _batch(far=True)
    state, lists = _rand_state(insts, 96)
    gpu, res, plan = _iterate(G, insts, state, 1, precision=G.NMPC_MIXED, strips=1,
                              strip_rows=strip_rows, strip_cols=strip_cols)
    assert plan["instances"] == 2 and plan["strip_x"] == strip_x
    _check_mixed_update(G, insts, state, lists, gpu, res)


@pytest.mark.parametrize("n_lo,strip_x", [(1, 60), (2, 56)])
def test_two_column_strips_over_several_iterations_and_inner_counts(G, n_lo, strip_x):
    """Two columns per lane for n_lo = 1 and 2, actuators on even and odd
    columns of a lane, three iterations against the oracle (mixed: 1e-4 of
    the iterate's change)."""
    insts = _batch(far=True)
    state, lists = _rand_state(insts, 98)
    gpu, res, plan = _iterate(G, insts, state, 3, precision=G.NMPC_MIXED, strips=1,
                              strip_rows=8, n_lo=n_lo, n_u_it=1)
    assert plan["strip_x"] == strip_x
    ora, norms = _oracle(insts, lists, 3, n_lo=n_lo, n_u_it=1)
    gx, gu, gl = _split(G, insts, *gpu)
    for b in range(len(insts)):
        X, U, L = ora[b]
        for g, o, i in ((gx[b], X, lists[0][b]), (gl[b], L, lists[2][b]), (gu[b], U, lists[1][b])):
            i = i.reshape(o.shape)
            d_or = o - i
            assert np.abs((g - i) - d_or).max() <= 1e-4 * np.abs(d_or).max(), b


def test_odd_grid_width_keeps_one_column_per_lane(G):
    """A strip instance of odd width (or odd array offsets) cannot move 16-byte
    column pairs: the handle falls back to one column per lane, with the same
    parity."""
    insts = _batch(far=True)
    odd = _with_act(wl.heat2d(31, 18, 3, 2, 2, seed=95), [(4, 4), (9, 30), (17, 15), (0, 17)])
    insts = [insts[0], odd, insts[2]]
    state, lists = _rand_state(insts, 99)
    gpu, res, plan = _iterate(G, insts, state, 1, precision=G.NMPC_MIXED, strips=1, strip_rows=8)
    assert plan["strip_x"] == 26
    _check_mixed_update(G, insts, state, lists, gpu, res)


def test_two_column_strips_reject_misaligned_state_pointers(G):
    """x and lam must be 16-byte aligned for the two-column strips: a pointer
    one double into a buffer is rejected on the host (nothing launched)."""
    import ctypes
    import torch
    insts = _batch(far=True)
    h = G.nmpc_setup(insts, precision=G.NMPC_MIXED, strips=1, strip_rows=8)
    assert G.nmpc_strip_plan(h)["strip_x"] == 56
    x0 = _t(G.pack_fields(insts, "x0"))
    ref = _t(G.pack_fields(insts, "ref"))
    (xs, us, ls), _ = _rand_state(insts, 100)
    xb = _t(np.concatenate([[0.0], xs]))
    u, lam = _t(us), _t(ls)
    out = np.zeros((len(insts), 2))
    rc = G.LIB.nmpc_residual(h, x0.data_ptr(), ref.data_ptr(), xb.data_ptr() + 8, u.data_ptr(),
                             lam.data_ptr(), out.ctypes.data, ctypes.c_void_p(0))
    torch.cuda.synchronize()
    G.nmpc_destroy(h)
    assert rc == G.NMPC_ERR_BAD_ARG


@pytest.mark.parametrize("precision", [0, 1])
def test_strip_solve_equals_cluster_solve(G, precision):
    """Solves to a tolerance on the strip path and on the cluster path: same
    iteration counts in FP64 and the same root (controls to 1e-9 relative);
    in mixed precision both stop on a float64 residual <= tol."""
    import torch
    insts = _batch(far=True)
    tol = 1e-8 if precision == 0 else 1e-6
    out = {}
    for strips in (1, 2):
        s = G.Solver(insts, tol=tol, precision=precision, max_iter=8000, strips=strips, strip_rows=8)
        rc, st = s.solve()
        torch.cuda.synchronize()
        assert rc == G.NMPC_OK
        x, u, lam = s.state()
        r = G.nmpc_residual(s.h, s.x0, s.ref, x, u, lam, len(insts))
        out[strips] = ([st[b].iters for b in range(3)], u.cpu().numpy(), r[:, 0])
        s.close()
    it_t, u_t, r_t = out[1]
    it_c, u_c, r_c = out[2]
    assert np.all(r_t <= tol) and np.all(r_c <= tol)
    if precision == 0:
        assert it_t == it_c
        assert np.abs(u_t - u_c).max() <= 1e-9 * np.abs(u_c).max()
    else:
        assert np.abs(u_t - u_c).max() <= 1e-3 * np.abs(u_c).max()


def test_strip_residual_entry_point_matches_oracle(G):
    import torch
    insts = _batch(far=True)
    state, lists = _rand_state(insts, 97)
    h = G.nmpc_setup(insts, precision=G.NMPC_MIXED, strips=1, strip_rows=8)
    x0 = _t(G.pack_fields(insts, "x0"))
    ref = _t(G.pack_fields(insts, "ref"))
    r = G.nmpc_residual(h, x0, ref, *(_t(a) for a in state), len(insts))
    torch.cuda.synchronize()
    G.nmpc_destroy(h)
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        K = O.kkt(p, lists[0][b].reshape((p.N,) + p.shape), lists[1][b],
                  lists[2][b].reshape((p.N,) + p.shape))
        inf, two = O.kkt_norms(*K)
        assert abs(r[b, 0] - inf) <= 1e-12 * inf
        assert abs(r[b, 1] - two) <= 1e-10 * two


def test_auto_routes_large_stages_to_strips(G):
    """strips = 0: a 256x256 stage goes to the strip path (two columns per
    lane: 56 own columns), a 64x64 stage stays on the cluster path and the 1D
    instance goes to the line path."""
    insts = [wl.heat2d(256, 256, 2, 4, 4, seed=98), wl.heat2d(64, 64, 2, 4, 2, seed=99),
             wl.heat1d(50, 3, 1, 0.01, seed=100)]
    h = G.nmpc_setup(insts, precision=G.NMPC_MIXED)
    plan, lp, ln = G.nmpc_strip_plan(h), G.nmpc_launch_plan(h), G.nmpc_line_plan(h)
    G.nmpc_destroy(h)
    ty = plan["strip_y"]
    assert plan["instances"] == 1 and plan["strip_x"] == 56 and 16 <= ty <= 256
    assert plan["strips"] == 2 * -(-256 // 56) * -(-256 // ty)
    assert lp["work_items"] == 2 and ln["instances"] == 1 and ln["lines"] == 3


@pytest.mark.parametrize("precision,rtol", [(0, 1e-5), (1, 1e-3)])
def test_full_size_grid_strip_solve_matches_oracle_solve(G, precision, rtol):
    """A 256x256 instance of the large closed-loop batch (16 actuators) on the
    strip path, horizon shortened to N = 10 so that the oracle's own Jacobi
    solve finishes in seconds: controls agree to 1e-5 (FP64) / 1e-3 (mixed)
    relative at ||K||_inf <= 1e-6, and the oracle's float64 residual of the
    GPU's returned state is <= 1e-6."""
    import torch
    inst = wl.heat2d_large_batch(n=1, base_seed=5000, m=256, horizon=10)[0]
    s = G.Solver([inst], tol=1e-6, precision=precision, max_iter=4000)
    assert G.nmpc_strip_plan(s.h)["instances"] == 1
    rc, st = s.solve()
    torch.cuda.synchronize()
    assert rc == G.NMPC_OK
    x, u, lam = (t.cpu().numpy() for t in s.state())
    s.close()
    p = O.Problem(inst)
    K = O.kkt(p, x.reshape((p.N,) + p.shape), u.reshape(p.N, p.nu), lam.reshape((p.N,) + p.shape))
    assert O.kkt_norms(*K)[0] <= 1e-6
    (X, U, L), info = O.solve_jacobi(p, tol=1e-6)
    assert info["converged"]
    err = np.abs(u.reshape(U.shape) - U).max() / np.abs(U).max()
    assert err <= rtol, err


def test_large_batch_horizon_100_state_passes_the_oracle_residual(G):
    """Two instances of the large closed-loop batch at full size (256x256,
    N = 100, mixed precision, strip path): the oracle's float64 KKT residual
    of each returned state is <= 1e-6."""
    import torch
    insts = wl.heat2d_large_batch(n=2, base_seed=5000, m=256, horizon=100)
    s = G.Solver(insts, tol=1e-6, precision=G.NMPC_MIXED, max_iter=4000)
    rc, st = s.solve()
    torch.cuda.synchronize()
    assert rc == G.NMPC_OK
    x, u, lam = (t.cpu().numpy() for t in s.state())
    s.close()
    xs, us, ls = G.split_stages(insts, x, "ng"), G.split_stages(insts, u, "nu"), \
        G.split_stages(insts, lam, "ng")
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        K = O.kkt(p, xs[b].reshape((p.N,) + p.shape), us[b], ls[b].reshape((p.N,) + p.shape))
        r = O.kkt_norms(*K)[0]
        assert r <= 1e-6, (b, r)
        assert abs(r - st[b].res_inf) <= 1e-9 * r


def test_strip_mixed_solve_reaches_a_tight_tolerance(G):
    """Mixed precision at tol = 1e-8 on the strip path: the split residual's
    float32 stage differences cannot resolve levels that low, so the handle
    switches to the float64 residual by 1e-6 at the latest and converges on
    it; the oracle's float64 residual of the returned state is <= 1e-8."""
    import torch
    insts = _batch(far=True)[:2]
    s = G.Solver(insts, tol=1e-8, precision=G.NMPC_MIXED, max_iter=8000, strips=1, strip_rows=8)
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
        assert O.kkt_norms(*K)[0] <= 1.0001e-8, b


@pytest.mark.parametrize("variant", [0, 1])
def test_tail_plan_solve_is_bit_identical_to_the_main_plan(G, variant):
    """A solve whose launches all take the tail plan (strips of 8 own rows,
    ragged against 30 grid rows, tail_below = every instance) gives the main
    plan's (24-row strips, no tail plan) iterations, statuses and iterates bit
    for bit: every own cell is computed from the same inputs by the same
    code, whichever strip holds it.  The automatic plan keeps a tail plan of
    64 rows for 256-row strips and none for short ones."""
    import torch
    insts = [wl.heat2d(40, 30, 12, 2, 2, seed=3), wl.heat2d(40, 30, 12, 2, 2, seed=5)]
    out = []
    for tail in (dict(tail_rows=-1), dict(tail_rows=8, tail_below=len(insts))):
        s = G.Solver(insts, tol=1e-7, precision=G.NMPC_MIXED, variant=variant, strips=1,
                     strip_rows=24, max_iter=4000, **tail)
        plan = G.nmpc_strip_plan(s.h)
        assert plan["strip_x"] == 56 and plan["strip_y"] == 24
        assert plan["tail_rows"] == (8 if "tail_below" in tail else 0)
        rc, st = s.solve()
        torch.cuda.synchronize()
        assert rc == G.NMPC_OK
        out.append(([(x.iters, x.status, x.res_inf, x.f64_iters) for x in st],
                    [t.cpu().numpy() for t in s.state()]))
        s.close()
    assert out[0][0] == out[1][0]
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)
    big = [wl.heat2d(256, 256, 4, 2, 2, seed=9)]
    s = G.Solver(big, precision=G.NMPC_MIXED, strips=1, strip_rows=256)
    plan = G.nmpc_strip_plan(s.h)
    assert plan["tail_rows"] == 64 and plan["tail_below"] >= 1
    s.close()
    s = G.Solver(big, precision=G.NMPC_MIXED, strips=1, strip_rows=128)
    assert G.nmpc_strip_plan(s.h)["tail_rows"] == 0
    s.close()
