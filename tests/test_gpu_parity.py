"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances, derived from the arithmetic:
* FP64 path, one or a few iterations from the same iterate: the kernel and
  the oracle evaluate the same formulas in a different order (stencil sums,
  fused multiply-adds), so results agree to a few ulps of the largest term;
  relative 1e-11 on states (scaled by the field's max) leaves 100x margin.
* MIXED path: the lower layer runs in float32 (unit roundoff 6e-8), so one
  update Delta s carries a relative error of about 1e-6 after ~20 dependent
  operations; the float64 master state then differs by <= 1e-5 * |Delta s|.
* Solves to a tolerance: the FP64 path follows the oracle's iterate sequence
  exactly, so the iteration count is equal and controls agree to 1e-9
  relative; the MIXED path reaches the same root (the fixed point depends
  only on the float64 residual) and its controls agree to 1e-3 relative at
  ||K||_inf <= 1e-6 and to 1e-5 relative when both are driven to 1e-10.
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


def _rand_state(insts, seed, sx=0.05, su=0.5, sl=1e-4):
    """A perturbed cold start per instance, packed (x, u, lam) + per-instance lists."""
    rng = np.random.default_rng(seed)
    Xs, Us, Ls = [], [], []
    for inst in insts:
        p = O.Problem(inst)
        X, U, L = p.cold_start()
        Xs.append(X + sx * rng.standard_normal(X.shape))
        Us.append(U + su * rng.standard_normal(U.shape))
        Ls.append(L + sl * rng.standard_normal(L.shape))
    pk = lambda A: np.concatenate([a.reshape(-1) for a in A])
    return (pk(Xs), pk(Us), pk(Ls)), (Xs, Us, Ls)


def _unpack(G, insts, x, u, lam):
    return (G.split_stages(insts, x, "ng"), G.split_stages(insts, u, "nu"),
            G.split_stages(insts, lam, "ng"))


def _iterate_gpu(G, insts, state, n_iter, **opts):
    import torch
    h = G.nmpc_setup(insts, **opts)
    x0 = _t(G.pack_fields(insts, "x0"))
    ref = _t(G.pack_fields(insts, "ref"))
    xi, ui, li = (_t(a) for a in state)
    xo, uo, lo = torch.empty_like(xi), torch.empty_like(ui), torch.empty_like(li)
    res = G.nmpc_iterate(h, x0, ref, xi, ui, li, xo, uo, lo, n_iter, len(insts))
    torch.cuda.synchronize()
    G.nmpc_destroy(h)
    return (xo.cpu().numpy(), uo.cpu().numpy(), lo.cpu().numpy()), res


def _oracle_iterate(insts, lists, n_iter):
    out = []
    norms = []
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        X, U, L = lists[0][b], lists[1][b], lists[2][b]
        for _ in range(n_iter):
            X, U, L, nm = O.jacobi_iteration(p, X, U, L)
        out.append((X.reshape(p.N, -1), U, L.reshape(p.N, -1)))
        norms.append(nm)
    return out, norms


def _cmp_iterates(G, insts, gpu, ora, rtol):
    gx, gu, gl = _unpack(G, insts, *gpu)
    for b in range(len(insts)):
        X, U, L = ora[b]
        for g, o in ((gx[b], X), (gl[b], L), (gu[b], U)):
            scale = max(np.abs(o).max(), 1e-300)
            err = np.abs(g - o).max() / scale
            assert err <= rtol, (b, err)


CASES = {
    "heat1d_M32_N20": lambda: [wl.heat1d_single()],
    "heat2d_16x12_N7": lambda: [wl.heat2d(16, 12, 7, 3, 2, seed=4)],
    "heat2d_64x64_N50": lambda: [wl.heat2d_single()],
    "ragged1d_x24": lambda: wl.heat1d_ragged_batch(24),
}


@pytest.mark.parametrize("case", list(CASES))
def test_one_iteration_fp64_matches_oracle(G, case):
    insts = CASES[case]()
    state, lists = _rand_state(insts, 1)
    gpu, res = _iterate_gpu(G, insts, state, 1, precision=G.NMPC_FP64)
    ora, norms = _oracle_iterate(insts, lists, 1)
    _cmp_iterates(G, insts, gpu, ora, 1e-11)
    for b in range(len(insts)):
        assert abs(res[b, 0] - norms[b][0]) <= 1e-12 * norms[b][0]
        assert abs(res[b, 1] - norms[b][1]) <= 1e-10 * norms[b][1]


@pytest.mark.parametrize("case", ["heat1d_M32_N20", "heat2d_16x12_N7", "ragged1d_x24"])
def test_several_iterations_fp64_match_oracle(G, case):
    insts = CASES[case]()
    state, lists = _rand_state(insts, 2)
    gpu, _ = _iterate_gpu(G, insts, state, 12, precision=G.NMPC_FP64)
    ora, _ = _oracle_iterate(insts, lists, 12)
    _cmp_iterates(G, insts, gpu, ora, 1e-10)


@pytest.mark.parametrize("case", list(CASES))
def test_one_iteration_mixed_matches_oracle(G, case):
    """Float32 lower layer: compare the update Delta s relative to its size."""
    insts = CASES[case]()
    state, lists = _rand_state(insts, 3)
    gpu, res = _iterate_gpu(G, insts, state, 1, precision=G.NMPC_MIXED)
    ora, norms = _oracle_iterate(insts, lists, 1)
    gx, gu, gl = _unpack(G, insts, *gpu)
    for b in range(len(insts)):
        X, U, L = ora[b]
        x_in, u_in, l_in = (lists[q][b].reshape(X.shape if q != 1 else U.shape) for q in range(3))
        for g, o, i in ((gx[b], X, x_in), (gl[b], L, l_in), (gu[b], U, u_in)):
            d_or = o - i
            err = np.abs((g - i) - d_or).max() / max(np.abs(d_or).max(), 1e-300)
            assert err <= 1e-4, (b, err)
        # the mixed path's iterations use the split residual: float64
        # differences, float32 O(h) terms and a float32 max-norm
        assert abs(res[b, 0] - norms[b][0]) <= 1e-5 * norms[b][0]


def _solve_gpu(G, insts, **opts):
    import torch
    s = G.Solver(insts, **opts)
    rc, stats = s.solve()
    torch.cuda.synchronize()
    u = s.u.cpu().numpy()
    x, uu, lam = (t.cpu().numpy() for t in s.state())
    st = [(stats[b].status, stats[b].iters, stats[b].res_inf) for b in range(len(insts))]
    s.close()
    return rc, st, u, (x, uu, lam)


@pytest.mark.parametrize("case", ["heat1d_M32_N20", "heat2d_16x12_N7"])
def test_solve_fp64_follows_the_oracle_iterates(G, case):
    insts = CASES[case]()
    rc, st, u, _ = _solve_gpu(G, insts, tol=1e-8, precision=G.NMPC_FP64)
    assert rc == G.NMPC_OK
    ug = G.split_stages(insts, u, "nu")
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        (X, U, L), info = O.solve_jacobi(p, tol=1e-8)
        assert st[b][0] == G.NMPC_STATUS_CONVERGED
        assert st[b][1] == info["iters"]
        assert abs(st[b][2] - info["res_inf"]) <= 1e-9 * info["res_inf"] + 1e-20
        assert st[b][2] <= 1e-8
        err = np.abs(ug[b] - U).max() / np.abs(U).max()
        assert err <= 1e-9, err


def test_solve_heat2d_64x64_fp64_and_mixed_reach_the_oracle_root(G):
    """The 2D 64x64, N=50 workload: both paths reach ||K||_inf <= 1e-6 and
    their controls match the oracle at the same tolerance; driven to 1e-10
    the mixed path matches the oracle's tight root to 1e-5."""
    insts = [wl.heat2d_single()]
    p = O.Problem(insts[0])
    (X6, U6, L6), info6 = O.solve_jacobi(p, tol=1e-6)
    rc, st, u, _ = _solve_gpu(G, insts, tol=1e-6, precision=G.NMPC_FP64)
    assert rc == G.NMPC_OK and st[0][1] == info6["iters"] and st[0][2] <= 1e-6
    ug = u.reshape(p.N, -1)
    assert np.abs(ug - U6).max() / np.abs(U6).max() <= 1e-9
    rc, st, u, _ = _solve_gpu(G, insts, tol=1e-6, precision=G.NMPC_MIXED)
    assert rc == G.NMPC_OK and st[0][2] <= 1e-6
    ug = u.reshape(p.N, -1)
    assert np.abs(ug - U6).max() / np.abs(U6).max() <= 1e-3
    (Xt, Ut, Lt), infot = O.solve_jacobi(p, tol=1e-10)
    rc, st, u, _ = _solve_gpu(G, insts, tol=1e-10, precision=G.NMPC_MIXED)
    assert rc == G.NMPC_OK and st[0][2] <= 1e-10
    ug = u.reshape(p.N, -1)
    assert np.abs(ug - Ut).max() / np.abs(Ut).max() <= 1e-5


def test_ragged_batch_solve_matches_each_instance_alone(G):
    insts = wl.heat1d_ragged_batch(40)
    rc, st, u, _ = _solve_gpu(G, insts, tol=1e-7, precision=G.NMPC_FP64)
    assert rc == G.NMPC_OK
    ug = G.split_stages(insts, u, "nu")
    for b in (0, 7, 19, 39):
        p = O.Problem(insts[b])
        (X, U, L), info = O.solve_jacobi(p, tol=1e-7)
        assert st[b][1] == info["iters"], (b, st[b], info["iters"])
        assert np.abs(ug[b] - U).max() / np.abs(U).max() <= 1e-9
        rc1, st1, u1, _ = _solve_gpu(G, [insts[b]], tol=1e-7, precision=G.NMPC_FP64)
        assert st1[0][1] == st[b][1]
        np.testing.assert_allclose(u1.reshape(ug[b].shape), ug[b], rtol=0, atol=1e-13 * np.abs(U).max())


def test_edge_cases_single_stage_tiny_grid_repeated_actuator(G):
    insts = [wl.heat1d(1, 1, 1, 0.01, seed=5),                       # M=1, N=1
             wl.heat1d(3, 2, 2, 0.05, seed=6, act_pos=[0.5, 0.5]),    # repeated actuator cell
             wl.heat2d(1, 5, 3, 1, 1, seed=7),                         # 2D with mx=1
             wl.heat1d(256, 60, 4, 1e-3, seed=8)]                      # largest ragged member
    state, lists = _rand_state(insts, 9)
    gpu, res = _iterate_gpu(G, insts, state, 2, precision=G.NMPC_FP64)
    ora, _ = _oracle_iterate(insts, lists, 2)
    _cmp_iterates(G, insts, gpu, ora, 1e-11)


def test_max_iter_and_divergence_are_reported_not_faulted(G):
    import torch
    insts = [wl.heat1d_single(), wl.heat1d_single()]
    insts[1].x0 = insts[1].x0.copy()
    insts[1].x0[3] = np.nan
    s = G.Solver(insts, tol=1e-12, max_iter=5, precision=G.NMPC_FP64)
    rc, stats = s.solve()
    torch.cuda.synchronize()
    assert rc in (G.NMPC_ERR_NOT_CONVERGED, G.NMPC_ERR_DIVERGED)
    assert stats[0].status == G.NMPC_STATUS_MAX_ITER and stats[0].iters == 5
    assert stats[1].status == G.NMPC_STATUS_DIVERGED
    # the handle stays usable
    s2 = G.Solver([wl.heat1d_single()], tol=1e-6)
    rc2, st2 = s2.solve()
    assert rc2 == G.NMPC_OK
    s.close()
    s2.close()


def test_host_pointer_solve_equals_device_solve(G):
    import torch
    insts = [wl.heat2d(20, 20, 10, 2, 2, seed=12)]
    s = G.Solver(insts, tol=1e-8, precision=G.NMPC_MIXED)
    rc, st = s.solve()
    ud = s.u.cpu().numpy()
    uh = np.zeros_like(ud)
    rc2, st2 = G.nmpc_solve_host(s.h, G.pack_fields(insts, "x0"), G.pack_fields(insts, "ref"),
                                 uh, len(insts))
    assert rc == rc2 == G.NMPC_OK and st[0].iters == st2[0].iters
    np.testing.assert_array_equal(ud, uh)
    # warm start from the solution converges at once
    rc3, st3 = s.solve(init=G.NMPC_INIT_WARM)
    assert rc3 == G.NMPC_OK and st3[0].iters == 0
    s.close()


def test_residual_entry_point_matches_oracle(G):
    insts = [wl.heat2d(24, 16, 9, 2, 2, seed=13), wl.heat1d(50, 12, 3, 0.02, seed=14)]
    state, lists = _rand_state(insts, 15)
    h = G.nmpc_setup(insts)
    out = G.nmpc_residual(h, _t(G.pack_fields(insts, "x0")), _t(G.pack_fields(insts, "ref")),
                          *(_t(a) for a in state), len(insts))
    G.nmpc_destroy(h)
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        r = O.kkt_norms(*O.kkt(p, lists[0][b], lists[1][b], lists[2][b]))
        assert abs(out[b, 0] - r[0]) <= 1e-12 * r[0]
        assert abs(out[b, 1] - r[1]) <= 1e-10 * r[1]


CLUSTER_CASES = {
    "heat2d_16x12_N7": lambda: [wl.heat2d(16, 12, 7, 3, 2, seed=4)],
    "heat1d_M50_N6": lambda: [wl.heat1d(50, 6, 3, 0.02, seed=21)],
    "mixed_2d_1d": lambda: [wl.heat2d(10, 9, 4, 2, 2, seed=22), wl.heat1d(40, 5, 2, 0.01, seed=23)],
}


def test_large_stage_without_staging_matches_oracle(G):
    """A 256x256 stage (16-CTA cluster, slab inputs read in place, not staged)
    and a one-CTA global-slab stage in FP64: one iteration each vs the oracle."""
    for prec in (G.NMPC_MIXED, G.NMPC_FP64):
        insts = [wl.heat2d(256, 256, 3, 4, 4, seed=61)]
        state, lists = _rand_state(insts, 62)
        gpu, res = _iterate_gpu(G, insts, state, 1, precision=prec)
        ora, norms = _oracle_iterate(insts, lists, 1)
        if prec == G.NMPC_FP64:
            _cmp_iterates(G, insts, gpu, ora, 1e-10)
        else:
            gx, gu, gl = _unpack(G, insts, *gpu)
            X, U, L = ora[0]
            d_or = X - lists[0][0].reshape(X.shape)
            assert np.abs((gx[0] - lists[0][0].reshape(X.shape)) - d_or).max() <= \
                1e-4 * np.abs(d_or).max()


@pytest.mark.parametrize("cluster", [2, 3, 5, 8, 16])
@pytest.mark.parametrize("case", list(CLUSTER_CASES))
def test_cluster_split_stage_matches_oracle(G, case, cluster):
    """A stage split over a thread-block cluster (slab halos read through
    distributed shared memory) gives the oracle's iterate."""
    insts = CLUSTER_CASES[case]()
    state, lists = _rand_state(insts, 30)
    gpu, res = _iterate_gpu(G, insts, state, 3, precision=G.NMPC_FP64, cluster=cluster)
    ora, norms = _oracle_iterate(insts, lists, 3)
    _cmp_iterates(G, insts, gpu, ora, 1e-10)


@pytest.mark.parametrize("n_lo,n_u_it", [(1, 1), (1, 2), (3, 2), (4, 3), (2, 1), (2, 3), (5, 2)])
@pytest.mark.parametrize("cluster", [1, 3])
@pytest.mark.parametrize("u_local", [1, 0])
def test_inner_iteration_counts_match_oracle(G, n_lo, n_u_it, cluster, u_local):
    """Both lower-layer orders (local actuator responses, literal full sweeps)
    give the oracle's iterate; actuators 2 cells apart make the responses
    overlap."""
    insts = [wl.heat2d(12, 14, 5, 2, 2, seed=31), wl.heat1d(33, 4, 3, 0.05, seed=32),
             wl.heat1d(20, 3, 2, 0.02, seed=34, act_pos=[0.45, 0.55])]
    state, lists = _rand_state(insts, 33)
    gpu, _ = _iterate_gpu(G, insts, state, 2, precision=G.NMPC_FP64, n_lo=n_lo,
                          n_u_it=n_u_it, cluster=cluster, u_local=u_local)
    out = []
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        X, U, L = lists[0][b], lists[1][b], lists[2][b]
        for _ in range(2):
            X, U, L, _n = O.jacobi_iteration(p, X, U, L, n_lo=n_lo, n_u_it=n_u_it)
        out.append((X.reshape(p.N, -1), U, L.reshape(p.N, -1)))
    _cmp_iterates(G, insts, gpu, out, 1e-10)


@pytest.mark.parametrize("cluster", [1, 2, 3])
def test_mixed_solve_certifies_with_a_float64_residual(G, cluster):
    """The mixed path iterates on the split residual and stops only on a
    float64 residual: the returned state's residual, recomputed by the FP64
    residual entry point and by the oracle, is below tol."""
    import torch
    insts = [wl.heat2d(32, 32, 20, 4, 2, seed=40)]
    s = G.Solver(insts, tol=1e-7, precision=G.NMPC_MIXED, cluster=cluster)
    rc, st = s.solve()
    assert rc == G.NMPC_OK and st[0].res_inf <= 1e-7
    x, u, lam = s.state()
    out = G.nmpc_residual(s.h, s.x0, s.ref, x, u, lam, 1)
    assert out[0, 0] <= 1e-7 and abs(out[0, 0] - st[0].res_inf) <= 1e-12 * st[0].res_inf + 1e-20
    p = O.Problem(insts[0])
    X = x.cpu().numpy().reshape((p.N,) + p.shape)
    L = lam.cpu().numpy().reshape((p.N,) + p.shape)
    U = u.cpu().numpy().reshape(p.N, -1)
    assert O.kkt_norms(*O.kkt(p, X, U, L))[0] <= 1e-7
    s.close()


# (instances, options, most float64-residual iterations per solve): the
# red-black iterates of the 32x32 instance and of one 1D instance first reach
# ||K|| ~ 0.98e-6, then dwell at 1.0-1.2e-6 for several iterations, which the
# split residual waits out
SWITCH_CASES = {
    "cluster_2d": (lambda: [wl.heat2d(32, 32, 20, 4, 2, seed=40)], {}, 3),
    "line_1d": (lambda: wl.heat1d_ragged_batch(8), {}, 3),
    "strip_2d": (lambda: [wl.heat2d(40, 30, 12, 2, 2, seed=3)], dict(strips=1, strip_rows=8), 3),
}


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("case", list(SWITCH_CASES))
def test_float64_residual_iterations_are_counted_and_few(G, case, variant):
    """nmpc_stats.f64_iters counts the iterations that evaluated the float64
    residual: all of them in FP64; in MIXED only those after a residual at or
    below the threshold (a float64 residual above it hands back to the split
    residual), so with tol above the split residual's rounding floor a solve
    takes a few."""
    mk, opts, most = SWITCH_CASES[case]
    insts = mk()
    s = G.Solver(insts, tol=1e-6, precision=G.NMPC_FP64, variant=variant, max_iter=4000, **opts)
    rc, st = s.solve()
    s.close()
    assert rc == G.NMPC_OK and all(s_.f64_iters == s_.iters + 1 for s_ in st)
    s = G.Solver(insts, tol=1e-6, precision=G.NMPC_MIXED, variant=variant, max_iter=4000, **opts)
    rc, st = s.solve()
    s.close()
    assert rc == G.NMPC_OK
    for s_ in st:
        assert 1 <= s_.f64_iters <= most, (s_.iters, s_.f64_iters)
        assert s_.res_inf <= 1e-6


def test_mixed_reaches_tight_tolerance_above_the_split_floor(G):
    """1D M=256, h=1e-4: the split residual's float32 floor (~1e-7) is above
    tol = 1e-8; the solve must switch to the float64 residual and converge to
    the oracle's root."""
    insts = [wl.heat1d(256, 20, 4, 1e-3, seed=71), wl.heat1d(200, 12, 2, 0.05, seed=72)]
    rc, st, u, _ = _solve_gpu(G, insts, tol=1e-8, precision=G.NMPC_MIXED, max_iter=20000)
    assert rc == G.NMPC_OK and all(s_[2] <= 1e-8 for s_ in st)
    ug = G.split_stages(insts, u, "nu")
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        (X, U, L), info = O.solve_jacobi(p, tol=1e-10, max_iter=50000)
        assert np.abs(ug[b] - U).max() <= 1e-4 * np.abs(U).max()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["c2", "ragged3", "heat1d_split"])
def test_persistent_solve_is_bit_identical_to_per_iteration_launches(G, precision, case):
    """One launch for the whole solve (grid barriers between iterations).  On
    the cluster path (the stage state resident in shared memory) it performs
    exactly the arithmetic of one launch per iteration: same iteration
    counts, same iterates.  On the line path, which the mixed-precision 1D
    cases take (the resident warps claiming the line list's items every
    iteration), the stage body is a separately compiled copy whose float32
    multiply-adds may be contracted differently: iteration counts within one,
    controls within 1e-5, both residuals at the tolerance."""
    import torch
    if case == "c2":
        insts, kw = [wl.heat2d_single()], dict(cluster=8)
    elif case == "ragged3":
        insts, kw = wl.heat1d_ragged_batch(3), {}
    else:
        insts, kw = [wl.heat1d(40, 9, 3, 0.02, seed=11)], dict(cluster=3)
    out = []
    for persistent in (1, 0):
        s = G.Solver(insts, tol=1e-6, precision=precision, max_iter=4000, persistent=persistent,
                     **kw)
        rc, st = s.solve()
        x, u, lam = s.state()
        torch.cuda.synchronize()
        out.append(([st[i].iters for i in range(len(insts))], [st[i].res_inf for i in range(len(insts))],
                    x.cpu().numpy(), u.cpu().numpy(), lam.cpu().numpy(), rc))
        s.close()
    a, b = out
    assert a[5] == b[5] == G.NMPC_OK
    if precision == 1 and case != "c2":  # the line path
        assert all(abs(p - q) <= 1 for p, q in zip(a[0], b[0]))
        assert max(a[1]) <= 1e-6 and max(b[1]) <= 1e-6
        assert np.abs(a[3] - b[3]).max() <= 1e-5 * np.abs(b[3]).max()
        return
    assert a[0] == b[0]
    assert a[1] == b[1]
    for i in (2, 3, 4):
        assert np.array_equal(a[i], b[i])


@pytest.mark.parametrize("precision", [0, 1])
def test_grid_barrier_timeout_falls_back_to_per_iteration_launches(G, precision):
    """A persistent launch whose grid-barrier waits may spin for only 100 SM
    cycles: the first cluster that has to wait gives up, raises the error word
    and every cluster leaves the launch (bounded waits: no hang, no fault);
    the host discards that launch's state and solves from S^0 with one launch
    per iteration, so the result is the one of a handle that never tried the
    persistent launch, and the handle stays in per-iteration mode."""
    import torch
    # lines=2 keeps the mixed-precision 1D instance on the cluster path (the
    # line path's persistent launch: the next test)
    insts, kw = [wl.heat1d(40, 9, 3, 0.02, seed=11)], dict(cluster=3, lines=2)
    out = []
    for persistent, wait in ((1, 100), (0, 0)):
        s = G.Solver(insts, tol=1e-6, precision=precision, max_iter=4000, persistent=persistent,
                     barrier_wait_cycles=wait, **kw)
        assert G.nmpc_launch_plan(s.h)["persistent"] == persistent
        rc, st = s.solve()
        x, u, lam = s.state()
        torch.cuda.synchronize()
        out.append((rc, st[0].iters, st[0].res_inf, x.cpu().numpy(), u.cpu().numpy(),
                    lam.cpu().numpy()))
        if persistent:
            assert G.nmpc_launch_plan(s.h)["persistent"] == 0  # fell back, and stays so
            rc2, st2 = s.solve()
            assert rc2 == G.NMPC_OK and st2[0].iters == st[0].iters
        s.close()
    a, b = out
    assert a[0] == b[0] == G.NMPC_OK
    assert a[1] == b[1] and a[2] == b[2]
    for i in (3, 4, 5):
        assert np.array_equal(a[i], b[i])


def test_line_path_grid_barrier_timeout_falls_back_to_per_iteration_launches(G):
    """The line path's persistent launch (a ragged 1D batch, mixed precision)
    with grid-barrier waits of at most 100 SM cycles: a CTA that has to wait
    gives up, raises the error word and every CTA leaves the launch (bounded
    waits: no hang, no fault); the host solves again from S^0 with one launch
    per iteration, with the result of a handle that never tried the
    persistent launch, and the handle stays in per-iteration mode."""
    import torch
    insts = wl.heat1d_ragged_batch(24)
    out = []
    for persistent, wait in ((1, 100), (0, 0)):
        s = G.Solver(insts, tol=1e-6, precision=G.NMPC_MIXED, max_iter=4000,
                     persistent=persistent, barrier_wait_cycles=wait)
        assert G.nmpc_line_plan(s.h)["instances"] == len(insts)
        assert G.nmpc_launch_plan(s.h)["persistent"] == persistent
        rc, st = s.solve()
        x, u, lam = s.state()
        torch.cuda.synchronize()
        out.append((rc, [t.iters for t in st], [t.res_inf for t in st], x.cpu().numpy(),
                    u.cpu().numpy(), lam.cpu().numpy()))
        if persistent:
            assert G.nmpc_launch_plan(s.h)["persistent"] == 0  # fell back, and stays so
        s.close()
    a, b = out
    assert a[0] == b[0] == G.NMPC_OK
    assert a[1] == b[1] and a[2] == b[2]
    for i in (3, 4, 5):
        assert np.array_equal(a[i], b[i])


def test_line_path_persistent_solve_matches_the_oracle(G):
    """The persistent line launch on a ragged 1D batch, solved to 1e-9: the
    oracle's float64 residual of every returned state is at the tolerance
    and the controls lie within 1e-4 (relative) of the oracle's root."""
    import torch
    insts = wl.heat1d_ragged_batch(16)
    s = G.Solver(insts, tol=1e-9, precision=G.NMPC_MIXED, max_iter=8000, persistent=1)
    assert G.nmpc_launch_plan(s.h)["persistent"] == 1
    rc, st = s.solve()
    x, u, lam = (t.cpu().numpy() for t in s.state())
    torch.cuda.synchronize()
    s.close()
    assert rc == G.NMPC_OK
    xs = G.split_stages(insts, x, "ng")
    us = G.split_stages(insts, u, "nu")
    ls = G.split_stages(insts, lam, "ng")
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        K = O.kkt(p, xs[b].reshape((p.N,) + p.shape), us[b].reshape(p.N, p.nu),
                  ls[b].reshape((p.N,) + p.shape))
        assert O.kkt_norms(*K)[0] <= 2e-9, b
        (X, U, L), info = O.solve_jacobi(p, tol=1e-10, max_iter=50000)
        assert np.abs(us[b].reshape(U.shape) - U).max() <= 1e-4 * np.abs(U).max(), b
