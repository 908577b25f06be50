"""GPU parity of the red-black Gauss-Seidel upper layer (NMPC_VARIANT_REDBLACK)
against the oracle's red-black sweep (oracle/nmpc.py gauss_seidel_iteration
with the even-then-odd stage order; the oracle's sweep is pinned to the
matrix definition (D + L_rb)^{-1} K and to Theorem 3 by
tests/test_oracle_variants.py).

Tolerances as in test_gpu_parity.py: FP64 iterates 1e-11 relative (one
iteration) and 1e-10 (twelve); the MIXED path's update Delta s to 1e-4 of its
size; FP64 solves follow the oracle's iterate sequence (equal iteration
count, controls 1e-9); MIXED solves are certified by the oracle's float64
residual of the returned state.
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


def _state(insts, seed, sx=0.05, su=0.5, sl=1e-4):
    rng = np.random.default_rng(seed)
    lists = ([], [], [])
    for inst in insts:
        X, U, L = O.Problem(inst).cold_start()
        lists[0].append(X + sx * rng.standard_normal(X.shape))
        lists[1].append(U + su * rng.standard_normal(U.shape))
        lists[2].append(L + sl * rng.standard_normal(L.shape))
    pk = lambda A: np.concatenate([a.reshape(-1) for a in A])
    return tuple(pk(l) for l in lists), lists


def _gpu_iterate(G, insts, state, n_iter, **opts):
    import torch
    h = G.nmpc_setup(insts, variant=G.NMPC_VARIANT_REDBLACK, **opts)
    x0, ref = _t(G.pack_fields(insts, "x0")), _t(G.pack_fields(insts, "ref"))
    xi, ui, li = (_t(a) for a in state)
    xo, uo, lo = torch.empty_like(xi), torch.empty_like(ui), torch.empty_like(li)
    res = G.nmpc_iterate(h, x0, ref, xi, ui, li, xo, uo, lo, n_iter, len(insts))
    torch.cuda.synchronize()
    G.nmpc_destroy(h)
    return (G.split_stages(insts, xo.cpu().numpy(), "ng"), G.split_stages(insts, uo.cpu().numpy(), "nu"),
            G.split_stages(insts, lo.cpu().numpy(), "ng")), res


def _oracle(insts, lists, n_iter, **kw):
    out, norms = [], []
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        X, U, L = lists[0][b], lists[1][b], lists[2][b]
        for _ in range(n_iter):
            X, U, L, nm = O.gauss_seidel_iteration(p, X, U, L, O.gs_order(p.N, "redblack"), **kw)
        out.append((X.reshape(p.N, -1), U, L.reshape(p.N, -1)))
        norms.append(nm)
    return out, norms


CASES = {
    "heat1d_M32_N20": lambda: [wl.heat1d_single()],
    "heat2d_16x12_N7": lambda: [wl.heat2d(16, 12, 7, 3, 2, seed=4)],
    "heat2d_64x64_N50": lambda: [wl.heat2d_single()],
    "ragged1d_x16": lambda: wl.heat1d_ragged_batch(16),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("n_iter,rtol", [(1, 1e-11), (12, 1e-10)])
def test_fp64_iterations_match_the_oracle_sweep(G, case, n_iter, rtol):
    insts = CASES[case]()
    state, lists = _state(insts, 1)
    gpu, res = _gpu_iterate(G, insts, state, n_iter, precision=G.NMPC_FP64)
    ora, norms = _oracle(insts, lists, n_iter)
    for b in range(len(insts)):
        for g, o in zip((gpu[0][b], gpu[1][b], gpu[2][b]), ora[b]):
            err = np.abs(g - o).max() / max(np.abs(o).max(), 1e-300)
            assert err <= rtol, (b, err)
        if n_iter == 1:
            # the norms of K(S^k) of whole iterates, from both halves
            assert abs(res[b, 0] - norms[b][0]) <= 1e-12 * norms[b][0]
            assert abs(res[b, 1] - norms[b][1]) <= 1e-10 * norms[b][1]


MIXED = {
    "cluster_2d": (lambda: [wl.heat2d(16, 12, 7, 3, 2, seed=4)], {}),
    "line_1d": (lambda: wl.heat1d_ragged_batch(8), {}),
    "strip_2d": (lambda: [wl.heat2d(40, 30, 6, 2, 2, seed=3)], dict(strips=1, strip_rows=8)),
    "strip_2d_nlo1": (lambda: [wl.heat2d(40, 30, 6, 2, 2, seed=3)],
                      dict(strips=1, strip_rows=8, n_lo=1, n_u_it=1)),
}


@pytest.mark.parametrize("case", list(MIXED))
def test_mixed_iteration_matches_the_oracle_sweep(G, case):
    mk, opts = MIXED[case]
    insts = mk()
    kw = {k: opts[k] for k in ("n_lo", "n_u_it") if k in opts}
    state, lists = _state(insts, 3)
    h = G.nmpc_setup(insts, precision=G.NMPC_MIXED, variant=G.NMPC_VARIANT_REDBLACK, **opts)
    if "strips" in opts:
        assert G.nmpc_strip_plan(h)["instances"] == len(insts)
    if case == "line_1d":
        assert G.nmpc_line_plan(h)["instances"] == len(insts)
    G.nmpc_destroy(h)
    gpu, res = _gpu_iterate(G, insts, state, 1, precision=G.NMPC_MIXED, **opts)
    ora, norms = _oracle(insts, lists, 1, **kw)
    for b in range(len(insts)):
        ins = [lists[0][b].reshape(ora[b][0].shape), lists[1][b], lists[2][b].reshape(ora[b][2].shape)]
        for g, o, i in zip((gpu[0][b], gpu[1][b], gpu[2][b]), ora[b], ins):
            d = o - i
            err = np.abs((g - i) - d).max() / max(np.abs(d).max(), 1e-300)
            assert err <= 1e-4, (b, err)
        assert abs(res[b, 0] - norms[b][0]) <= 1e-5 * norms[b][0]


@pytest.mark.parametrize("case", ["heat1d_M32_N20", "heat2d_16x12_N7"])
def test_fp64_solve_follows_the_oracle_iterates(G, case):
    import torch
    insts = CASES[case]()
    s = G.Solver(insts, tol=1e-8, precision=G.NMPC_FP64, variant=G.NMPC_VARIANT_REDBLACK)
    rc, st = s.solve()
    torch.cuda.synchronize()
    ug = G.split_stages(insts, s.u.cpu().numpy(), "nu")
    s.close()
    assert rc == G.NMPC_OK
    for b, inst in enumerate(insts):
        (X, U, L), info = O.solve_variant(O.Problem(inst), "redblack", tol=1e-8)
        assert st[b].iters == info["iters"]
        # the residual's O(1) differences round at ~1e-16 absolute
        assert abs(st[b].res_inf - info["res_inf"]) <= 1e-9 * info["res_inf"] + 1e-15
        assert np.abs(ug[b] - U).max() <= 1e-9 * np.abs(U).max()


SOLVES = {
    "cluster_2d_64": (lambda: [wl.heat2d_single()], dict(n_lo=1, n_u_it=1, cluster=8)),
    "line_ragged": (lambda: wl.heat1d_ragged_batch(24), {}),
    "strip_2d": (lambda: [wl.heat2d(40, 30, 12, 2, 2, seed=3), wl.heat2d(40, 30, 12, 2, 2, seed=5)],
                 dict(strips=1, strip_rows=8)),
}


@pytest.mark.parametrize("case", list(SOLVES))
@pytest.mark.parametrize("graph", [1, 0])
def test_mixed_solve_is_certified_and_needs_fewer_iterations(G, case, graph):
    import torch
    mk, opts = SOLVES[case]
    insts = mk()
    its = {}
    for var in (G.NMPC_VARIANT_JACOBI, G.NMPC_VARIANT_REDBLACK):
        s = G.Solver(insts, tol=1e-6, precision=G.NMPC_MIXED, variant=var, use_graph=graph,
                     max_iter=4000, **opts)
        rc, st = s.solve()
        torch.cuda.synchronize()
        assert rc == G.NMPC_OK
        its[var] = [st[b].iters for b in range(len(insts))]
        x, u, lam = (t.cpu().numpy() for t in s.state())
        s.close()
    # the red-black state is certified by the oracle's float64 residual
    xs, us, ls = (G.split_stages(insts, x, "ng"), G.split_stages(insts, u, "nu"),
                  G.split_stages(insts, lam, "ng"))
    for b, inst in enumerate(insts):
        p = O.Problem(inst)
        K = O.kkt(p, xs[b].reshape((p.N,) + p.shape), us[b], ls[b].reshape((p.N,) + p.shape))
        assert O.kkt_norms(*K)[0] <= 1e-6
    rb, jac = np.array(its[G.NMPC_VARIANT_REDBLACK]), np.array(its[G.NMPC_VARIANT_JACOBI])
    assert rb.sum() <= 0.7 * jac.sum(), (rb, jac)


def test_redblack_rejects_damped_steps_and_the_allocation_free_entry(G):
    import torch
    inst = wl.heat1d_single()
    with pytest.raises(G.NmpcError) as e:
        G.nmpc_setup([inst], variant=G.NMPC_VARIANT_REDBLACK, alpha=0.5)
    assert e.value.code == G.NMPC_ERR_BAD_ARG
    x0 = _t(inst.x0)
    u = torch.zeros(inst.horizon * len(inst.act), dtype=torch.float64, device="cuda")
    with pytest.raises(G.NmpcError) as e:
        G.nmpc_solve_noalloc(inst, x0, x0, u, variant=G.NMPC_VARIANT_REDBLACK)
    assert e.value.code == G.NMPC_ERR_UNSUPPORTED
