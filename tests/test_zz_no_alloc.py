"""The allocation-free solve against the handle-based solve (GPU).

nmpc_solve_noalloc serves callers that may not allocate device memory when
they solve (a real-time control loop that forbids allocation after start-up,
code whose device memory belongs to another allocator, code that must avoid
the device-wide synchronization of cudaMalloc/cudaFree).  It keeps its whole
workspace in a static device array inside the library.  These tests call it
through the C ABI twice in a row (different inputs, so nothing may leak from
the previous call's leftover workspace) and compare each result with the
existing nmpc_setup/nmpc_solve path on the same inputs, within the
tolerance the FP64 solve tests use (1e-9 relative on the controls).
"""
import numpy as np
import pytest

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


def _handle_solve(G, inst, **opts):
    import torch
    s = G.Solver([inst], **opts)
    rc, st = s.solve()
    torch.cuda.synchronize()
    u = s.u.cpu().numpy()
    out = (rc, st[0].status, st[0].iters, st[0].res_inf, u)
    s.close()
    return out


def _noalloc_solve(G, inst, **opts):
    import torch
    x0 = torch.from_numpy(np.ascontiguousarray(inst.x0, dtype=np.float64)).cuda()
    ref = torch.from_numpy(np.ascontiguousarray(inst.ref, dtype=np.float64)).cuda()
    u = torch.full((inst.horizon * len(inst.act),), np.nan, dtype=torch.float64, device="cuda")
    rc, st = G.nmpc_solve_noalloc(inst, x0, ref, u, **opts)
    torch.cuda.synchronize()
    return rc, st.status, st.iters, st.res_inf, u.cpu().numpy()


@pytest.mark.parametrize("mk,opts", [
    (lambda seed: wl.heat1d(32, 20, 2, 0.01, seed=seed, act_pos=[0.25, 0.75]),
     dict(tol=1e-8, precision=0)),
    (lambda seed: wl.heat2d(64, 64, 50, 4, 2, seed=seed), dict(tol=1e-6, precision=1)),
])
def test_noalloc_matches_handle_solve_on_two_calls(G, mk, opts):
    for seed in (1, 2):  # two calls in a row, different inputs
        inst = mk(seed)
        ref = _handle_solve(G, inst, **opts)
        got = _noalloc_solve(G, inst, **opts)
        assert ref[0] == G.NMPC_OK and got[0] == G.NMPC_OK
        assert got[1] == G.NMPC_STATUS_CONVERGED and got[2] == ref[2]
        assert got[3] <= opts["tol"]
        scale = np.abs(ref[4]).max()
        assert np.abs(got[4] - ref[4]).max() <= 1e-9 * scale


def test_noalloc_rejects_instances_beyond_the_static_workspace(G):
    import torch
    inst = wl.heat2d(256, 256, 100, 4, 4, seed=3)  # ~210 MB of state copies
    x0 = torch.zeros(inst.mx * inst.my, dtype=torch.float64, device="cuda")
    u = torch.zeros(inst.horizon * 16, dtype=torch.float64, device="cuda")
    with pytest.raises(G.NmpcError) as e:
        G.nmpc_solve_noalloc(inst, x0, x0, u)
    assert e.value.code == G.NMPC_ERR_UNSUPPORTED
