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

The entry point always runs the cluster path (or, for a stage too large for
a cluster, one CTA per stage over a slab in the static array).  Where the
handle would pick another path (the line path for a mixed-precision 1D
instance, the strip path for a large 2D stage) both results are roots of the
same KKT system to the same float64 tolerance, so their controls agree to
the float32-path bound of 1e-3 relative.
"""
import os
import subprocess
import sys

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


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_noalloc_mixed_1d_instance_against_the_line_path(G):
    # the handle runs this instance on the line path (one warp per stage);
    # the allocation-free entry point on the cluster path
    inst = wl.heat1d(96, 30, 3, 0.01, seed=41)
    opts = dict(tol=1e-6, precision=1)
    ref = _handle_solve(G, inst, **opts)
    got = _noalloc_solve(G, inst, **opts)
    assert ref[0] == G.NMPC_OK and got[0] == G.NMPC_OK
    assert got[1] == G.NMPC_STATUS_CONVERGED and got[3] <= 1e-6
    assert _rel(got[4], ref[4]) <= 1e-3


def test_noalloc_global_slab_stage_against_the_strip_path(G):
    # a 320x320 stage fits no cluster of shared-memory slabs, so this entry
    # point runs one CTA per stage over a slab in the static array (about
    # 23 MB of its 32 MiB); the handle puts the instance on the strip path
    inst = wl.heat2d(320, 320, 3, 2, 2, seed=43)
    opts = dict(tol=1e-6, precision=1)
    ref = _handle_solve(G, inst, **opts)
    got = _noalloc_solve(G, inst, **opts)
    assert ref[0] == G.NMPC_OK and got[0] == G.NMPC_OK
    assert got[1] == G.NMPC_STATUS_CONVERGED and got[3] <= 1e-6
    assert _rel(got[4], ref[4]) <= 1e-3


def test_noalloc_rejects_a_forced_strip_or_line_path(G):
    import torch
    inst = wl.heat1d(32, 4, 1, 0.01, seed=5)
    x0 = torch.zeros(inst.mx, dtype=torch.float64, device="cuda")
    u = torch.zeros(inst.horizon, dtype=torch.float64, device="cuda")
    for forced in (dict(lines=1), dict(strips=1)):
        with pytest.raises(G.NmpcError) as e:
            G.nmpc_solve_noalloc(inst, x0, x0, u, precision=1, **forced)
        assert e.value.code == G.NMPC_ERR_UNSUPPORTED


_FIRST_CALL_SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2004_02484_gb300 import nmpc as G
from paper_2004_02484_gb300 import workloads as wl
torch.cuda.set_device(0)
inst = wl.heat2d(64, 64, 50, 4, 2, seed=7)
x0 = torch.from_numpy(inst.x0).cuda()
rf = torch.from_numpy(inst.ref).cuda()
u = torch.zeros(inst.horizon * len(inst.act), dtype=torch.float64, device="cuda")
rc, st = G.nmpc_solve_noalloc(inst, x0, rf, u, tol=1e-8, precision=0)
torch.cuda.synchronize()
s = G.Solver([inst], tol=1e-8, precision=0)
rc2, st2 = s.solve()
torch.cuda.synchronize()
ref_u = s.u.cpu().numpy()
s.close()
got_u = u.cpu().numpy()
err = float(np.abs(got_u - ref_u).max() / np.abs(ref_u).max())
print("RESULT", rc, rc2, st.iters, st2[0].iters, err)
"""


def test_noalloc_first_call_in_a_fresh_process_matches_the_handle_solve():
    # the very first library call of the process is the allocation-free
    # solve (no handle has configured the kernels before it): its launch plan,
    # hence its iterates, must be the handle's
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    from paper_2004_02484_gb300 import build as b
    b.build()
    out = subprocess.run([sys.executable, "-c", _FIRST_CALL_SCRIPT, root], capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [l for l in out.stdout.splitlines() if l.startswith("RESULT")][-1].split()
    rc, rc2, it, it2, err = int(line[1]), int(line[2]), int(line[3]), int(line[4]), float(line[5])
    assert rc == 0 and rc2 == 0
    assert it == it2
    assert err <= 1e-9
