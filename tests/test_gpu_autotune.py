"""Autotuner (GPU): picks a converging launch shape / inner-iteration setting,
caches it by problem signature, and the tuned solve reaches the same root."""
import json
import os

import numpy as np
import pytest

from paper_2004_02484_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_tune_caches_and_keeps_the_root(tmp_path):
    from paper_2004_02484_gb300 import build as b
    b.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2004_02484_gb300 import autotune as AT
    from paper_2004_02484_gb300 import nmpc as G
    insts = wl.heat1d_ragged_batch(16)
    cache = str(tmp_path / "tune.json")
    res = AT.tune(insts, G.NMPC_MIXED, tol=1e-7, cache_path=cache)
    assert res["s_per_solve"] > 0
    assert os.path.exists(cache)
    key = AT.signature(insts, G.NMPC_MIXED)
    assert key in json.load(open(cache))
    again = AT.tune(insts, G.NMPC_MIXED, tol=1e-7, cache_path=cache)
    assert again == res  # served from the cache
    s1 = G.Solver(insts, tol=1e-8, precision=G.NMPC_MIXED)
    s2 = G.Solver(insts, tol=1e-8, precision=G.NMPC_MIXED, **AT.solver_opts(res))
    rc1, st1 = s1.solve()
    rc2, st2 = s2.solve()
    assert rc1 == rc2 == G.NMPC_OK
    u1, u2 = s1.u.cpu().numpy(), s2.u.cpu().numpy()
    assert np.abs(u1 - u2).max() <= 1e-3 * np.abs(u1).max()
    s1.close()
    s2.close()


def test_tune_large_2d_batch_over_strip_shapes(tmp_path):
    from paper_2004_02484_gb300 import build as b
    b.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2004_02484_gb300 import autotune as AT
    from paper_2004_02484_gb300 import nmpc as G
    insts = wl.heat2d_large_batch(n=2, m=256, horizon=8)
    res = AT.tune(insts, G.NMPC_MIXED, tol=1e-6, cache_path=str(tmp_path / "t.json"))
    opts = AT.solver_opts(res)
    assert opts["strips"] == 1 and opts["strip_rows"] in (0, 64)
    s = G.Solver(insts, tol=1e-6, precision=G.NMPC_MIXED, **opts)
    assert G.nmpc_strip_plan(s.h)["instances"] == 2
    rc, st = s.solve()
    assert rc == G.NMPC_OK and all(st[b].res_inf <= 1e-6 for b in range(2))
    s.close()
