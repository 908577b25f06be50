"""Autotuner for the solve's launch shape and inner-iteration counts.

For a batch of instances it times complete solves (through the C ABI, on the
GPU) over a small candidate set and keeps the fastest configuration that
converges: CTAs per stage (thread-block cluster size), threads per CTA,
iterations per host poll (graph chunk length), lower-layer sweeps n_lo and
u-iterations n_u_it.  The KKT root does not depend on these (the lower layer
is a fixed linear approximation of D_i^{-1} and the iteration's fixed point
is K(S) = 0), only the iteration count and the time per iteration do.  The
u-iteration's form (through the actuators' local responses or full-field
sweeps) is a candidate as well.  Batches of large 2D stages (the strip path:
one warp per strip of the stage grid) are tuned over the strip's own rows
and the inner counts instead, and mixed-precision batches of 1D stages (the
line path: one warp per stage) over the inner counts, with the cluster path
as one more candidate.

Results are cached in a JSON file keyed by a bucketed signature of the batch
(dimension, grid size, horizon, actuators, batch size, precision).
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time
from typing import Dict, List, Sequence

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json")


def _bucket(v: float) -> int:
    return int(round(math.log2(max(1.0, float(v)))))


def signature(instances: Sequence, precision: int) -> str:
    ng = [i.mx * i.my for i in instances]
    return json.dumps({
        "dim": sorted({i.dim for i in instances}),
        "ng": [_bucket(min(ng)), _bucket(max(ng))],
        "N": [_bucket(min(i.horizon for i in instances)), _bucket(max(i.horizon for i in instances))],
        "nu": _bucket(max(len(i.act) for i in instances)),
        "batch": _bucket(len(instances)),
        "precision": int(precision),
    }, sort_keys=True)


# stages from this many cells up are on the strip path (the auto rule of the
# library: larger than a cluster of 8 CTAs with staged inputs holds)
STRIP_CELLS = 16384


# 1D stages of at most this many cells run on the line path (mixed precision)
LINE_MAX_CELLS = 256
MIXED = 1  # NMPC_MIXED


def candidates(instances: Sequence, quick: bool = True, precision: int = -1) -> List[Dict]:
    """Option sets to time.  With ``precision`` = NMPC_MIXED, batches of 1D
    instances that all run on the line path (one warp per stage; no launch
    shape to choose) are tuned over the inner counts, plus the cluster path
    with its automatic shape as a fallback candidate."""
    ngmax = max(i.mx * i.my for i in instances)
    if precision == MIXED and all(i.dim == 1 and i.mx <= LINE_MAX_CELLS for i in instances):
        inner = [(2, 1), (2, 2), (1, 1)] if quick else [(2, 1), (2, 2), (1, 1), (1, 2), (3, 1)]
        out = [{"lines": 0, "n_lo": nlo, "n_u_it": nut, "check_every": 16} for nlo, nut in inner]
        return out + [{"lines": 2, "n_lo": 2, "n_u_it": 1, "check_every": 16}]
    if all(i.dim == 2 and i.mx * i.my >= STRIP_CELLS for i in instances):
        rows = (0, 64) if quick else (0, 32, 64, 128)
        inner = [(2, 1), (2, 2), (1, 1)] if quick else [(2, 1), (2, 2), (1, 1), (1, 2), (3, 1)]
        return [{"strips": 1, "strip_rows": r, "n_lo": nlo, "n_u_it": nut, "check_every": 16}
                for r in rows for nlo, nut in inner]
    clusters = [0, 1] if ngmax < 1024 else [0, 2, 4, 8]
    threads = [0, 256] if quick else [0, 64, 128, 256, 512]
    inner = ([(2, 2), (2, 1), (2, 3), (1, 1), (1, 2), (3, 2)] if not quick
             else [(2, 2), (2, 1), (1, 1)])
    out = []
    cells = (0,) if quick else (0, 4)
    for c, t, (nlo, nut), ul, ce in itertools.product(clusters, threads, inner, (1, 0), cells):
        if ce == 4 and t > 384:
            continue
        out.append({"cluster": c, "threads": t, "n_lo": nlo, "n_u_it": nut, "u_local": ul,
                    "cells": ce, "check_every": 16})
    return out


def _time_config(G, instances, precision, tol, cfg, reps=2):
    """(seconds per solve, None) or (None, reason)."""
    import torch
    try:
        s = G.Solver(instances, tol=tol, precision=precision, max_iter=6000, **cfg)
    except Exception as e:  # an invalid combination for this batch
        return None, f"setup: {e}"
    try:
        rc, st = s.solve()  # warm-up (graph capture)
        if rc != G.NMPC_OK:
            return None, f"solve rc {rc}"
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            rc, _ = s.solve()
            if rc != G.NMPC_OK:
                return None, f"solve rc {rc}"
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps, None
    finally:
        s.close()


def tune(instances: Sequence, precision: int, tol: float = 1e-6, cache_path: str = DEFAULT_CACHE,
         quick: bool = True, force: bool = False, verbose: bool = False) -> Dict:
    """Best option set for this batch (cached).  Returns the nmpc_opts fields
    to pass to ``Solver``/``nmpc_setup`` plus the measured seconds per solve."""
    from . import nmpc as G
    key = signature(instances, precision)
    cache = {}
    if os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache and not force:
        return cache[key]
    best, best_t, reasons = None, float("inf"), []
    for cfg in candidates(instances, quick, precision):
        t, why = _time_config(G, instances, precision, tol, cfg)
        if verbose:
            print(json.dumps({"cfg": cfg, "s_per_solve": t, "error": why}), flush=True)
        if why:
            reasons.append(why)
        if t is not None and t < best_t:
            best, best_t = cfg, t
    if best is None:
        raise RuntimeError("no candidate configuration converged: " + "; ".join(reasons[:4]))
    result = dict(best, s_per_solve=best_t)
    cache[key] = result
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return result


def solver_opts(result: Dict) -> Dict:
    """The nmpc_opts fields of a tuning result."""
    return {k: v for k, v in result.items() if k in ("cluster", "threads", "n_lo", "n_u_it",
                                                     "u_local", "cells", "check_every",
                                                     "strips", "strip_rows", "lines")}
