"""Measurements of the batched and closed-loop workloads (GPU).

    python -m paper_2004_02484_gb300.experiments batch1d   [--n 1024]
    python -m paper_2004_02484_gb300.experiments closedloop [--n 64 --steps 200 --grid 256]
        [--variant 1 --graph 0 --tail-rows -1 --tail-below 0]
    python -m paper_2004_02484_gb300.experiments solve      [--n 8 --grid 256 --graph 1]

batch1d:    the ragged 1D batch (M ~ U{32..256}, N ~ U{10..60}, n_u ~ U{1..4},
            R = 10^U[-3,-1]) solved in one handle, mixed precision, to
            ||K||_inf <= 1e-6, launch shape and inner counts from the
            autotuner (--tune 0: the library defaults; --lines 2 keeps the
            1D stages off the line path); reports solves/s and iterations;
            --graph 0 launches the iterations from the host (a profiler can
            then capture single iteration kernels).
closedloop: the 2D 256x256, N = 100, 16-actuator batch in a receding-horizon
            loop (shifted warm starts, explicit-Euler plant), mixed precision;
            reports solves/s (instances x steps / time), iterations per step,
            the iteration kernel's algorithmic HBM bandwidth and, with
            --check, the float64 residual of sampled returned states.
closedloop_learned: the same loop with the learned start (controls from a
            network on 4x4-pooled plant state and reference, trained on plain
            closed loops of disjoint seeds; state and costate from the
            controls' rollout) against the plain loop on the same instances,
            both as one CUDA graph: iterations per step and solves/s; with
            --rules 1 also the host-driven variants (per-instance choice by
            float64 residual, or always the learned start, rollout or not).
solve:      cold-start solves of the 2D 256x256, N = 100 batch (mixed, to
            ||K||_inf <= 1e-6), one warm-up and --reps timed; with --graph 0
            the iteration loop is launched from the host in chunks instead of
            one graph (a profiler can then capture single iteration kernels);
            reports iterations, ms per iteration and the launch plans.
plate:      the paper's own closed loop (Sec. 5.3, Table 2): one 13x13
            copper plate from the ambient temperature, 200 periods of 5 s,
            the slope reference up to 500 s and then moving linearly to the V
            reference within 50 s; each period one solve from the shifted
            previous solution, stopping at ||K||_inf < --plate-tol (Table 2:
            1), then the plant one period with the first inputs.  Reports
            iterations per period, time per iteration (min over --reps runs
            of each period, the paper's protocol; and device time of 200
            back-to-back iterations), the input range against the bounds and
            the tracking error; then cold solves of --n plates to 1e-6
            (solves/s, iterations).
wave:       second-order-in-time batches (damped nonlinear string, 1D
            m = 64, N = 20; membrane, 2D 32x32, N = 10), cold solves to
            ||K||_inf <= 1e-6 of --n instances each with seeded initial
            fields: solves/s, iterations, time per batch iteration.
Prints one JSON line per experiment.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as wl

G = None  # the library binding, imported by main() once the library is built

BYTES_PER_CELL_STAGE = 32  # read x, lambda; write x, lambda (float64)


def batch1d(n: int, tol: float = 1e-6, reps: int = 3, tune: int = 1, use_graph: int = 1,
            lines: int = 0, persistent: int = 0):
    import torch
    insts = wl.heat1d_ragged_batch(n)
    opts = {}
    if tune:
        from . import autotune as AT
        opts = AT.solver_opts(AT.tune(insts, G.NMPC_MIXED, tol=tol))
    kw = dict(opts)
    if lines or "lines" not in kw:
        kw["lines"] = lines  # an explicit choice overrides the tuned one
    if persistent:
        kw["persistent"] = 1
    s = G.Solver(insts, tol=tol, precision=G.NMPC_MIXED, max_iter=20000, use_graph=use_graph,
                 **kw)
    rc, st = s.solve()
    assert rc == G.NMPC_OK, rc
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        rc, st = s.solve()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    its = np.array([st[b].iters for b in range(n)])
    cells = sum(i.mx * i.horizon for i in insts)
    out = {"experiment": "batch1d", "instances": n, "s_per_batch": dt, "solves_per_s": n / dt,
           "iters_mean": float(its.mean()), "iters_max": int(its.max()),
           "cell_stages": cells, "launches": G.nmpc_launch_count(s.h), "opts": opts,
           "line_plan": G.nmpc_line_plan(s.h),
           "persistent": G.nmpc_launch_plan(s.h)["persistent"]}
    s.close()
    return out


def closedloop(n: int, steps: int, grid: int, horizon: int, n_sub: int, check: int,
               **opts):
    import torch
    insts = wl.heat2d_large_batch(n=n, m=grid, horizon=horizon)
    s = G.Solver(insts, tol=1e-6, precision=G.NMPC_MIXED, max_iter=4000, **opts)
    strip_plan = G.nmpc_strip_plan(s.h)
    w = s.x0.clone()
    nu_tot = sum(len(i.act) for i in insts)
    u_hist = torch.zeros(steps * nu_tot, dtype=torch.float64, device="cuda")
    l0 = G.nmpc_launch_count(s.h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, iters, res = G.nmpc_closed_loop(s.h, w, s.ref, steps, n_sub, n, u_hist)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    launches = G.nmpc_launch_count(s.h) - l0
    iter_launches = int(iters.max(axis=1).sum() + steps)  # kernels that did work (approx.)
    cells = n * horizon * grid * grid
    out = {"experiment": "closedloop", "instances": n, "steps": steps, "grid": grid,
           "horizon": horizon, "rc": rc, "s_total": dt, "solves_per_s": n * steps / dt,
           "iters_first_step_mean": float(iters[0].mean()),
           "iters_later_mean": float(iters[1:].mean()) if steps > 1 else None,
           "res_max": float(res.max()), "launches": launches,
           "iters": iters.tolist(),
           "hbm_gbs_algorithmic": BYTES_PER_CELL_STAGE * cells * iter_launches / dt / 1e9,
           "strip_plan": strip_plan}
    if check:
        # one more solve from the final plant state, then its float64 residual
        rc2, st = G.nmpc_solve(s.h, w, s.ref, s.u, n, init=G.NMPC_INIT_SHIFT)
        x, u, lam = s.state()
        r = G.nmpc_residual(s.h, w, s.ref, x, u, lam, n)
        out["float64_residual_max_recomputed"] = float(r[:, 0].max())
    s.close()
    return out


def solve(n: int, grid: int, horizon: int, reps: int, use_graph: int, **opts):
    import torch
    insts = wl.heat2d_large_batch(n=n, m=grid, horizon=horizon)
    s = G.Solver(insts, tol=1e-6, precision=G.NMPC_MIXED, max_iter=4000, use_graph=use_graph,
                 **opts)
    rc, st = s.solve()
    assert rc == G.NMPC_OK, rc
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        rc, st = s.solve()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    its = np.array([st[b].iters for b in range(n)])
    out = {"experiment": "solve", "instances": n, "grid": grid, "horizon": horizon,
           "use_graph": use_graph, "rc": rc, "s_per_solve": dt, "iters_mean": float(its.mean()),
           "ms_per_iteration": 1e3 * dt / (int(its.max()) + 1),
           "strip_plan": G.nmpc_strip_plan(s.h), "launch_plan": G.nmpc_launch_plan(s.h)}
    s.close()
    return out


def closedloop_learned(n_train: int, train_steps: int, n_test: int, steps: int, grid: int,
                       horizon: int, n_sub: int, fit_steps: int, rules: int = 1):
    import torch
    from . import warmstart as WS
    t0 = time.perf_counter()
    X, U = [], []
    train = wl.heat2d_large_batch(n=n_train, base_seed=7000, m=grid, horizon=horizon)
    for b0 in range(0, n_train, 8):
        x, u = WS.closed_loop_data(train[b0:b0 + 8], train_steps, n_sub)
        X.append(x)
        U.append(u)
    X, U = np.concatenate(X), np.concatenate(U)
    t_gen = time.perf_counter() - t0
    lcs = WS.LearnedControlStart(train[0])
    losses = lcs.fit(X, U, steps=fit_steps)
    test = wl.heat2d_large_batch(n=n_test, base_seed=5000, m=grid, horizon=horizon)
    res = {"experiment": "closedloop_learned", "train_samples": int(X.shape[0]), "gen_s": t_gen,
           "loss_first": losses[0], "loss_last": losses[-1], "instances": n_test, "steps": steps}
    # plain loop (one graph) and learned loop on the same instances
    s = G.Solver(test, tol=1e-6, precision=G.NMPC_MIXED, max_iter=4000)
    w = s.x0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, iters, r = G.nmpc_closed_loop(s.h, w, s.ref, steps, n_sub, n_test)
    torch.cuda.synchronize()
    res.update({"plain_s": time.perf_counter() - t0, "plain_iters_per_step": iters.mean(axis=1).tolist(),
                "plain_rc": rc})
    s.close()
    # the learned loop as one graph (network kernels captured into each step)
    s = G.Solver(test, tol=1e-6, precision=G.NMPC_MIXED, max_iter=4000)
    w = s.x0.clone()
    WS.closed_loop_learned_graph(s, lcs, w, 1, n_sub)  # warm-up (buffers, module load)
    w = s.x0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, iters, r = WS.closed_loop_learned_graph(s, lcs, w, steps, n_sub)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    res.update({"learned_graph_s": dt, "learned_graph_rc": rc,
                "learned_graph_iters_per_step": iters.mean(axis=1).tolist(),
                "learned_graph_solves_per_s": n_test * steps / dt,
                "plain_solves_per_s": n_test * steps / res["plain_s"]})
    s.close()
    for rule, decode in ((("residual", "rollout"), ("always", "rollout"), ("always", "controls"))
                         if rules else ()):
        s = G.Solver(test, tol=1e-6, precision=G.NMPC_MIXED, max_iter=4000)
        w = s.x0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = WS.closed_loop_learned(s, lcs, w, steps, n_sub, rule=rule, decode=decode)
        torch.cuda.synchronize()
        res[rule + "_" + decode] = {"s": time.perf_counter() - t0,
                     "iters_per_step": out["iters"].mean(axis=1).tolist(),
                     "learned_used_per_step": out["learned"].mean(axis=1).tolist(),
                     "res_plain_first_step": float(out["res_plain"][0].max()),
                     "res_learned_first_step": float(out["res_learned"][0].max())}
        s.close()
    return res


def gemm_bench(shapes, reps: int, path_list=(0, 1)):
    """CUDA-event time of nmpc_gemm_bf16 (C = A B^T, BF16 in, FP32 out) per
    shape and GEMM path (0: tcgen05 where the operands allow, 1: mma.sync),
    and of the network passes of the learned start (split-K inside)."""
    import torch
    from . import mlp as GM
    out = []
    for (M, N, K) in shapes:
        A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda").to(torch.bfloat16)
        C = torch.empty(M, N, device="cuda")
        for path in path_list:
            GM.nmpc_gemm_set_path(path)
            for _ in range(3):
                GM.nmpc_gemm_bf16(A, B, C=C)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                GM.nmpc_gemm_bf16(A, B, C=C)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out.append({"M": M, "N": N, "K": K, "path": "tcgen05" if path == 0 else "mma.sync",
                        "us": 1e3 * ms, "tflops": 2.0 * M * N * K / (ms / 1e3) / 1e12})
    GM.nmpc_gemm_set_path(0)
    for widths, batch in (([8192, 512, 512, 512, 1600], 64), ([8192, 512, 512, 512, 6800], 256)):
        for path in path_list:
            GM.nmpc_gemm_set_path(path)
            net = GM.MLP(widths, batch, 0)
            x = torch.randn(batch, widths[0], device="cuda")
            t = torch.randn(batch, widths[-1], device="cuda")
            y = torch.empty(batch, widths[-1], device="cuda")
            for _ in range(3):
                net.forward(x, y)
                net.train_step(x, t, 1e-4, want_loss=False)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            for _ in range(reps):
                net.forward(x, y)
            e[1].record()
            for _ in range(reps):
                net.train_step(x, t, 1e-4, want_loss=False)
            e[2].record()
            torch.cuda.synchronize()
            fl = sum(2.0 * batch * widths[l] * widths[l + 1] for l in range(len(widths) - 1))
            fwd = e[0].elapsed_time(e[1]) / reps
            trn = e[1].elapsed_time(e[2]) / reps
            out.append({"net": widths, "batch": batch,
                        "path": "tcgen05" if path == 0 else "mma.sync",
                        "forward_us": 1e3 * fwd, "forward_tflops": fl / (fwd / 1e3) / 1e12,
                        "train_step_us": 1e3 * trn, "train_tflops": 3 * fl / (trn / 1e3) / 1e12})
            net.close()
    GM.nmpc_gemm_set_path(0)
    return {"experiment": "gemm", "results": out, "tc_error": GM.nmpc_gemm_error(True)}


def plate(n_batch: int, steps: int, variant: int, tol_loop: float, reps: int, n_sub: int,
          precision: int = 0):
    import torch
    from . import plate as GP
    inst = wl.plate_instance()
    slope = wl.plate_reference(inst.m, "slope")
    vee = wl.plate_reference(inst.m, "V")
    is_act = np.zeros(inst.ng, dtype=bool)
    is_act[inst.act] = True
    dt = inst.h

    def reference(t):
        s = min(max((t - 500.0) / 50.0, 0.0), 1.0)
        full = (1.0 - s) * slope + s * vee
        return full[~is_act], full[is_act]

    per_step = np.full(steps, np.inf)
    iters = np.zeros(steps, dtype=np.int64)
    u_hist = np.zeros((steps, len(inst.act)))
    err = np.zeros(steps)
    for rep in range(reps):
        sol = GP.PlateSolver([inst], tol=tol_loop, variant=variant, max_iter=5000,
                             precision=precision)
        w = torch.from_numpy(np.asarray(inst.x0, dtype=np.float64)).cuda()
        for k in range(steps):
            xr, ur = reference(k * dt)
            sol.x_ref.copy_(torch.from_numpy(xr))
            sol.u_ref.copy_(torch.from_numpy(ur))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, st = sol.solve(G.NMPC_INIT_COLD if k == 0 else G.NMPC_INIT_SHIFT, x0=w)
            t1 = time.perf_counter()
            per_step[k] = min(per_step[k], t1 - t0)
            iters[k] = st[0].iters
            u_hist[k] = sol.u[:len(inst.act)].cpu().numpy()
            sol.plant_step(w, dt, n_sub)
            torch.cuda.synchronize()
            err[k] = float(np.abs(w.cpu().numpy() - xr).max())
        sol.close()
    # device time of back-to-back iterations (no convergence polls)
    sol = GP.PlateSolver([inst], variant=variant, precision=precision)
    x = torch.from_numpy(np.tile(inst.x0, inst.horizon)).cuda()
    u = torch.full((inst.horizon * len(inst.act),), 0.5 * (inst.u_lo + inst.u_hi),
                   dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(x)
    sol.iterate(x, u, lam, 20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sol.iterate(x, u, lam, 200)
    e1.record()
    torch.cuda.synchronize()
    it_us = 1e3 * e0.elapsed_time(e1) / 200
    sol.close()
    out = {"experiment": "plate", "variant": "redblack" if variant else "jacobi",
           "precision": "mixed" if precision else "fp64",
           "loop": {"steps": steps, "tol": tol_loop, "n_sub": n_sub,
                    "iters_mean": float(iters.mean()), "iters_max": int(iters.max()),
                    "iters_first": int(iters[0]),
                    "ms_per_iter_min_of_reps": 1e3 * float(per_step.sum() / iters.sum()),
                    "ms_per_step_mean": 1e3 * float(per_step.mean()),
                    "u_min": float(u_hist.min()), "u_max": float(u_hist.max()),
                    "track_err_t500": float(err[min(steps, 100) - 1]),
                    "track_err_end": float(err[-1])},
           "us_per_iter_device": it_us}
    if n_batch:
        insts = wl.plate_batch(n_batch)
        sol = GP.PlateSolver(insts, tol=1e-6, variant=variant, max_iter=20000,
                             precision=precision)
        sol.solve()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = sol.solve()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        its = np.array([s_.iters for s_ in st])
        sol.close()
        out["batch"] = {"n": n_batch, "rc": rc, "solves_per_s": n_batch / t, "ms": 1e3 * t,
                        "iters_mean": float(its.mean()), "iters_max": int(its.max()),
                        "us_per_iter": 1e6 * t / int(its.max())}
    return out


def wave(n: int, variant: int, reps: int, dims=(1, 2), single: bool = True, precision: int = 0):
    import torch
    from . import wave as GW
    out = {"experiment": "wave", "variant": "redblack" if variant else "jacobi",
           "precision": "mixed" if precision else "fp64", "results": []}
    cases = {1: dict(dim=1, m=64, horizon=20), 2: dict(dim=2, m=32, horizon=10, n_act=3)}
    for kw in (cases[d] for d in dims):
        for nb in ((1, n) if single and n > 1 else (n,)):
            insts = [wl.wave_instance(seed=s_, **kw) for s_ in range(nb)]
            sol = GW.WaveSolver(insts, tol=1e-6, variant=variant, max_iter=20000,
                                precision=precision)
            sol.solve()
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                t0 = time.perf_counter()
                rc, st = sol.solve()
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            its = np.array([s_.iters for s_ in st])
            sol.close()
            out["results"].append({"workload": f"wave{kw['dim']}d_m{kw['m']}_N{kw['horizon']}",
                                   "n": nb, "rc": rc, "solves_per_s": nb / best,
                                   "ms": 1e3 * best, "iters_mean": float(its.mean()),
                                   "iters_max": int(its.max()),
                                   "us_per_iter": 1e6 * best / int(its.max())})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["batch1d", "closedloop", "closedloop_learned", "solve",
                                      "gemm", "plate", "wave"])
    ap.add_argument("--shapes", default="4096x4096x4096,256x512x8192,256x6800x512,64x512x8192",
                    help="gemm: MxNxK list")
    ap.add_argument("--paths", default="0,1", help="gemm: 0 tcgen05, 1 mma.sync")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--horizon", type=int, default=100)
    ap.add_argument("--n-sub", type=int, default=2)
    ap.add_argument("--check", type=int, default=1)
    ap.add_argument("--cluster", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--strips", type=int, default=0)
    ap.add_argument("--strip-rows", type=int, default=0)
    ap.add_argument("--n-lo", type=int, default=2, help="solve: Jacobi sweeps per P^-1 solve")
    ap.add_argument("--n-u-it", type=int, default=2, help="solve: u fixed-point iterations")
    ap.add_argument("--strip-cols", type=int, default=0,
                    help="strip path: 0 auto (two columns per lane where eligible), 1 one")
    ap.add_argument("--n-train", type=int, default=64)
    ap.add_argument("--train-steps", type=int, default=12)
    ap.add_argument("--fit-steps", type=int, default=2000)
    ap.add_argument("--graph", type=int, default=1)
    ap.add_argument("--persistent", type=int, default=0,
                    help="batch1d: one launch for the whole solve (line path)")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--rules", type=int, default=1)
    ap.add_argument("--tune", type=int, default=1)
    ap.add_argument("--lines", type=int, default=0)
    ap.add_argument("--plate-tol", type=float, default=1.0)
    ap.add_argument("--precision", type=int, default=0,
                    help="plate, wave: 0 float64, 1 float32 lower layer (NMPC_MIXED)")
    ap.add_argument("--wave-dims", default="1,2", help="wave: 1 string, 2 membrane")
    ap.add_argument("--wave-single", type=int, default=1, help="wave: also time one instance")
    ap.add_argument("--variant", type=int, default=0,
                    help="upper layer: 0 Jacobi (eq. 15), 1 red-black Gauss-Seidel")
    ap.add_argument("--tail-rows", type=int, default=0,
                    help="closedloop: rows of the strip path's tail plan (0 auto, -1 none)")
    ap.add_argument("--tail-below", type=int, default=0,
                    help="closedloop: running instances that select the tail plan (0 auto)")
    a = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    from . import build
    build.build()  # before the binding loads the library (a rebuilt one, if sources changed)
    global G
    from . import nmpc as G
    if a.which == "gemm":
        shapes = [tuple(int(v) for v in sh.split("x")) for sh in a.shapes.split(",") if sh]
        paths = tuple(int(v) for v in a.paths.split(","))
        print(json.dumps(gemm_bench(shapes, a.reps, paths)), flush=True)
    elif a.which == "wave":
        print(json.dumps(wave(256 if a.n is None else a.n, a.variant, max(a.reps, 1),
                              tuple(int(v) for v in a.wave_dims.split(",")), a.wave_single != 0,
                              a.precision)),
              flush=True)
    elif a.which == "plate":
        print(json.dumps(plate(1024 if a.n is None else a.n, a.steps, a.variant, a.plate_tol,
                               max(a.reps, 1), 10 if a.n_sub == 2 else a.n_sub, a.precision)),
              flush=True)
    elif a.which == "batch1d":
        print(json.dumps(batch1d(a.n or 1024, reps=a.reps, tune=a.tune, use_graph=a.graph,
                                 lines=a.lines, persistent=a.persistent)), flush=True)
    elif a.which == "solve":
        print(json.dumps(solve(a.n or 8, a.grid, a.horizon, a.reps, a.graph, strips=a.strips,
                               strip_rows=a.strip_rows, variant=a.variant,
                               strip_cols=a.strip_cols, n_lo=a.n_lo, n_u_it=a.n_u_it)),
              flush=True)
    elif a.which == "closedloop_learned":
        print(json.dumps(closedloop_learned(a.n_train, a.train_steps, a.n or 8, a.steps, a.grid,
                                            a.horizon, a.n_sub, a.fit_steps, a.rules)), flush=True)
    else:
        res = closedloop(a.n or 64, a.steps, a.grid, a.horizon, a.n_sub, a.check,
                         cluster=a.cluster, threads=a.threads, strips=a.strips,
                         strip_rows=a.strip_rows, variant=a.variant, use_graph=a.graph,
                         tail_rows=a.tail_rows, tail_below=a.tail_below)
        res.update({"cluster": a.cluster, "threads": a.threads})
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
