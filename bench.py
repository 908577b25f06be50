"""Benchmark: solves/s of the double-layer Jacobi NMPC method on one GB300.

Headline workload: a batch of 64 instances of the 2D nonlinear heat equation
(256 x 256 cells, N = 100 stages, 16 actuators, dt = 2e-5) in a receding-
horizon closed loop, FP32 lower layer with float64 residual, norms and
update, every solve to ||K||_inf <= 1e-6.  A step is one step of the loop:
one solve of each of the 64 instances (64 solves) plus the plant's advance.
The loop runs as one CUDA graph; K steps are timed from the loop's start
(first solve from the cold or learned start, later ones warm).  The upper
layer is the red-black ordering of the block Gauss-Seidel variant (two
stage-parallel half-sweeps per iteration; Theorem 3: the Jacobi factor
squared); ``--variant jacobi`` times the stage-parallel Jacobi iteration of
eq. 15, and the line also carries the plain loop of the other variant.

Two arms in one run, on the same instances:
  plain    the plain method: cold first step, then the shifted previous
           solution (Sec. 5.3's warm start);
  learned  every step starts from a network's control trajectory (4x4-pooled
           plant state and reference in, BF16 tensor-core MLP), completed by
           its state and costate trajectories; the network is trained before
           the timed region on plain closed loops of 64 other instances.
value = learned solves/s; the plain rate and the gain are reported beside it.
The state (6.7 GB per iterate) is far larger than the 129 MB L2, so no L2
flush is needed between steps.

Also in the JSON line: the strip kernel's HBM roofline (algorithmic bytes
over its CUDA-event time, from a timing leg outside the graph), the float64
oracle on the host cores (a complete solve of one instance, and the control
error of the GPU's first-step solves against it), an end-to-end rate with
host buffers, and the 64x64 single-instance workload as a secondary line.

Under torchrun (N > 1) every rank runs its own 64 instances (disjoint seeds;
instances are independent, so there is no data-path collective): value =
solves of all ranks / max-over-ranks time.

``--impl reference`` times the FP64 C oracle on the host cores on the same
workload: complete solves of the batch's instances, one after the other.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Solves/s to KKT res≤1e-6, batched+learned vs plain; HBM GB/s vs peak"
WORKLOAD = ("heat2d_256x256_N100_x64_closed_loop: 64 instances of the 2D nonlinear heat eq. "
            "k(w)=0.1(1+0.5w), 256x256 grid, dt=2e-5, N=100, 16 actuators (4x4), Gaussian-bump "
            "references (centre U[0.3,0.7]^2, amp U[0.5,1.5]), 16-mode sine initial fields; "
            "receding-horizon loop in one CUDA graph, FP32 lower layer + FP64 residual, "
            "tol ||K||_inf<=1e-6 per solve")
WORKLOAD_2 = ("heat2d_64x64_N50: 64x64 grid, dt=2e-5, N=50, 8 actuators (2x4), single instance, "
              "plain double-layer Jacobi from the cold start, tol 1e-6")
TOL = 1e-6
N_INST = 64
N_SUB = 2          # explicit-Euler plant sub-steps per sampling period
TRAIN_STEPS = 12   # closed-loop steps of the training instances
TRAIN_BATCHES = 8  # batches of training instances (8 x 64 instances: 6144 samples)
FIT_STEPS = 1500   # Adam steps of the learned start
# algorithmic bytes per cell-stage per iteration: read x_i, lambda_i and write
# them back in float64 (the neighbour-stage reads are the same arrays)
BYTES_PER_POINT_STAGE = 32
# DRAM bytes over algorithmic bytes of the strip kernel (two columns per
# lane), from ncu captures on 8 instances (dram__bytes_read.sum + write.sum
# per launch over 32 B x the launch's cell-stages): Jacobi 1.741 GB / 1.678
# GB; red-black half 0 1.317 GB and half 1 1.307 GB over 0.839 GB each (the
# neighbouring stages' x_{i-1}, lambda_{i+1} are not processed in the same
# launch, so they come from DRAM rather than L2)
TRAFFIC_RATIO = {"jacobi": 1.741 / 1.678, "redblack": (1.317 + 1.307) / (2 * 0.839)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances", type=int, default=N_INST)
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--horizon", type=int, default=100)
    ap.add_argument("--oracle", type=int, default=1,
                    help="1: time the C oracle on the host (rank 0) and compare controls")
    ap.add_argument("--secondary", type=int, default=1,
                    help="1: also time the 64x64 single-instance workload")
    ap.add_argument("--variant", default="redblack", choices=["jacobi", "redblack"],
                    help="upper-layer iteration: the red-black ordering of the block Gauss-Seidel "
                         "variant (default; Theorem 3: the Jacobi factor squared) or the "
                         "stage-parallel Jacobi iteration of eq. 15")
    ap.add_argument("--compare", type=int, default=1,
                    help="1: also time the plain loop with the other upper-layer variant")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def batch_seed(rank: int, train: bool = False) -> int:
    """First seed of a rank's batch: ranks solve disjoint instances (replicas,
    no data-path collective); training instances never overlap test ones."""
    return (7000 if train else 5000) + 100_000 * rank


def step_seed(step: int, rank: int) -> int:
    """Seed of the secondary workload's field at a rank's step: step 0 of
    rank 0 is the canonical seed-1 field."""
    return 1 if (step == 0 and rank == 0) else 100_000 + 1000 * rank + step


def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks of the process group (x itself when
    there is none): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, solves: int, seconds: float) -> float:
    """Whole-job solves/s: every rank's solves over the slowest rank's time."""
    return world * solves / seconds


def ref_chunk(steps: int, iters_budget: int = 300) -> int:
    """Oracle iterations per reference step: the K timed steps together run
    about iters_budget iterations (more than one complete solve of an
    instance of the batch), at least one per step."""
    return max(1, math.ceil(iters_budget / max(1, steps)))


class ClockSampler:
    """nvidia-smi samples every 100 ms during the timed region: entering
    waits (up to 3 s) for the sampler's first line, and the summary covers
    the lines read from then on."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index  # nvidia-smi -i selector: a GPU UUID or a physical index
        self.rows = []
        self.proc = None
        self.start = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.time() + 3.0
            while not self.rows and time.time() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
            self.start = len(self.rows)  # samples from here on fall in the timed region
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # the timed region's samples (the last one before it when it was too
        # short to hold one)
        rows = self.rows[self.start:] or self.rows[-1:]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for n, v in zip(names, r[4:8]):
                    if v.lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def smi_selector(dev: int) -> str:
    """The nvidia-smi -i selector of CUDA device `dev` of this process.

    nvidia-smi numbers physical GPUs and ignores CUDA_VISIBLE_DEVICES, so the
    device's UUID is used (torch reports it without the "GPU-" prefix); failing
    that, the dev-th entry of a numeric CUDA_VISIBLE_DEVICES, else dev."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(dev).uuid)
        if u and u.lower() != "none":
            return u if u.startswith(("GPU-", "MIG-")) else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    if dev < len(ids):
        return ids[dev]
    return str(dev)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def batch(args, rank, train=False, part=0):
    """The rank's test batch, or part `part` of its training instances (seeds
    following one another from the training base)."""
    from paper_2004_02484_gb300 import workloads as wl
    return wl.heat2d_large_batch(n=args.instances,
                                 base_seed=batch_seed(rank, train) + part * args.instances,
                                 m=args.grid, horizon=args.horizon)


# ---------------------------------------------------------------------------
# reference arm: the FP64 C oracle on the host cores
# ---------------------------------------------------------------------------
def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import c_oracle as C
    cores = C.set_threads(host_cores())
    insts = batch(args, 0)
    chunk = ref_chunk(args.steps)
    # warm-up: single iterations of the last instance (untimed)
    pw = C.Problem(insts[-1])
    S = pw.cold_start()
    for _ in range(args.warmup):
        X, U, L, _ = C.jacobi_iteration(pw, *S)
        S = (X, U, L)
    # timed: the batch's instances solved from the cold start one after the
    # other, `chunk` iterations per step (a solve resumes across steps)
    b = 0
    p = C.Problem(insts[b])
    S = p.cold_start()
    done_at, n_done, t_steps = [], 0, []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ts = time.perf_counter()
        left = chunk
        while left > 0:
            S, info = C.solve_jacobi(p, S0=S, tol=TOL, max_iter=left)
            left -= max(1, info["iters"])
            if info["converged"] or info["diverged"]:
                n_done += 1
                done_at.append(time.perf_counter() - t0)
                b = (b + 1) % len(insts)
                p = C.Problem(insts[b])
                S = p.cold_start()
        t_steps.append(time.perf_counter() - ts)
    total = time.perf_counter() - t0
    value = n_done / done_at[-1] if n_done else 0.0
    sample = (f"complete FP64 C-oracle solves (cold start, n_lo=2, n_u_it=2, tol 1e-6) of the "
              f"batch's instances one after the other, {chunk} iterations per step, {cores} "
              f"threads over stages; value = {n_done} completed solve(s) / their time")
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": WORKLOAD, "tol": TOL},
                      "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores,
                                       "kind": "oracle", "sample": sample},
                      "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def solver_opts(args):
    from paper_2004_02484_gb300 import nmpc as G
    o = dict(tol=TOL, precision=G.NMPC_MIXED, max_iter=4000)
    if args.variant == "redblack":
        o["variant"] = G.NMPC_VARIANT_REDBLACK
    return o


def secondary(args, rank, world, dev):
    """The 64x64 single-instance workload: 50 timed solves of distinct fields
    (L2 flushed between them, outside the per-solve events)."""
    import torch
    from paper_2004_02484_gb300 import nmpc as G
    from paper_2004_02484_gb300 import workloads as wl
    n_steps, n_warm = 50, 3
    insts = [wl.heat2d_single(seed=step_seed(s, rank)) for s in range(n_warm + n_steps)]
    # the settings the autotuner picks for this workload (n_lo = 1, n_u_it = 1,
    # clusters of 8 CTAs per stage)
    # (the Jacobi upper layer: on this latency-bound workload, ~20 us per
    # launch, red-black's two launches per iteration cost more than its
    # halved iteration count saves: 2.72 against 2.3 ms per solve)
    o = dict(tol=TOL, precision=G.NMPC_MIXED, max_iter=5000, n_lo=1, n_u_it=1, cluster=8)
    s = G.Solver([insts[0]], **o)
    x0s = [torch.from_numpy(G.pack_fields([i], "x0")).to(dev) for i in insts]
    refs = [torch.from_numpy(G.pack_fields([i], "ref")).to(dev) for i in insts]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    for k in range(n_warm):
        rc, _ = G.nmpc_solve(s.h, x0s[k], refs[k], s.u, 1, stream=st)
        assert rc == G.NMPC_OK, rc
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(n_steps)]
    its = []
    torch.cuda.synchronize()
    for k in range(n_steps):
        flush.zero_()
        ev[k][0].record(st)
        rc, stt = G.nmpc_solve(s.h, x0s[n_warm + k], refs[n_warm + k], s.u, 1, stream=st)
        ev[k][1].record(st)
        assert rc == G.NMPC_OK and stt[0].res_inf <= TOL, rc
        its.append(stt[0].iters)
    torch.cuda.synchronize()
    t_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev)
    # kernel timing: the same solves without graphs, CUDA events per launch
    s2 = G.Solver([insts[0]], use_graph=0, **o)
    G.nmpc_kernel_timing(s2.h, True)
    kits = 0
    for k in range(5):
        rc, stt = G.nmpc_solve(s2.h, x0s[n_warm + k], refs[n_warm + k], s2.u, 1, stream=st)
        kits += stt[0].iters
    kt = G.nmpc_kernel_times(s2.h)
    s2.close()
    s.close()
    n_l, ms_l = kt["k_iterate"]
    cells = insts[0].horizon * insts[0].ng
    peaks, which = measured_peaks()
    ach = BYTES_PER_POINT_STAGE * cells / (ms_l / max(1, n_l) / 1e3) / 1e9 if n_l else None
    return {"workload": WORKLOAD_2, "value": job_rate(world, n_steps, t_ms / 1e3),
            "unit": "solves/s", "ms_per_solve": t_ms / n_steps,
            "iterations_per_solve": {"min": min(its), "max": max(its),
                                     "mean": sum(its) / len(its)},
            "roofline": {"bound": "latency (L2-resident, ~10 warps/SM)", "kernel": "k_iterate",
                         "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"] if ach else None,
                         "avg_launch_us": 1e3 * ms_l / max(1, n_l), "timed_launches": n_l},
            "opts": {k: v for k, v in o.items() if k != "precision"}}


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2004_02484_gb300 import build as b
    b.build()
    from paper_2004_02484_gb300 import nmpc as G
    from paper_2004_02484_gb300 import warmstart as WS
    dev = torch.device("cuda", local)
    opts = solver_opts(args)
    test = batch(args, rank)
    train = [batch(args, rank, train=True, part=q) for q in range(TRAIN_BATCHES)]
    K, W, B = args.steps, args.warmup, len(test)
    ng, N = test[0].mx * test[0].my, test[0].horizon
    nu = len(test[0].act)

    # ---- learned start: trained on plain closed loops of other instances ----
    t0 = time.perf_counter()
    # plain closed loops of the training instances, one batch at a time
    data = [WS.closed_loop_data(tb, TRAIN_STEPS, N_SUB) for tb in train]
    X, U = np.concatenate([d[0] for d in data]), np.concatenate([d[1] for d in data])
    del data
    lcs = WS.LearnedControlStart(train[0][0], max_batch=max(256, B))
    losses = lcs.fit(X, U, steps=FIT_STEPS)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    def plain_loop(steps, u_hist=None):
        s = G.Solver(test, **opts)
        w = s.x0.clone()
        torch.cuda.synchronize()
        return s, w

    # ---- plain arm ----
    s, w = plain_loop(W)
    G.nmpc_closed_loop(s.h, w, s.ref, W, N_SUB, B)  # warm-up loop (graph build, clocks)
    s.close()
    s, w = plain_loop(K)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(smi_selector(local)) as clk_p:
        e0.record(stream)
        rc_p, it_p, res_p = G.nmpc_closed_loop(s.h, w, s.ref, K, N_SUB, B)
        e1.record(stream)
        torch.cuda.synchronize()
    t_plain = max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
    assert rc_p == G.NMPC_OK and float(res_p.max()) <= TOL, (rc_p, float(res_p.max()))
    s.close()

    # ---- learned arm ----
    s = G.Solver(test, **opts)
    w = s.x0.clone()
    WS.closed_loop_learned_graph(s, lcs, w, W, N_SUB)  # warm-up loop
    s.close()
    s = G.Solver(test, **opts)
    w = s.x0.clone()
    u_guess = torch.empty(s.n_u, dtype=torch.float64, device=dev)
    m0 = lcs.net.launch_count()
    lcs.predict_u_into(w, s.ref, B, u_guess)  # buffers for this batch, outside the capture
    mlp_launches = lcs.net.launch_count() - m0 + 3  # + 2 pooling launches + 1 cast
    l0 = G.nmpc_launch_count(s.h)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(smi_selector(local)) as clk_l:
        e0.record(stream)
        rc_l, it_l, res_l = G.nmpc_closed_loop_learned(
            s.h, w, s.ref, K, N_SUB, B,
            lambda st: lcs.predict_u_into(w, s.ref, B, u_guess, st), u_guess)
        e1.record(stream)
        torch.cuda.synchronize()
    t_learned = max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
    launches = G.nmpc_launch_count(s.h) - l0 + K * mlp_launches
    assert rc_l == G.NMPC_OK and float(res_l.max()) <= TOL, (rc_l, float(res_l.max()))
    s.close()

    # ---- the plain loop with the other upper-layer variant (context) ----
    other = None
    if args.compare:
        from paper_2004_02484_gb300 import nmpc as G2
        o2 = dict(opts)
        o2["variant"] = (G2.NMPC_VARIANT_JACOBI if args.variant == "redblack"
                         else G2.NMPC_VARIANT_REDBLACK)
        s = G.Solver(test, **o2)
        w = s.x0.clone()
        torch.cuda.synchronize()
        e0.record(stream)
        rc_o, it_o, res_o = G.nmpc_closed_loop(s.h, w, s.ref, K, N_SUB, B)
        e1.record(stream)
        torch.cuda.synchronize()
        t_o = max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
        s.close()
        other = {"variant": "jacobi" if args.variant == "redblack" else "redblack",
                 "plain_value": job_rate(world, B * K, t_o), "unit": "solves/s",
                 "iterations_per_solve_mean": float(np.mean(it_o)), "rc": rc_o}

    # ---- end to end through host buffers: every step the measured plant
    # state goes host -> device, one loop step runs, the applied controls and
    # the plant's next state come back ----
    s = G.Solver(test, **opts)
    w = s.x0.clone()
    w_host = s.x0.cpu().pin_memory()
    u1_host = torch.empty(B * nu, dtype=torch.float64).pin_memory()
    u1_dev = torch.empty(B * nu, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        w.copy_(w_host, non_blocking=True)
        rc, _, _ = G.nmpc_closed_loop_learned(
            s.h, w, s.ref, 1, N_SUB, B,
            lambda st: lcs.predict_u_into(w, s.ref, B, u_guess, st), u_guess, u_hist=u1_dev)
        u1_host.copy_(u1_dev, non_blocking=True)
        w_host.copy_(w, non_blocking=True)
        torch.cuda.synchronize()
        assert rc == G.NMPC_OK
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    s.close()

    # ---- strip-kernel roofline: the learned loop's first steps without the
    # graph, a CUDA event pair around every launch ----
    s = G.Solver(test, use_graph=0, **opts)
    w = s.x0.clone()
    G.nmpc_kernel_timing(s.h, True)
    t0 = time.perf_counter()
    kt_steps = 2
    rc, it_k, _ = G.nmpc_closed_loop_learned(
        s.h, w, s.ref, kt_steps, N_SUB, B,
        lambda st: lcs.predict_u_into(w, s.ref, B, u_guess, st), u_guess)
    torch.cuda.synchronize()
    t_kt = time.perf_counter() - t0
    kt = G.nmpc_kernel_times(s.h)
    plan = G.nmpc_strip_plan(s.h)
    s.close()
    n_s, ms_s = kt["k_strip"]
    # units: every running instance's full iterations (the final residual-only
    # pass of each solve is not counted)
    cell_stage_iters = float(np.asarray(it_k).sum()) * N * ng
    alg_bytes = BYTES_PER_POINT_STAGE * cell_stage_iters
    peaks, which = measured_peaks()
    achieved = alg_bytes / (ms_s / 1e3) / 1e9 if ms_s > 0 else None
    traffic = TRAFFIC_RATIO[args.variant] * alg_bytes / max(1, n_s)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"] if achieved else None, "traffic": traffic,
            "traffic_source": "ncu dram__bytes_read.sum + write.sum of the same kernels on 8 "
                              "instances, scaled by the cell-stages per launch",
            "peak_source": which,
            "kernel": (f"k_strip2<2> (strip path, two columns per lane: residual, lower layer "
                       f"and update of {plan['strip_x']}-column strips of 256x256 stages)"
                       if plan["strip_x"] > 32 else
                       f"k_strip<float,2> (strip path: residual, lower layer and update of "
                       f"{plan['strip_x']}-column strips of 256x256 stages)"),
            "algorithmic_bytes_per_launch": alg_bytes / max(1, n_s),
            # the DRAM bytes a launch moves (traffic) over its live duration:
            # the red-black halves read the other half's stages from DRAM
            "dram_achieved": (traffic / (ms_s / max(1, n_s) / 1e3) / 1e9) if ms_s > 0 else None,
            "dram_frac": (traffic / (ms_s / max(1, n_s) / 1e3) / 1e9 / peaks["hbm_gbs"])
                         if ms_s > 0 else None,
            "avg_launch_ms": ms_s / max(1, n_s), "timed_launches": n_s,
            "kernel_share_of_step": {k: v[1] / (1e3 * t_kt) for k, v in kt.items() if v[0]},
            "strip_plan": plan,
            "per_unit": "32 B per cell-stage per iteration (x_i, lambda_i read and written "
                        "in float64); units = sum over solves of iterations x N x cells"}

    # ---- float64 oracle on the host (rank 0): a complete solve of instance 0
    # from its cold start (the timed CPU baseline), then the same solve
    # continued to 1e-8 as the reference for the GPU's first-step controls ----
    cpu, ctrl_err = None, None
    if rank == 0 and args.oracle:
        from oracle import c_oracle as C
        cores = C.set_threads(host_cores())
        p = C.Problem(test[0])
        t0 = time.perf_counter()
        S, info = C.solve_jacobi(p, tol=TOL, max_iter=4000)
        t_or = time.perf_counter() - t0
        cpu = {"value": 1.0 / t_or, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": f"one complete FP64 C-oracle solve (cold start, n_lo=2, n_u_it=2, "
                         f"tol 1e-6: {info['iters']} iterations, {t_or:.1f} s) of instance 0 "
                         f"of the batch, {cores} threads over stages"}
        S8, info8 = C.solve_jacobi(p, S0=S, tol=1e-8, max_iter=4000)
        U_ora = S8[1]
        # the GPU's first-step solves of instance 0: plain (cold) and learned
        errs = {}
        for arm in ("plain", "learned"):
            s1 = G.Solver([test[0]], **opts)
            w1 = s1.x0.clone()
            if arm == "plain":
                rc1, _ = s1.solve()
            else:
                ug = torch.empty(s1.n_u, dtype=torch.float64, device=dev)
                lcs.predict_u_into(w1, s1.ref, 1, ug)
                torch.cuda.synchronize()
                rc1, _, _ = G.nmpc_closed_loop_learned(
                    s1.h, w1, s1.ref, 1, N_SUB, 1,
                    lambda st: lcs.predict_u_into(w1, s1.ref, 1, ug, st), ug)
            _, u_gpu, _ = s1.state()
            u_gpu = u_gpu.cpu().numpy().reshape(N, nu)
            s1.close()
            errs[arm] = float(np.abs(u_gpu - U_ora).max() / np.abs(U_ora).max())
        ctrl_err = {"max_rel_error_first_step": errs, "instances": [0],
                    "reference": f"FP64 C oracle solved to ||K||_inf<=1e-8 "
                                 f"({info['iters'] + info8['iters']} iterations)",
                    "definition": "max|U_gpu - U_oracle| / max|U_oracle| over the 100x16 "
                                  "control trajectory"}

    sec = secondary(args, rank, world, dev) if args.secondary else None

    if rank == 0:
        value = job_rate(world, B * K, t_learned)
        plain = job_rate(world, B * K, t_plain)
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
               "steps": K, "warmup": W, "ms_per_step": 1e3 * t_learned / K,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f32+f64", "data": "synthetic",
               "config": {"workload": WORKLOAD, "instances_per_rank": B, "steps_timed": K,
                          "variant": args.variant, "n_sub_plant": N_SUB,
                          "solves_per_step": B, "timed_from": "the loop's first step",
                          "l2": "state of 6.7 GB per iterate, far larger than L2 (no flush)",
                          "learned_start": {"train_instances": sum(len(tb) for tb in train),
                                            "train_samples": int(X.shape[0]),
                                            "fit_steps": FIT_STEPS, "train_s": t_train,
                                            "loss_first": losses[0], "loss_last": losses[-1],
                                            "widths": lcs.widths}},
               "plain": {"value": plain, "unit": "solves/s", "ms_per_step": 1e3 * t_plain / K,
                         "iterations_per_solve_mean": float(np.mean(it_p)),
                         "iterations_first_step_mean": float(np.mean(it_p[0])),
                         "clocks": clk_p.summary()},
               "learned": {"iterations_per_solve_mean": float(np.mean(it_l)),
                           "iterations_first_step_mean": float(np.mean(it_l[0]))},
               "gain_learned_vs_plain": value / plain,
               "other_variant": other,
               "e2e": {"value": job_rate(world, B * K, e2e_s), "unit": "solves/s",
                       "h2d_bytes_per_step": 8 * B * ng,
                       "d2h_bytes_per_step": 8 * B * ng + 8 * B * nu},
               "gpu_launches": launches,
               "roofline": roof,
               "control_error_vs_oracle": ctrl_err,
               "cpu_baseline": cpu,
               "secondary": sec,
               "clocks": clk_l.summary()}
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
