"""Benchmark: solves/s of the double-layer Jacobi NMPC method on one GB300.

A step is one complete solve, from the cold start S^0, of the 2D nonlinear
heat workload (64x64 grid, N = 50 stages, 8 actuators, dt = 2e-5) to
||K||_inf <= 1e-6, with a fresh seeded initial field every step, on the
MIXED path (float32 lower layer, float64 KKT residual / norms / update).
Inputs are resident in HBM when a step starts; the L2 cache is flushed
(256 MiB write) between steps, outside the per-step CUDA events.

Under torchrun (N > 1) every rank solves its own replicas (the instances are
independent; there is no data-path collective): value = solves of all ranks
/ max-over-ranks time.

``--impl reference`` times the FP64 CPU oracle on the host cores for the same
workload and metric (bounded sample: a fixed number of oracle iterations per
step, converted to solves/s with the oracle's own iteration count).
"""
import argparse
import json
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
WORKLOAD = ("heat2d_64x64_N50: 2D nonlinear heat eq. k(w)=0.1(1+0.5w), 64x64 grid, dt=2e-5, "
            "N=50, 8 actuators (2x4), Gaussian-bump reference, 16-mode sine initial field; "
            "plain double-layer Jacobi, cold start, tol ||K||_inf<=1e-6")
TOL = 1e-6
# algorithmic bytes per cell-stage per iteration: read x_i, lambda_i and write
# them back in float64 (the neighbour-stage reads are the same arrays)
BYTES_PER_POINT_STAGE = 32

def fp32_flops_per_point_stage(n_lo: int, n_u_it: int) -> int:
    """Algorithmic float32 flops per cell-stage per iteration of the mixed
    path: split residual ~30 and coefficients ~10, then n_u_it + 1
    applications of P^-1 (eq. 24), each 2 n_lo sweeps of ~10 flops plus ~2."""
    return 30 + 10 + (n_u_it + 1) * (2 * n_lo * 10 + 2)

# float32 FMA peak: 128 lanes x 2 flops x 152 SMs x 2.07 GHz (unit counts and
# maximum SM clock of the part)
FP32_PEAK_TFLOPS = 128 * 2 * 152 * 2.07e9 / 1e12
# dram__bytes_read.sum + dram__bytes_write.sum of one iteration launch of this
# workload from the committed ncu capture of the iteration kernel (cold
# caches); None once the kernel changes after that capture
TRAFFIC_BYTES_PER_LAUNCH = 3.48e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--ref-iters", type=int, default=300,
                    help="oracle iterations timed on the host in all: the cpu_baseline sample, "
                         "and the reference arm's (spread over its steps, at least one per "
                         "step); ~30 ms each on the GPU box's Grace cores")
    ap.add_argument("--graph", type=int, default=1,
                    help="1: the solve loop is one CUDA graph; 0: chunks of iteration launches "
                         "from the host (the same kernels; a profiler can capture them)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def step_seed(step: int, rank: int) -> int:
    """Seed of the initial field of a rank's step: step 0 of rank 0 is the
    canonical seed-1 field, every other (rank, step) a fresh field of its own
    (ranks solve disjoint instances: replicas, no data-path collective)."""
    return 1 if (step == 0 and rank == 0) else 100_000 + 1000 * rank + step


def step_instance(step: int, rank: int):
    from paper_2004_02484_gb300 import workloads as wl
    return wl.heat2d_single(seed=step_seed(step, rank))


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


def job_rate(world: int, steps: int, seconds: float) -> float:
    """Whole-job solves/s: every rank's steps over the slowest rank's time."""
    return world * steps / seconds


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


def run_oracle_sample(iters: int):
    """Bounded oracle sample on the host: `iters` upper-layer iterations of the
    workload, and the oracle's own iteration count to the tolerance."""
    from oracle import nmpc as O
    inst = step_instance(0, 0)
    p = O.Problem(inst)
    X, U, L = p.cold_start()
    t0 = time.perf_counter()
    for _ in range(iters):
        X, U, L, _ = O.jacobi_iteration(p, X, U, L)
    return time.perf_counter() - t0


def oracle_iters_to_tol():
    from oracle import nmpc as O
    p = O.Problem(step_instance(0, 0))
    _, info = O.solve_jacobi(p, tol=TOL)
    return info["iters"]


def ref_iters_per_step(total: int, steps: int) -> int:
    """Oracle iterations per reference step: about `total` over the run (a
    bounded sample whatever the step count), at least one per step."""
    return max(1, round(total / max(1, steps)))


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    n_it = oracle_iters_to_tol()  # part of warm-up: the oracle's own iteration count
    for _ in range(args.warmup):
        run_oracle_sample(1)
    per_step = ref_iters_per_step(args.ref_iters, args.steps)
    t = 0.0
    for _ in range(args.steps):
        t += run_oracle_sample(per_step)
    sec_per_iter = t / (args.steps * per_step)
    value = 1.0 / (sec_per_iter * n_it)
    cb = {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
          "sample": f"{per_step} FP64 numpy oracle iterations per step x {args.steps} steps; "
                    f"solves/s = 1 / (s per iteration x {n_it} oracle iterations to 1e-6)"}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * sec_per_iter * n_it, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": WORKLOAD, "tol": TOL},
                      "cpu_baseline": cb,
                      "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


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

    prec = G.NMPC_MIXED if args.precision == "mixed" else G.NMPC_FP64
    insts = [step_instance(s, rank) for s in range(args.warmup + args.steps)]
    # launch shape and inner-iteration counts chosen by the autotuner (timed
    # solves of this workload, outside the timed region)
    from paper_2004_02484_gb300 import autotune as AT
    tuned = AT.tune([insts[0]], prec, tol=TOL, cache_path=AT.DEFAULT_CACHE + f".rank{rank}")
    solver = G.Solver([insts[0]], tol=TOL, precision=prec, max_iter=5000, use_graph=args.graph,
                      **AT.solver_opts(tuned))
    dev = solver.u.device
    x0s = [torch.from_numpy(G.pack_fields([i], "x0")).to(dev) for i in insts]
    refs = [torch.from_numpy(G.pack_fields([i], "ref")).to(dev) for i in insts]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def one(step):
        return G.nmpc_solve(solver.h, x0s[step], refs[step], solver.u, 1, stream=stream)

    for s in range(args.warmup):
        rc, st = one(s)
        assert rc == G.NMPC_OK, rc
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    iters, launches0 = [], G.nmpc_launch_count(solver.h)
    it_launches0 = G.nmpc_launch_plan(solver.h)["iteration_launches"]
    torch.cuda.synchronize()
    with ClockSampler(smi_selector(local)) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            rc, st = one(args.warmup + k)
            ev[k][1].record(stream)
            assert rc == G.NMPC_OK and st[0].res_inf <= TOL, (rc, st[0].res_inf)
            iters.append(st[0].iters)
        torch.cuda.synchronize()
    launches = G.nmpc_launch_count(solver.h) - launches0
    it_launches = G.nmpc_launch_plan(solver.h)["iteration_launches"] - it_launches0
    t_ms = max_over_ranks(sum(a.elapsed_time(b_) for a, b_ in ev), dev)
    if world > 1:
        torch.distributed.barrier()
    value = job_rate(world, args.steps, t_ms / 1e3)

    # end to end through the host-pointer entry point (pinned host buffers)
    x0h = [torch.from_numpy(G.pack_fields([i], "x0")).pin_memory().numpy() for i in insts]
    refh = [torch.from_numpy(G.pack_fields([i], "ref")).pin_memory().numpy() for i in insts]
    uh = torch.zeros(solver.n_u, dtype=torch.float64).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        rc, st = G.nmpc_solve_host(solver.h, x0h[args.warmup + k], refh[args.warmup + k], uh, 1)
        assert rc == G.NMPC_OK
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)

    # roofline of the dominant kernel (the fused iteration kernel, one launch
    # per iteration): the timed region divided by its launches (the region
    # also holds the launch gaps, the host polls between chunks of launches
    # and the small control kernels, so this over-estimates the kernel's
    # duration)
    ins = insts[0]
    cells = ins.horizon * ins.mx * ins.my
    avg_launch_ms = t_ms / max(1, it_launches)
    peaks, which = measured_peaks()
    achieved = BYTES_PER_POINT_STAGE * cells / (avg_launch_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": TRAFFIC_BYTES_PER_LAUNCH,
            "peak_source": which,
            "kernel": "k_iterate<float,SOLVE> (fused residual + lower layer + update)",
            "algorithmic_bytes_per_launch": BYTES_PER_POINT_STAGE * cells,
            "avg_launch_ms": avg_launch_ms, "iteration_launches": it_launches,
            "plan": {k: v for k, v in G.nmpc_launch_plan(solver.h).items()
                     if k in ("threads", "cluster", "cells", "staged", "persistent")}}
    # the same launches against the float32 ALU ceiling (the 64x64 stage slabs
    # live in shared memory; the kernel is latency-bound)
    flops_cs = fp32_flops_per_point_stage(tuned.get("n_lo", 2), tuned.get("n_u_it", 2))
    ach_alu = flops_cs * cells / (avg_launch_ms / 1e3) / 1e12
    roof_alu = {"bound": "alu", "achieved": ach_alu, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach_alu / FP32_PEAK_TFLOPS, "peak_source": "derived (unit counts x clock)",
                "flops_per_cell_stage": flops_cs}
    cpu = None
    if rank == 0:
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        n_it = oracle_iters_to_tol()
        t_or = run_oracle_sample(args.ref_iters)
        sec_per_iter = t_or / args.ref_iters
        cpu = {"value": 1.0 / (sec_per_iter * n_it), "unit": "solves/s", "cores": 1,
               "kind": "oracle",
               "sample": f"{args.ref_iters} FP64 numpy oracle iterations of the seed-1 field; "
                         f"solves/s = 1 / (s per iteration x {n_it} oracle iterations to 1e-6)"}
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f32+f64" if prec == G.NMPC_MIXED else "f64", "data": "synthetic",
               "config": {"workload": WORKLOAD, "precision": args.precision, "tol": TOL,
                          "instances_per_rank": 1, "tuned": AT.solver_opts(tuned),
                          "solve_loop": "one CUDA graph" if args.graph else "host-launched chunks",
                          "l2": "flushed between steps (256 MiB write) outside the per-step events",
                          "iterations_per_solve": {"min": min(iters), "max": max(iters),
                                                   "mean": sum(iters) / len(iters)}},
               "e2e": {"value": job_rate(world, args.steps, e2e_s), "unit": "solves/s",
                       "h2d_bytes_per_step": 2 * 8 * ins.mx * ins.my,
                       "d2h_bytes_per_step": 8 * ins.horizon * len(ins.act)},
               "gpu_launches": launches,
               "roofline": roof,
               "roofline_alu": roof_alu,
               "cpu_baseline": cpu,
               "clocks": clk.summary()}
        print(json.dumps(out), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
