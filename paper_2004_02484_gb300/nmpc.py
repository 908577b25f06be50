"""Thin Python binding of the C ABI in ``include/nmpc.h`` (ctypes).

Argument marshalling only: every step of the solve runs in the CUDA library.
Functions keep the C names (``nmpc_setup``, ``nmpc_solve``, ...); device
arrays are torch CUDA float64 tensors passed by ``data_ptr()``, streams are
``torch.cuda.Stream`` objects (default: the current stream).  Importing this
module loads the library and raises if it is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

NMPC_OK = 0
NMPC_ERR_BAD_ARG = -1
NMPC_ERR_CUDA = -2
NMPC_ERR_NOT_CONVERGED = -3
NMPC_ERR_DIVERGED = -4
NMPC_ERR_NO_DEVICE = -5
NMPC_ERR_UNSUPPORTED = -6
NMPC_FP64 = 0
NMPC_MIXED = 1
NMPC_VARIANT_JACOBI = 0
NMPC_VARIANT_REDBLACK = 1
NMPC_INIT_COLD = 0
NMPC_INIT_WARM = 1
NMPC_INIT_GUESS = 2
NMPC_INIT_SHIFT = 3
NMPC_STATUS_CONVERGED = 1
NMPC_STATUS_DIVERGED = 2
NMPC_STATUS_MAX_ITER = 3


class nmpc_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("mx", ctypes.c_int), ("my", ctypes.c_int),
                ("horizon", ctypes.c_int), ("n_u", ctypes.c_int),
                ("act_cell", ctypes.POINTER(ctypes.c_int)),
                ("h", ctypes.c_double), ("q", ctypes.c_double), ("r", ctypes.c_double),
                ("qf", ctypes.c_double), ("gamma", ctypes.c_double), ("k0", ctypes.c_double),
                ("k1", ctypes.c_double), ("act_gain", ctypes.c_double)]


class nmpc_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("n_lo", ctypes.c_int),
                ("n_u_it", ctypes.c_int), ("precision", ctypes.c_int),
                ("check_every", ctypes.c_int), ("alpha", ctypes.c_double),
                ("div_limit", ctypes.c_double), ("threads", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("cluster", ctypes.c_int),
                ("split_min", ctypes.c_double), ("u_local", ctypes.c_int),
                ("cells", ctypes.c_int), ("persistent", ctypes.c_int),
                ("strips", ctypes.c_int), ("strip_rows", ctypes.c_int),
                ("lines", ctypes.c_int), ("variant", ctypes.c_int),
                ("barrier_wait_cycles", ctypes.c_int64), ("strip_cols", ctypes.c_int),
                ("tail_rows", ctypes.c_int), ("tail_below", ctypes.c_int)]


class nmpc_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int),
                ("res_inf", ctypes.c_double), ("res_2", ctypes.c_double),
                ("f64_iters", ctypes.c_int)]


EXPORTED = ["nmpc_default_opts", "nmpc_setup", "nmpc_solve", "nmpc_solve_host",
            "nmpc_residual", "nmpc_iterate", "nmpc_get_state", "nmpc_set_state",
            "nmpc_sizes", "nmpc_launch_count", "nmpc_launch_plan", "nmpc_strip_plan", "nmpc_line_plan", "nmpc_start_state", "nmpc_rollout", "nmpc_rollout_fused", "nmpc_destroy",
            "nmpc_strerror",
            "nmpc_solve_noalloc", "nmpc_plant_step", "nmpc_closed_loop",
            "nmpc_closed_loop_learned", "nmpc_kernel_timing", "nmpc_kernel_times"]


# step start of nmpc_closed_loop_learned: void (*)(void* ctx, void* stream)
START_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def _load() -> ctypes.CDLL:
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing; run "
                          "paper_2004_02484_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P, D, I, V = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, None
    sig = {
        "nmpc_default_opts": (V, [ctypes.POINTER(nmpc_opts)]),
        "nmpc_setup": (I, [ctypes.POINTER(nmpc_desc), I, ctypes.POINTER(nmpc_opts),
                           ctypes.POINTER(P)]),
        "nmpc_solve": (I, [P, P, P, I, P, I, P, ctypes.POINTER(nmpc_stats), P]),
        "nmpc_solve_host": (I, [P, P, P, I, P, I, P, ctypes.POINTER(nmpc_stats), P]),
        "nmpc_residual": (I, [P, P, P, P, P, P, P, P]),
        "nmpc_iterate": (I, [P, P, P, P, P, P, P, P, P, I, P, P]),
        "nmpc_get_state": (I, [P, P, P, P, P]),
        "nmpc_set_state": (I, [P, P, P, P, P]),
        "nmpc_sizes": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
        "nmpc_launch_plan": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
        "nmpc_strip_plan": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
        "nmpc_line_plan": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
        "nmpc_start_state": (I, [P, I, P, P, P, P, P]),
        "nmpc_rollout": (I, [P, P, P, P, P, P, P]),
        "nmpc_rollout_fused": (I, [P, P, P, P, P, P, P]),
        "nmpc_launch_count": (ctypes.c_int64, [P]),
        "nmpc_destroy": (V, [P]),
        "nmpc_strerror": (ctypes.c_char_p, [I]),
        "nmpc_solve_noalloc": (I, [ctypes.POINTER(nmpc_desc), ctypes.POINTER(nmpc_opts), P, P,
                                   P, ctypes.POINTER(nmpc_stats), P]),
        "nmpc_plant_step": (I, [P, P, D, I, P, P]),
        "nmpc_closed_loop": (I, [P, P, P, I, I, P, P, P, P]),
        "nmpc_closed_loop_learned": (I, [P, P, P, I, I, START_FN, P, P, P, P, P, P]),
        "nmpc_kernel_timing": (I, [P, I]),
        "nmpc_kernel_times": (I, [P, ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


class NmpcError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {LIB.nmpc_strerror(code).decode()} ({code})")
        self.code = code


def _check(code: int, where: str, allow=()):
    if code != NMPC_OK and code not in allow:
        raise NmpcError(code, where)
    return code


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float64 tensor")
    return t.data_ptr()


def _stream(stream):
    """A torch stream, a raw cudaStream_t (int) or None (torch's current stream)."""
    import torch
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def nmpc_default_opts() -> nmpc_opts:
    o = nmpc_opts()
    LIB.nmpc_default_opts(ctypes.byref(o))
    return o


def make_descs(instances: Sequence) -> tuple:
    """nmpc_desc array for workload instances (keeps the actuator arrays alive)."""
    arr = (nmpc_desc * len(instances))()
    keep = []
    for d, inst in zip(arr, instances):
        act = np.ascontiguousarray(np.asarray(inst.act, dtype=np.int32))
        keep.append(act)
        d.dim, d.mx, d.my, d.horizon, d.n_u = inst.dim, inst.mx, inst.my, inst.horizon, len(act)
        d.act_cell = act.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        d.h, d.q, d.r, d.qf = inst.h, inst.q, inst.r, inst.qf
        d.gamma, d.k0, d.k1 = inst.gamma, inst.k0, inst.k1
        d.act_gain = getattr(inst, "act_gain", 32.0)
    return arr, keep


def nmpc_setup(instances: Sequence, **opts) -> ctypes.c_void_p:
    o = nmpc_default_opts()
    for k, v in opts.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    descs, keep = make_descs(instances)
    h = ctypes.c_void_p()
    _check(LIB.nmpc_setup(descs, len(instances), ctypes.byref(o), ctypes.byref(h)), "nmpc_setup")
    del keep
    return h


def nmpc_strip_plan(h) -> dict:
    """The handle's strip path (strips per iteration, strip shape, threads, shared
    memory, actuator patches per iteration, instances on the path, region
    cells, the tail plan's rows and the running count that selects it)."""
    out = (ctypes.c_int64 * 10)()
    _check(LIB.nmpc_strip_plan(h, out), "nmpc_strip_plan")
    keys = ("strips", "strip_x", "strip_y", "threads", "smem", "patches", "instances", "region",
            "tail_rows", "tail_below")
    return {k: int(v) for k, v in zip(keys, out)}


def nmpc_line_plan(h) -> dict:
    """The line path of a handle: line work items per iteration (one warp
    each), instances on it, threads and dynamic shared memory per CTA."""
    out = (ctypes.c_int64 * 4)()
    _check(LIB.nmpc_line_plan(h, out), "nmpc_line_plan")
    return {k: int(v) for k, v in zip(("lines", "instances", "threads", "smem"), out)}


KERNEL_KINDS = ("k_iterate", "k_patch", "k_strip", "k_line")


def nmpc_kernel_timing(h, enable: bool = True) -> None:
    """Start (or stop) CUDA-event timing of the iteration kernels' launches
    outside graphs; clears the totals."""
    _check(LIB.nmpc_kernel_timing(h, 1 if enable else 0), "nmpc_kernel_timing")


def nmpc_kernel_times(h) -> dict:
    """{kernel: (timed launches, summed device ms)} since the last
    nmpc_kernel_timing call (waits for the recorded events)."""
    n = (ctypes.c_int64 * 4)()
    ms = (ctypes.c_double * 4)()
    _check(LIB.nmpc_kernel_times(h, n, ms), "nmpc_kernel_times")
    return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(KERNEL_KINDS)}


def nmpc_launch_plan(h) -> dict:
    """The launch plan of a handle (threads, cluster, cells, staged, persistent,
    smem, grid, local_u, resident_clusters, work_items, iteration_launches)."""
    out = (ctypes.c_int64 * 11)()
    _check(LIB.nmpc_launch_plan(h, out), "nmpc_launch_plan")
    keys = ("threads", "cluster", "cells", "staged", "persistent", "smem", "grid", "local_u",
            "resident_clusters", "work_items", "iteration_launches")
    return {k: int(v) for k, v in zip(keys, out)}


def nmpc_sizes(h) -> tuple:
    out = (ctypes.c_int64 * 3)()
    _check(LIB.nmpc_sizes(h, out), "nmpc_sizes")
    return int(out[0]), int(out[1]), int(out[2])


def nmpc_solve(h, x0, ref, u_out, n_inst: int, horizon: int = 0, weights=None,
               init: int = NMPC_INIT_COLD, stream=None) -> tuple:
    stats = (nmpc_stats * n_inst)()
    rc = LIB.nmpc_solve(h, _ptr(x0), _ptr(ref), horizon, _ptr(weights), init, _ptr(u_out),
                        stats, _stream(stream))
    _check(rc, "nmpc_solve", allow=(NMPC_ERR_NOT_CONVERGED, NMPC_ERR_DIVERGED))
    return rc, stats


def nmpc_solve_host(h, x0: np.ndarray, ref: np.ndarray, u_out: np.ndarray, n_inst: int,
                    horizon: int = 0, weights: Optional[np.ndarray] = None,
                    init: int = NMPC_INIT_COLD, stream=None) -> tuple:
    for a in (x0, ref, u_out) + ((weights,) if weights is not None else ()):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected C-contiguous float64 arrays")
    stats = (nmpc_stats * n_inst)()
    rc = LIB.nmpc_solve_host(h, x0.ctypes.data, ref.ctypes.data, horizon,
                             None if weights is None else weights.ctypes.data, init,
                             u_out.ctypes.data, stats, _stream(stream))
    _check(rc, "nmpc_solve_host", allow=(NMPC_ERR_NOT_CONVERGED, NMPC_ERR_DIVERGED))
    return rc, stats


def nmpc_residual(h, x0, ref, x, u, lam, n_inst: int, stream=None) -> np.ndarray:
    out = np.zeros((n_inst, 2))
    _check(LIB.nmpc_residual(h, _ptr(x0), _ptr(ref), _ptr(x), _ptr(u), _ptr(lam),
                             out.ctypes.data, _stream(stream)), "nmpc_residual")
    return out


def nmpc_iterate(h, x0, ref, x_in, u_in, lam_in, x_out, u_out, lam_out, n_iter: int,
                 n_inst: int, stream=None) -> np.ndarray:
    out = np.zeros((n_inst, 2))
    _check(LIB.nmpc_iterate(h, _ptr(x0), _ptr(ref), _ptr(x_in), _ptr(u_in), _ptr(lam_in),
                            _ptr(x_out), _ptr(u_out), _ptr(lam_out), n_iter, out.ctypes.data,
                            _stream(stream)), "nmpc_iterate")
    return out


def nmpc_get_state(h, x, u, lam, stream=None):
    _check(LIB.nmpc_get_state(h, _ptr(x), _ptr(u), _ptr(lam), _stream(stream)), "nmpc_get_state")


def nmpc_set_state(h, x, u, lam, stream=None):
    _check(LIB.nmpc_set_state(h, _ptr(x), _ptr(u), _ptr(lam), _stream(stream)), "nmpc_set_state")


def nmpc_plant_step(h, w, dt: float, n_sub: int, u_rec=None, stream=None):
    _check(LIB.nmpc_plant_step(h, _ptr(w), dt, n_sub, _ptr(u_rec), _stream(stream)),
           "nmpc_plant_step")


def nmpc_closed_loop(h, w, ref, steps: int, n_sub: int, n_inst: int, u_hist=None,
                     stream=None):
    """Returns (rc, iters [steps, n], res [steps, n])."""
    iters = np.zeros((steps, n_inst), dtype=np.int32)
    res = np.zeros((steps, n_inst), dtype=np.float64)
    rc = LIB.nmpc_closed_loop(h, _ptr(w), _ptr(ref), steps, n_sub, _ptr(u_hist),
                              iters.ctypes.data, res.ctypes.data, _stream(stream))
    _check(rc, "nmpc_closed_loop", allow=(NMPC_ERR_NOT_CONVERGED, NMPC_ERR_DIVERGED))
    return rc, iters, res


def nmpc_closed_loop_learned(h, w, ref, steps: int, n_sub: int, n_inst: int, start, u_guess,
                             u_hist=None, stream=None):
    """Closed loop with a learned start.  start(stream_ptr: int) enqueues, on
    the given raw stream, kernels that write the control guess into u_guess
    from the plant state w (kernel launches only: they are captured into the
    loop's graph).  Returns (rc, iters [steps, n], res [steps, n])."""
    iters = np.zeros((steps, n_inst), dtype=np.int32)
    res = np.zeros((steps, n_inst), dtype=np.float64)
    errors = []

    def _cb(ctx, st):
        try:
            start(int(st or 0))
        except BaseException as e:  # reported after the call: the C side cannot see it
            errors.append(e)

    cb = START_FN(_cb)
    rc = LIB.nmpc_closed_loop_learned(h, _ptr(w), _ptr(ref), steps, n_sub, cb, None, _ptr(u_guess),
                                      _ptr(u_hist), iters.ctypes.data, res.ctypes.data,
                                      _stream(stream))
    if errors:
        raise errors[0]
    _check(rc, "nmpc_closed_loop_learned", allow=(NMPC_ERR_NOT_CONVERGED, NMPC_ERR_DIVERGED))
    return rc, iters, res


def nmpc_start_state(h, init: int, x0, x, u, lam, stream=None):
    """Start iterate of `init` (NMPC_INIT_COLD from x0, or NMPC_INIT_SHIFT of the
    current state) into device float64 arrays x, u, lam."""
    _check(LIB.nmpc_start_state(h, init, _ptr(x0), _ptr(x), _ptr(u), _ptr(lam), _stream(stream)),
           "nmpc_start_state")


def nmpc_rollout(h, x0, ref, u, x, lam, stream=None):
    """State (forward) and costate (backward) trajectories of the controls u."""
    _check(LIB.nmpc_rollout(h, _ptr(x0), _ptr(ref), _ptr(u), _ptr(x), _ptr(lam), _stream(stream)),
           "nmpc_rollout")


def nmpc_rollout_fused(h, x0, ref, u, x, lam, stream=None):
    """nmpc_rollout in one launch, float32 arithmetic (a start guess)."""
    _check(LIB.nmpc_rollout_fused(h, _ptr(x0), _ptr(ref), _ptr(u), _ptr(x), _ptr(lam),
                                  _stream(stream)), "nmpc_rollout_fused")


def nmpc_launch_count(h) -> int:
    return int(LIB.nmpc_launch_count(h))


def nmpc_destroy(h):
    LIB.nmpc_destroy(h)


def nmpc_solve_noalloc(inst, x0, ref, u_out, stream=None, **opts) -> tuple:
    """Allocation-free single-instance solve (static device workspace)."""
    o = nmpc_default_opts()
    for k, v in opts.items():
        setattr(o, k, v)
    descs, keep = make_descs([inst])
    st = nmpc_stats()
    rc = LIB.nmpc_solve_noalloc(descs, ctypes.byref(o), _ptr(x0), _ptr(ref), _ptr(u_out),
                                ctypes.byref(st), _stream(stream))
    del keep
    _check(rc, "nmpc_solve_noalloc", allow=(NMPC_ERR_NOT_CONVERGED, NMPC_ERR_DIVERGED))
    return rc, st


# ---------------------------------------------------------------------------
# Packing of per-instance arrays into the packed layout of the header
# ---------------------------------------------------------------------------
def pack_fields(instances: Sequence, name: str) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([np.asarray(getattr(i, name), dtype=np.float64)
                                                for i in instances]))


def split_stages(instances: Sequence, flat: np.ndarray, per: str) -> List[np.ndarray]:
    """Split a packed x/lam ('ng') or u ('nu') array into per-instance (N, ...) arrays."""
    out, o = [], 0
    for inst in instances:
        n = inst.mx * inst.my if per == "ng" else len(inst.act)
        m = inst.horizon * n
        out.append(flat[o:o + m].reshape(inst.horizon, n))
        o += m
    return out


class Solver:
    """Owns one handle; convenience wrapper over the functions above."""

    def __init__(self, instances: Sequence, **opts):
        import torch
        self.instances = list(instances)
        self.n = len(self.instances)
        self.h = nmpc_setup(self.instances, **opts)
        self.n_g, self.n_s, self.n_u = nmpc_sizes(self.h)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.x0 = torch.from_numpy(pack_fields(self.instances, "x0")).to(dev)
        self.ref = torch.from_numpy(pack_fields(self.instances, "ref")).to(dev)
        self.u = torch.zeros(self.n_u, dtype=torch.float64, device=dev)

    def solve(self, init: int = NMPC_INIT_COLD, weights=None, stream=None):
        rc, stats = nmpc_solve(self.h, self.x0, self.ref, self.u, self.n, 0, weights, init, stream)
        return rc, stats

    def state(self):
        import torch
        x = torch.empty(self.n_s, dtype=torch.float64, device=self.u.device)
        l = torch.empty_like(x)
        u = torch.empty(self.n_u, dtype=torch.float64, device=self.u.device)
        nmpc_get_state(self.h, x, u, l)
        return x, u, l

    def close(self):
        if self.h:
            nmpc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
