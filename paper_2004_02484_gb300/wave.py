"""ctypes binding of the second-order-in-time solver (include/nmpc_wave.h).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  Instances are ``workloads.WaveInstance`` objects.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import nmpc as _G  # loads the library (raises if it is missing)

LIB = _G.LIB
nmpc_stats = _G.nmpc_stats
_ptr, _stream, _check = _G._ptr, _G._stream, _G._check

EXPORTED = ["nmpc_wave_default_opts", "nmpc_wave_setup", "nmpc_wave_sizes", "nmpc_wave_solve",
            "nmpc_wave_iterate", "nmpc_wave_get_state", "nmpc_wave_plant_step",
            "nmpc_wave_closed_loop", "nmpc_wave_destroy"]


class nmpc_wave_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("m", ctypes.c_int), ("bc", ctypes.c_int),
                ("horizon", ctypes.c_int), ("n_u", ctypes.c_int),
                ("act_cell", ctypes.POINTER(ctypes.c_int)),
                ("h", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("c", ctypes.c_double), ("kappa", ctypes.c_double), ("gain", ctypes.c_double),
                ("q", ctypes.c_double), ("qv", ctypes.c_double), ("r", ctypes.c_double),
                ("qf", ctypes.c_double), ("gamma", ctypes.c_double)]


class nmpc_wave_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("n_lo", ctypes.c_int),
                ("n_u_it", ctypes.c_int), ("variant", ctypes.c_int),
                ("check_every", ctypes.c_int), ("precision", ctypes.c_int)]


_P, _I = ctypes.c_void_p, ctypes.c_int
_SIG = {
    "nmpc_wave_default_opts": (None, [ctypes.POINTER(nmpc_wave_opts)]),
    "nmpc_wave_setup": (_I, [ctypes.POINTER(nmpc_wave_desc), _I, ctypes.POINTER(nmpc_wave_opts),
                             ctypes.POINTER(_P)]),
    "nmpc_wave_sizes": (_I, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "nmpc_wave_solve": (_I, [_P, _P, _P, _P, _I, _P, ctypes.POINTER(nmpc_stats), _P]),
    "nmpc_wave_iterate": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _P, _P]),
    "nmpc_wave_get_state": (_I, [_P, _P, _P, _P, _P]),
    "nmpc_wave_plant_step": (_I, [_P, _P, ctypes.c_double, _I, _P]),
    "nmpc_wave_closed_loop": (_I, [_P, _P, _P, _P, _I, _I, _P, _P, _P, _P]),
    "nmpc_wave_destroy": (None, [_P]),
}
for _name, (_res, _args) in _SIG.items():
    _fn = getattr(LIB, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def default_opts(**kw) -> nmpc_wave_opts:
    o = nmpc_wave_opts()
    LIB.nmpc_wave_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def make_descs(instances: Sequence):
    descs = (nmpc_wave_desc * len(instances))()
    keep = []
    for d, inst in zip(descs, instances):
        act = (ctypes.c_int * len(inst.act))(*[int(a) for a in inst.act])
        keep.append(act)
        d.dim, d.m, d.bc = int(inst.dim), int(inst.m), 0 if inst.bc == "neumann" else 1
        d.horizon, d.n_u, d.act_cell = int(inst.horizon), len(inst.act), act
        d.h, d.a, d.b, d.c = float(inst.h), float(inst.a), float(inst.b), float(inst.c)
        d.kappa, d.gain = float(inst.kappa), float(inst.gain)
        d.q, d.qv, d.r, d.qf = float(inst.q), float(inst.qv), float(inst.r), float(inst.qf)
        d.gamma = float(inst.gamma)
    return descs, keep


def pack(instances: Sequence, name: str) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([np.asarray(getattr(i, name), dtype=np.float64)
                                                for i in instances]))


class WaveSolver:
    """One handle over nmpc_wave_*; x0, w_ref, u_ref from the instances."""

    def __init__(self, instances: Sequence, **opts):
        import torch
        self.instances = list(instances)
        self.n = len(self.instances)
        descs, keep = make_descs(self.instances)
        o = default_opts(**opts)
        h = ctypes.c_void_p()
        _check(LIB.nmpc_wave_setup(descs, self.n, ctypes.byref(o), ctypes.byref(h)),
               "nmpc_wave_setup")
        del keep
        self.h = h
        sz = (ctypes.c_int64 * 5)()
        _check(LIB.nmpc_wave_sizes(h, sz), "nmpc_wave_sizes")
        self.n_g, self.n_x, self.n_u, self.n_a, self.n_w = (int(v) for v in sz)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.x0 = torch.from_numpy(pack(self.instances, "x0")).to(dev)
        self.w_ref = torch.from_numpy(pack(self.instances, "w_ref")).to(dev)
        self.u_ref = torch.from_numpy(pack(self.instances, "u_ref")).to(dev)
        self.u = torch.zeros(self.n_u, dtype=torch.float64, device=dev)

    def solve(self, init: int = _G.NMPC_INIT_COLD, x0=None, stream=None):
        stats = (nmpc_stats * self.n)()
        rc = LIB.nmpc_wave_solve(self.h, _ptr(self.x0 if x0 is None else x0), _ptr(self.w_ref),
                                 _ptr(self.u_ref), init, _ptr(self.u), stats, _stream(stream))
        _check(rc, "nmpc_wave_solve", allow=(_G.NMPC_ERR_NOT_CONVERGED, _G.NMPC_ERR_DIVERGED))
        return rc, stats

    def iterate(self, x, u, lam, n_iter: int, stream=None):
        import torch
        xo, uo, lo = torch.empty_like(x), torch.empty_like(u), torch.empty_like(lam)
        out = np.zeros((self.n, 3))
        _check(LIB.nmpc_wave_iterate(self.h, _ptr(self.x0), _ptr(self.w_ref), _ptr(self.u_ref),
                                     _ptr(x), _ptr(u), _ptr(lam), _ptr(xo), _ptr(uo), _ptr(lo),
                                     n_iter, out.ctypes.data, _stream(stream)),
               "nmpc_wave_iterate")
        return (xo, uo, lo), out

    def state(self):
        import torch
        x = torch.empty(self.n_x, dtype=torch.float64, device=self.u.device)
        lam = torch.empty_like(x)
        u = torch.empty(self.n_u, dtype=torch.float64, device=self.u.device)
        _check(LIB.nmpc_wave_get_state(self.h, _ptr(x), _ptr(u), _ptr(lam), _stream(None)),
               "nmpc_wave_get_state")
        return x, u, lam

    def plant_step(self, x, dt: float, n_sub: int, stream=None):
        _check(LIB.nmpc_wave_plant_step(self.h, _ptr(x), float(dt), int(n_sub), _stream(stream)),
               "nmpc_wave_plant_step")

    def closed_loop(self, x, steps: int, n_sub: int, u_hist=None, stream=None):
        iters = np.zeros((steps, self.n), dtype=np.int32)
        res = np.zeros((steps, self.n), dtype=np.float64)
        rc = LIB.nmpc_wave_closed_loop(self.h, _ptr(x), _ptr(self.w_ref), _ptr(self.u_ref), steps,
                                       n_sub, _ptr(u_hist), iters.ctypes.data, res.ctypes.data,
                                       _stream(stream))
        _check(rc, "nmpc_wave_closed_loop", allow=(_G.NMPC_ERR_NOT_CONVERGED, _G.NMPC_ERR_DIVERGED))
        return rc, iters, res

    def close(self):
        if self.h:
            LIB.nmpc_wave_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
