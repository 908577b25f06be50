"""ctypes binding of the plain C FP64 oracle (oracle/nmpc_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may import it.  It computes exactly what
``oracle/nmpc.py`` computes (its tests compare the two element by element)
and exists for host solves of instances too large for the numpy oracle to
finish in reasonable time.  ``build()`` compiles the library in-tree with the
host C compiler (``gcc -O2``, OpenMP over stages when available, no
floating-point contraction); the CUDA path never loads it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nmpc_oracle.c")
LIB = os.path.join(HERE, "_lib", "libnmpc_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle library if its source is newer (or it is missing)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off"]
    tmp = LIB + ".tmp"
    try:
        subprocess.run(base + ["-fopenmp", SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [SRC, "-o", tmp, "-lm"], check=True)  # serial build
    os.replace(tmp, LIB)
    return LIB


class _Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("mx", ctypes.c_int), ("my", ctypes.c_int),
                ("N", ctypes.c_int), ("nu", ctypes.c_int),
                ("act", ctypes.POINTER(ctypes.c_int)),
                ("h", ctypes.c_double), ("q", ctypes.c_double), ("r", ctypes.c_double),
                ("qf", ctypes.c_double), ("gamma", ctypes.c_double), ("k0", ctypes.c_double),
                ("k1", ctypes.c_double), ("b0", ctypes.c_double),
                ("x0", ctypes.POINTER(ctypes.c_double)),
                ("ref", ctypes.POINTER(ctypes.c_double))]


class _Info(ctypes.Structure):
    _fields_ = [("res_inf", ctypes.c_double), ("res_2", ctypes.c_double),
                ("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("diverged", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Problem)
        L.orc_kkt_norms.argtypes = [pp, dp, dp, dp, dp]
        L.orc_jacobi_iteration.argtypes = [pp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, dp, dp, dp, dp]
        L.orc_solve_jacobi.argtypes = [pp, dp, dp, dp, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(_Info)]
        L.orc_plant_step.argtypes = [pp, dp, dp, ctypes.c_double, ctypes.c_int]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        for f in (L.orc_kkt_norms, L.orc_jacobi_iteration, L.orc_solve_jacobi,
                  L.orc_plant_step, L.orc_set_threads):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the stage loops (n <= 0 leaves the default); returns the count."""
    return int(lib().orc_set_threads(int(n)))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Problem:
    """One instance (the attributes oracle/nmpc.py reads) as the C struct."""

    def __init__(self, inst):
        self.dim, self.mx, self.my = int(inst.dim), int(inst.mx), int(inst.my)
        self.N = int(inst.horizon)
        self.act = np.ascontiguousarray(inst.act, dtype=np.int32)
        self.nu = len(self.act)
        self.ng = self.mx * self.my
        self.shape = (self.my, self.mx)
        self.h = float(inst.h)
        self.x0 = np.ascontiguousarray(inst.x0, dtype=np.float64).reshape(-1).copy()
        self.ref = np.ascontiguousarray(inst.ref, dtype=np.float64).reshape(-1).copy()
        self.c = _Problem(self.dim, self.mx, self.my, self.N, self.nu,
                          self.act.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          self.h, float(inst.q), float(inst.r), float(inst.qf),
                          float(inst.gamma), float(inst.k0), float(inst.k1),
                          float(getattr(inst, "act_gain", 32.0)), _dptr(self.x0),
                          _dptr(self.ref))

    def cold_start(self):
        X = np.broadcast_to(self.x0.reshape(self.shape), (self.N,) + self.shape).copy()
        return X, np.zeros((self.N, self.nu)), np.zeros((self.N,) + self.shape)

    def _arrs(self, X, U, L):
        return (np.ascontiguousarray(X, dtype=np.float64).reshape((self.N,) + self.shape).copy(),
                np.ascontiguousarray(U, dtype=np.float64).reshape(self.N, self.nu).copy(),
                np.ascontiguousarray(L, dtype=np.float64).reshape((self.N,) + self.shape).copy())


def kkt_norms(p: Problem, X, U, L):
    X, U, L = p._arrs(X, U, L)
    out = np.zeros(2)
    if lib().orc_kkt_norms(ctypes.byref(p.c), _dptr(X), _dptr(U), _dptr(L), _dptr(out)):
        raise MemoryError("oracle workspace")
    return float(out[0]), float(out[1])


def jacobi_iteration(p: Problem, X, U, L, n_lo=2, n_u_it=2, alpha=1.0):
    """One iteration of eq. 15; returns (X, U, L) of iterate k+1 and the norms of K^k."""
    X, U, L = p._arrs(X, U, L)
    Xo, Uo, Lo = np.empty_like(X), np.empty_like(U), np.empty_like(L)
    out = np.zeros(2)
    if lib().orc_jacobi_iteration(ctypes.byref(p.c), _dptr(X), _dptr(U), _dptr(L), n_lo, n_u_it,
                                  alpha, _dptr(Xo), _dptr(Uo), _dptr(Lo), _dptr(out)):
        raise MemoryError("oracle workspace")
    return Xo, Uo, Lo, (float(out[0]), float(out[1]))


def solve_jacobi(p: Problem, S0=None, tol=1e-6, max_iter=10000, n_lo=2, n_u_it=2, alpha=1.0):
    """Iterate eq. 15 until ||K^k||_inf <= tol; returns ((X, U, L), info) like
    oracle/nmpc.py's solve_jacobi (without the history)."""
    X, U, L = p._arrs(*(p.cold_start() if S0 is None else S0))
    info = _Info()
    if lib().orc_solve_jacobi(ctypes.byref(p.c), _dptr(X), _dptr(U), _dptr(L), tol, max_iter,
                              n_lo, n_u_it, alpha, ctypes.byref(info)):
        raise MemoryError("oracle workspace")
    return (X, U, L), dict(iters=info.iters, res_inf=info.res_inf, res_2=info.res_2,
                           converged=bool(info.converged), diverged=bool(info.diverged))


def plant_step(p: Problem, w, u1, dt, n_sub):
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1).copy()
    u1 = np.ascontiguousarray(u1, dtype=np.float64).reshape(-1).copy()
    lib().orc_plant_step(ctypes.byref(p.c), _dptr(w), _dptr(u1), float(dt), int(n_sub))
    return w


def closed_loop(inst, steps, n_sub, tol=1e-10, max_iter=20000, n_lo=2, n_u_it=2):
    """oracle/nmpc.py's closed_loop: every step a cold-start solve from the
    plant state, u_1 applied for one stage length, the plant advanced."""
    import copy
    cur = copy.copy(inst)
    w = np.asarray(inst.x0, dtype=np.float64).copy()
    U1, W, its = [], [w.copy()], []
    for _ in range(steps):
        cur.x0 = w.copy()
        p = Problem(cur)
        (X, U, L), info = solve_jacobi(p, tol=tol, max_iter=max_iter, n_lo=n_lo, n_u_it=n_u_it)
        U1.append(U[0].copy())
        its.append(info["iters"])
        w = plant_step(p, w, U[0], p.h, n_sub)
        W.append(w.copy())
    return np.array(U1), np.array(W), its
