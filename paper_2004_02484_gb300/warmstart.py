"""Learned warm start for the double-layer Jacobi solve.

The method needs only a starting iterate close enough to the root (Theorem 1:
the root is a point of attraction); the cold start x_i = x0, u = 0,
lambda = 0 leaves the controls and costates to be found by the iteration,
which propagates information one stage per iteration (Lemma 4: the
stage-coupling part is nilpotent).  A network that maps the current field
and the reference to a trajectory guess shortens that transient.

Pipeline (every arithmetic step in the library's CUDA kernels):
* targets: batched solves of seeded instances (``workloads.
  heat2d_learning_instance``) with the solver itself, to ||K|| <= tol;
* spatial POD bases (rank r) of the state deviation x_i - x0 and of the
  costate lambda_i, by the method of snapshots: Gram matrix S S^T on the
  tensor cores (BF16 operands, FP32 accumulation), its eigenvectors on the
  host in float64, basis V = S^T U_r diag(1/sqrt(sigma_r)) by a GEMM;
* network: [x0; ref] (2 ng) -> 512 -> 512 -> 512 (GELU) -> [u trajectory;
  POD coefficients of x - x0; POD coefficients of lambda], trained on
  standardised targets with Adam (the standardisation is folded into the last
  layer afterwards);
* inference: forward pass, GEMM decode x_i = x0 + V_x c_i, lambda_i =
  V_l d_i, cast to float64, ``nmpc_set_state`` and a warm-started solve.
"""
from __future__ import annotations

import time
from typing import Dict, List, Sequence

import numpy as np

from . import mlp as GM
from . import nmpc as G
from . import workloads as wl


def _torch():
    import torch
    return torch


def generate(seeds: Sequence[int], batch: int = 128, tol: float = 1e-7,
             precision: int = G.NMPC_MIXED) -> Dict[str, np.ndarray]:
    """Solve the learning instances for `seeds`; returns float32 arrays
    x0, ref [n, ng]; u [n, N*nu]; dx = x - x0 and lam [n, N, ng]."""
    torch = _torch()
    out = {k: [] for k in ("x0", "ref", "u", "dx", "lam", "iters")}
    for b0 in range(0, len(seeds), batch):
        insts = [wl.heat2d_learning_instance(s) for s in seeds[b0:b0 + batch]]
        s = G.Solver(insts, tol=tol, precision=precision, max_iter=6000)
        rc, st = s.solve()
        if rc != G.NMPC_OK:
            raise RuntimeError(f"training solve failed: {rc}")
        x, u, lam = s.state()
        ng, N, nu = insts[0].ng, insts[0].horizon, len(insts[0].act)
        n = len(insts)
        x = x.view(n, N, ng)
        x0 = s.x0.view(n, 1, ng)
        out["x0"].append(s.x0.view(n, ng).float().cpu().numpy())
        out["ref"].append(s.ref.view(n, ng).float().cpu().numpy())
        out["u"].append(u.view(n, N * nu).float().cpu().numpy())
        out["dx"].append((x - x0).float().cpu().numpy())
        out["lam"].append(lam.view(n, N, ng).float().cpu().numpy())
        out["iters"].append(np.array([st[b].iters for b in range(n)]))
        s.close()
    return {k: np.concatenate(v) for k, v in out.items()}


def pod_basis(snap: np.ndarray, rank: int) -> np.ndarray:
    """Rank-r POD basis [ng, r] of snapshot rows snap [n_snap, ng] (method of
    snapshots: Gram on the tensor cores, float64 eigensolve on the host)."""
    torch = _torch()
    S = torch.from_numpy(np.ascontiguousarray(snap, dtype=np.float32)).cuda()
    ns, ng = S.shape
    scale = float(np.abs(snap).max()) or 1.0
    Sb = torch.empty((ns, ng), dtype=torch.bfloat16, device="cuda")
    GM.nmpc_cast_f32_bf16((S / scale).contiguous(), Sb)
    Gm = torch.zeros((ns, ns), dtype=torch.float32, device="cuda")
    GM.nmpc_gemm_bf16(Sb, Sb, C=Gm)
    ev, U = np.linalg.eigh(Gm.cpu().numpy().astype(np.float64))
    order = np.argsort(ev)[::-1][:rank]
    ev, U = np.maximum(ev[order], 1e-30), U[:, order]
    W = (U / np.sqrt(ev)[None, :]).T  # [r, ns]
    Wb = torch.from_numpy(np.ascontiguousarray(W, dtype=np.float32)).cuda().to(torch.bfloat16)
    St = torch.empty((ng, ns), dtype=torch.bfloat16, device="cuda")
    GM.nmpc_transpose_bf16(Sb, St)
    V = torch.zeros((ng, rank), dtype=torch.float32, device="cuda")
    GM.nmpc_gemm_bf16(St, Wb, C=V)
    Vn = V.cpu().numpy().astype(np.float64)
    # re-orthonormalise the float32 columns (Gram-Schmidt by QR, host float64)
    q, _ = np.linalg.qr(Vn)
    return q.astype(np.float32)


def project(fields: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Coefficients fields @ V on the tensor cores: [rows, ng] x [ng, r]."""
    torch = _torch()
    F = torch.from_numpy(np.ascontiguousarray(fields, dtype=np.float32)).cuda()
    Fb = torch.empty(F.shape, dtype=torch.bfloat16, device="cuda")
    GM.nmpc_cast_f32_bf16(F, Fb)
    Vt = torch.from_numpy(np.ascontiguousarray(V.T, dtype=np.float32)).cuda().to(torch.bfloat16)
    C = torch.zeros((F.shape[0], V.shape[1]), dtype=torch.float32, device="cuda")
    GM.nmpc_gemm_bf16(Fb, Vt.contiguous(), C=C)
    return C.cpu().numpy()


class LearnedWarmStart:
    """Trained predictor of (u, x, lambda) trajectory guesses for one problem
    shape (grid, horizon, actuators)."""

    def __init__(self, template, rank: int = 64, hidden: Sequence[int] = (512, 512, 512),
                 max_batch: int = 256, seed: int = 0):
        self.ng = template.mx * template.my
        self.N = template.horizon
        self.nu = len(template.act)
        self.rank = rank
        self.n_out = self.N * self.nu + 2 * self.N * rank
        self.widths = [2 * self.ng] + list(hidden) + [self.n_out]
        self.net = GM.MLP(self.widths, max_batch, seed)
        self.Vx = self.Vl = None
        self.mean = self.std = None

    # ---- training ----
    def fit(self, data: Dict[str, np.ndarray], steps: int = 1500, batch: int = 256,
            lr: float = 1e-3, n_pod: int = 4096, seed: int = 0, log=None) -> List[float]:
        torch = _torch()
        n = data["x0"].shape[0]
        rng = np.random.default_rng(seed)
        pick = rng.choice(n * self.N, size=min(n_pod, n * self.N), replace=False)
        self.Vx = pod_basis(data["dx"].reshape(-1, self.ng)[pick], self.rank)
        self.Vl = pod_basis(data["lam"].reshape(-1, self.ng)[pick], self.rank)
        cx = project(data["dx"].reshape(-1, self.ng), self.Vx).reshape(n, self.N * self.rank)
        cl = project(data["lam"].reshape(-1, self.ng), self.Vl).reshape(n, self.N * self.rank)
        T = np.concatenate([data["u"], cx, cl], axis=1).astype(np.float64)
        self.mean = T.mean(axis=0)
        self.std = T.std(axis=0) + 1e-12 * np.abs(T).max()
        Ts = ((T - self.mean) / self.std).astype(np.float32)
        X = np.concatenate([data["x0"], data["ref"]], axis=1).astype(np.float32)
        Xd = torch.from_numpy(X).cuda()
        Td = torch.from_numpy(Ts).cuda()
        losses = []
        batch = min(batch, self.net.max_batch, n - n % 8)
        for it in range(steps):
            idx = torch.from_numpy(rng.choice(n, size=batch, replace=False)).cuda()
            lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * it / steps))  # cosine decay
            want = (it % 50 == 0) or it == steps - 1
            loss = self.net.train_step(Xd[idx].contiguous(), Td[idx].contiguous(), lr_t,
                                       want_loss=want)
            if want:
                losses.append(loss)
                if log:
                    log(f"step {it} loss {loss:.4e}")
        self._fold_standardisation()
        return losses

    def _fold_standardisation(self):
        """y = std * y_s + mean: scale the last layer's rows and bias."""
        p = self.net.get_params().astype(np.float64)
        nin = self.widths[-2]
        nout = self.widths[-1]
        o = len(p) - (nin * nout + nout)
        W = p[o:o + nin * nout].reshape(nout, nin)
        b = p[o + nin * nout:]
        p[o:o + nin * nout] = (W * self.std[:, None]).ravel()
        p[o + nin * nout:] = b * self.std + self.mean
        self.net.set_params(p.astype(np.float32))

    # ---- inference ----
    def _forward(self, x0, ref):
        """Network output [B, n_out] (float32) and x0 as float32 [B, ng]."""
        torch = _torch()
        dev = x0.device
        B = x0.numel() // self.ng
        ng = self.ng
        x0v, rv = x0.view(B, ng), ref.view(B, ng)
        inp = torch.empty((B, 2 * ng), dtype=torch.float32, device=dev)
        x0f = torch.empty((B, ng), dtype=torch.float32, device=dev)
        for b in range(B):
            GM.nmpc_cast_f64_f32(x0v[b], x0f[b])
            GM.nmpc_cast_f64_f32(x0v[b], inp[b, :ng])
            GM.nmpc_cast_f64_f32(rv[b], inp[b, ng:])
        y = torch.empty((B, self.n_out), dtype=torch.float32, device=dev)
        self.net.forward(inp, y)
        return y, x0f

    def predict_controls(self, x0, ref):
        """Float64 device control guesses u [B*N*nu] only (the POD part of the
        output unused)."""
        torch = _torch()
        y, _ = self._forward(x0, ref)
        B, Nu = y.shape[0], self.N * self.nu
        u = torch.empty(B * Nu, dtype=torch.float64, device=x0.device)
        for b in range(B):
            GM.nmpc_cast_f32_f64(y[b, :Nu], u[b * Nu:(b + 1) * Nu])
        return u

    def predict_state(self, x0, ref):
        """Float64 device guesses (x [B*N*ng], u [B*N*nu], lam [B*N*ng]) for
        device float64 x0, ref [B*ng] (all on the GPU, all in library kernels)."""
        torch = _torch()
        dev = x0.device
        B = x0.numel() // self.ng
        ng, N, R, Nu = self.ng, self.N, self.rank, self.N * self.nu
        y, x0f = self._forward(x0, ref)
        yb = torch.empty((B, self.n_out), dtype=torch.bfloat16, device=dev)
        GM.nmpc_cast_f32_bf16(y, yb)
        Vx, Vl = self._vb(self.Vx), self._vb(self.Vl)
        xs = torch.empty((B, N, ng), dtype=torch.float32, device=dev)
        ls = torch.empty((B, N, ng), dtype=torch.float32, device=dev)
        for b in range(B):
            cx = yb[b, Nu:Nu + N * R].view(N, R)
            cl = yb[b, Nu + N * R:].view(N, R)
            # x_i = x0 + V_x c_i: the GEMM's bias adds x0 to every stage row
            GM.nmpc_gemm_bf16(cx, Vx, C=xs[b], bias=x0f[b])
            GM.nmpc_gemm_bf16(cl, Vl, C=ls[b])
        x = torch.empty(B * N * ng, dtype=torch.float64, device=dev)
        lam = torch.empty(B * N * ng, dtype=torch.float64, device=dev)
        u = torch.empty(B * Nu, dtype=torch.float64, device=dev)
        GM.nmpc_cast_f32_f64(xs.view(-1), x)
        GM.nmpc_cast_f32_f64(ls.view(-1), lam)
        for b in range(B):
            GM.nmpc_cast_f32_f64(y[b, :Nu], u[b * Nu:(b + 1) * Nu])
        return x, u, lam

    def _vb(self, V):
        torch = _torch()
        key = id(V)
        cache = getattr(self, "_vcache", {})
        if key not in cache:
            cache[key] = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float32)).cuda() \
                .to(torch.bfloat16).contiguous()
            self._vcache = cache
        return cache[key]

    def solve(self, solver: "G.Solver", check_residual: bool = False, decode: str = "pod"):
        """Solve `solver`'s instances from the predicted state.  decode "pod":
        state and costate from the predicted POD coefficients; "rollout": from
        the predicted controls' state and costate trajectories
        (nmpc_rollout).  The plain method stays the fallback: if the guessed
        start does not converge (diverged or max_iter) the instances are
        re-solved from the cold start.  Returns (rc, stats, used) with used
        "learned" or "cold"; with check_residual, stats gain the guess's
        float64 residual norms."""
        if decode == "rollout":
            torch = _torch()
            u = self.predict_controls(solver.x0, solver.ref)
            x = torch.empty(solver.n_s, dtype=torch.float64, device=u.device)
            lam = torch.empty_like(x)
            G.nmpc_rollout_fused(solver.h, solver.x0, solver.ref, u, x, lam)
        else:
            x, u, lam = self.predict_state(solver.x0, solver.ref)
        r_guess = None
        if check_residual:
            r_guess = G.nmpc_residual(solver.h, solver.x0, solver.ref, x, u, lam, solver.n)
        G.nmpc_set_state(solver.h, x, u, lam)
        rc, st = solver.solve(init=G.NMPC_INIT_GUESS)
        used = "learned"
        if rc != G.NMPC_OK:
            rc, st = solver.solve(init=G.NMPC_INIT_COLD)
            used = "cold"
        if check_residual:
            self.last_guess_residual = r_guess
        return rc, st, used

    # ---- checkpoint ----
    def save(self, path: str):
        np.savez(path, params=self.net.get_params(), widths=np.array(self.widths),
                 Vx=self.Vx, Vl=self.Vl, mean=self.mean, std=self.std,
                 shape=np.array([self.ng, self.N, self.nu, self.rank]))

    @classmethod
    def load(cls, path: str, template, max_batch: int = 256) -> "LearnedWarmStart":
        d = np.load(path)
        ng, N, nu, rank = (int(v) for v in d["shape"])
        ws = cls(template, rank=rank, hidden=list(d["widths"][1:-1]), max_batch=max_batch)
        assert (ws.ng, ws.N, ws.nu) == (ng, N, nu)
        ws.net.set_params(d["params"])
        ws.Vx, ws.Vl, ws.mean, ws.std = d["Vx"], d["Vl"], d["mean"], d["std"]
        return ws


class LearnedControlStart:
    """Learned start of the receding-horizon loop on large grids: a network
    maps the plant state and the reference, each reduced to f x f block means
    (library pooling kernel), to the control trajectory; the loops complete it
    with the state and costate trajectories the controls generate
    (nmpc_rollout) and start the solve there (closed_loop_learned_graph, or
    the host-driven closed_loop_learned with its other rules)."""

    def __init__(self, template, pool: int = 4, hidden: Sequence[int] = (512, 512, 512),
                 max_batch: int = 256, seed: int = 0):
        if template.mx % pool or template.my % pool:
            raise ValueError("grid not divisible by the pooling factor")
        self.mx, self.my, self.pool = template.mx, template.my, pool
        self.ngp = (template.mx // pool) * (template.my // pool)
        self.N, self.nu = template.horizon, len(template.act)
        self.n_out = self.N * self.nu
        self.widths = [2 * self.ngp] + list(hidden) + [self.n_out]
        self.net = GM.MLP(self.widths, max_batch, seed)
        self.mean = self.std = None

    def features(self, w, ref, B: int, out=None, stream=None):
        """Pooled [w; ref] rows, float32 device [B, 2 ngp] (into `out` if given;
        kernels only, so the call can be captured into a graph)."""
        torch = _torch()
        f = out if out is not None else torch.empty((B, 2 * self.ngp), dtype=torch.float32,
                                                    device=w.device)
        GM.nmpc_pool_avg(w, f, B, self.mx, self.my, self.pool, 2 * self.ngp, stream)
        GM.nmpc_pool_avg(ref, f[:, self.ngp:], B, self.mx, self.my, self.pool, 2 * self.ngp, stream)
        return f

    def fit(self, X: np.ndarray, U: np.ndarray, steps: int = 2000, batch: int = 128,
            lr: float = 1e-3, seed: int = 0) -> List[float]:
        """Train on pooled inputs X [n, 2 ngp] and control trajectories U [n, N nu]."""
        torch = _torch()
        n = X.shape[0]
        T = U.astype(np.float64)
        self.mean = T.mean(axis=0)
        self.std = T.std(axis=0) + 1e-12 * max(np.abs(T).max(), 1.0)
        Td = torch.from_numpy(((T - self.mean) / self.std).astype(np.float32)).cuda()
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        rng = np.random.default_rng(seed)
        batch = min(batch, self.net.max_batch, n - n % 8)
        losses = []
        for it in range(steps):
            idx = torch.from_numpy(rng.choice(n, size=batch, replace=False)).cuda()
            lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * it / steps))
            want = (it % 50 == 0) or it == steps - 1
            loss = self.net.train_step(Xd[idx].contiguous(), Td[idx].contiguous(), lr_t,
                                       want_loss=want)
            if want:
                losses.append(loss)
        LearnedWarmStart._fold_standardisation(self)
        return losses

    def predict_u(self, w, ref, B: int):
        """Control trajectory guesses, float64 device [B N nu]."""
        torch = _torch()
        u = torch.empty(B * self.n_out, dtype=torch.float64, device=w.device)
        self.predict_u_into(w, ref, B, u)
        return u

    def predict_u_into(self, w, ref, B: int, u, stream=None):
        """predict_u into the float64 device array u [B N nu] with buffers kept
        for the batch size: only kernel launches on `stream`, so the call can
        be captured into a CUDA graph (after one call outside the capture)."""
        torch = _torch()
        if getattr(self, "_buf_b", None) != B:
            self._f = torch.empty((B, 2 * self.ngp), dtype=torch.float32, device=w.device)
            self._y = torch.empty((B, self.n_out), dtype=torch.float32, device=w.device)
            self._buf_b = B
        self.net.forward(self.features(w, ref, B, self._f, stream), self._y, stream)
        GM.nmpc_cast_f32_f64(self._y.view(-1), u, stream)


def closed_loop_data(instances, steps: int, n_sub: int, pool: int = 4, tol: float = 1e-6,
                     precision: int = G.NMPC_MIXED):
    """Plain closed loops of `instances` (cold first step, shifted starts): per
    step the pooled [plant state; reference] rows and the solved control
    trajectories.  Returns X float32 [steps B, 2 ngp], U float32 [steps B, N nu]."""
    torch = _torch()
    B = len(instances)
    lcs = LearnedControlStart(instances[0], pool=pool, max_batch=8)
    s = G.Solver(instances, tol=tol, precision=precision, max_iter=6000)
    w = s.x0.clone()
    X, U = [], []
    for t in range(steps):
        rc, st = G.nmpc_solve(s.h, w, s.ref, s.u, B,
                              init=G.NMPC_INIT_COLD if t == 0 else G.NMPC_INIT_SHIFT)
        if rc != G.NMPC_OK:
            raise RuntimeError(f"training solve failed: {rc}")
        X.append(lcs.features(w, s.ref, B).cpu().numpy())
        U.append(s.u.view(B, -1).float().cpu().numpy())
        G.nmpc_plant_step(s.h, w, 0.0, n_sub)
    s.close()
    return np.concatenate(X), np.concatenate(U)


def closed_loop_learned(solver: "G.Solver", lcs: LearnedControlStart, w, steps: int,
                        n_sub: int, rule: str = "always",
                        decode: str = "rollout") -> Dict[str, object]:
    """Receding-horizon loop with the learned start: per step the plain
    candidate (cold at the first step, then the shifted previous solution)
    and the learned one: the predicted controls with, for decode "rollout",
    the state and costate trajectories they generate (nmpc_rollout), or, for
    decode "controls", the plain candidate's state and costate.  rule
    "residual": per instance the candidate with the smaller float64 residual
    starts the solve (NMPC_INIT_GUESS); rule "always": the learned candidate
    starts it, and a solve that does not converge is repeated from the plain
    one.  Then the plant moves one stage length.  w (device float64 plant
    state) is updated in place.  The initial residual predicts the iteration
    count poorly: the rollout start has the larger residual on the 256x256,
    N = 100 loop yet converges in fewer iterations, hence rule "always"."""
    torch = _torch()
    B = solver.n
    dev = w.device
    x = torch.empty(solver.n_s, dtype=torch.float64, device=dev)
    lam = torch.empty_like(x)
    x_l = torch.empty_like(x)
    lam_l = torch.empty_like(x)
    u_p = torch.empty(solver.n_u, dtype=torch.float64, device=dev)
    iters, chosen, r_plain, r_learn = [], [], [], []
    u_offs = np.cumsum([0] + [i.horizon * len(i.act) for i in solver.instances])
    s_offs = np.cumsum([0] + [i.horizon * i.mx * i.my for i in solver.instances])
    first = True
    for t in range(steps):
        init = G.NMPC_INIT_COLD if first else G.NMPC_INIT_SHIFT
        G.nmpc_start_state(solver.h, init, w, x, u_p, lam)
        u_l = lcs.predict_u(w, solver.ref, B)
        if decode == "rollout":
            G.nmpc_rollout(solver.h, w, solver.ref, u_l, x_l, lam_l)
        else:
            x_l.copy_(x)
            lam_l.copy_(lam)
        rp = G.nmpc_residual(solver.h, w, solver.ref, x, u_p, lam, B)[:, 0]
        rl = G.nmpc_residual(solver.h, w, solver.ref, x_l, u_l, lam_l, B)[:, 0]
        pick = (rl < rp) if rule == "residual" else np.ones(B, dtype=bool)
        xs, us, ls = x.clone(), u_p.clone(), lam.clone()
        for b in range(B):
            if pick[b]:
                us[u_offs[b]:u_offs[b + 1]].copy_(u_l[u_offs[b]:u_offs[b + 1]])
                xs[s_offs[b]:s_offs[b + 1]].copy_(x_l[s_offs[b]:s_offs[b + 1]])
                ls[s_offs[b]:s_offs[b + 1]].copy_(lam_l[s_offs[b]:s_offs[b + 1]])
        G.nmpc_set_state(solver.h, xs, us, ls)
        rc, st = G.nmpc_solve(solver.h, w, solver.ref, solver.u, B, init=G.NMPC_INIT_GUESS)
        if rc != G.NMPC_OK and pick.any():
            # the plain method is the fallback
            G.nmpc_set_state(solver.h, x, u_p, lam)
            rc, st = G.nmpc_solve(solver.h, w, solver.ref, solver.u, B, init=G.NMPC_INIT_GUESS)
            pick[:] = False
        if rc != G.NMPC_OK:
            raise RuntimeError(f"closed-loop solve failed: {rc}")
        iters.append([st[b].iters for b in range(B)])
        chosen.append(pick.astype(int).tolist())
        r_plain.append(rp.tolist())
        r_learn.append(rl.tolist())
        G.nmpc_plant_step(solver.h, w, 0.0, n_sub)
        first = False
    return {"iters": np.array(iters), "learned": np.array(chosen),
            "res_plain": np.array(r_plain), "res_learned": np.array(r_learn)}


def closed_loop_learned_graph(solver: "G.Solver", lcs: LearnedControlStart, w, steps: int,
                              n_sub: int, u_hist=None):
    """The closed loop with the learned start in one CUDA graph (with the
    handle's graph option): every step the network's controls (pooled plant
    state and reference -> controls), completed by their state and costate
    trajectories, start the solve.  w (device float64 plant state) is updated
    in place.  Returns (rc, iters [steps, n], res [steps, n])."""
    torch = _torch()
    B = solver.n
    u_guess = torch.empty(solver.n_u, dtype=torch.float64, device=w.device)
    lcs.predict_u_into(w, solver.ref, B, u_guess)  # buffers for this batch, outside any capture
    torch.cuda.synchronize()
    return G.nmpc_closed_loop_learned(
        solver.h, w, solver.ref, steps, n_sub, B,
        lambda st: lcs.predict_u_into(w, solver.ref, B, u_guess, st), u_guess, u_hist)


def evaluate(ws: LearnedWarmStart, seeds: Sequence[int], tol: float = 1e-6,
             precision: int = G.NMPC_MIXED, decode: str = "pod") -> Dict[str, float]:
    """Iterations and wall time to ||K||_inf <= tol from the cold start and
    from the learned start (decode as in LearnedWarmStart.solve; the cold
    start is the fallback when the learned one does not converge), one
    instance at a time."""
    torch = _torch()
    it_c, it_l, t_c, t_l, used = [], [], [], [], []
    for s in seeds:
        inst = wl.heat2d_learning_instance(s)
        sol = G.Solver([inst], tol=tol, precision=precision, max_iter=6000)
        sol.solve()  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = sol.solve(init=G.NMPC_INIT_COLD)
        torch.cuda.synchronize()
        t_c.append(time.perf_counter() - t0)
        it_c.append(st[0].iters)
        t0 = time.perf_counter()
        rc2, st2, u2 = ws.solve(sol, decode=decode)
        torch.cuda.synchronize()
        t_l.append(time.perf_counter() - t0)
        it_l.append(st2[0].iters)
        used.append(u2)
        assert rc == G.NMPC_OK and rc2 == G.NMPC_OK and st2[0].res_inf <= tol
        sol.close()
    return {"iters_cold": float(np.mean(it_c)), "iters_learned": float(np.mean(it_l)),
            "ms_cold": 1e3 * float(np.mean(t_c)), "ms_learned": 1e3 * float(np.mean(t_l)),
            "learned_used": used.count("learned") / len(used), "n": len(seeds),
            "decode": decode}


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train and evaluate the learned warm start")
    ap.add_argument("--train", type=int, default=2048)
    ap.add_argument("--test", type=int, default=32)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--rank", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    torch = _torch()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    data = generate(list(range(1_000_000, 1_000_000 + a.train)))
    t_gen = time.perf_counter() - t0
    ws = LearnedWarmStart(wl.heat2d_learning_instance(1_000_000), rank=a.rank)
    t0 = time.perf_counter()
    losses = ws.fit(data, steps=a.steps, lr=a.lr)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    if a.out:
        ws.save(a.out)
    res = evaluate(ws, list(range(2_000_000, 2_000_000 + a.test)))
    res["rollout"] = evaluate(ws, list(range(2_000_000, 2_000_000 + a.test)), decode="rollout")
    res.update({"train": a.train, "gen_s": t_gen, "fit_s": t_fit, "loss_first": losses[0],
                "loss_last": losses[-1], "mean_train_iters": float(data["iters"].mean())})
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
