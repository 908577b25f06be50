"""FP64 CPU oracle of second-order-in-time problems: a damped nonlinear wave.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may import this module; it shares no code with the
CUDA path.

Problem (Sec. 2, eq. 1 with a != 0; eqs. 4-5; Sec. 3, eqs. 6-8):
* grid: m points (dim 1) or m x m points (dim 2).  ``bc = "dirichlet"``:
  interior points of [0, 1]^dim, spacing 1 / (m + 1), zero outside;
  ``bc = "neumann"``: the points include the boundary, spacing 1 / (m - 1),
  mirrored fictitious points (eq. 3).
* PDE: a w_tt + b w_t = c Lap w + d(u, w) with constant a, b, c and
  d(u, w) = -kappa w^3 + sum_a gain u_a delta_a: the inputs are point
  forces at the actuator points ``act`` (force gain per unit input).
* state (eq. 5): x = (W, V), V = dW/dt, all W first, then all V (n_x = 2 n_g);
  f(u, x) = [V; g(u, x)], g = (c L W - b V - kappa W^3 + B u) / a, B the
  n_g x n_u matrix with ``gain`` at (act[a], a).
* NLP (eqs. 6-8): backward Euler x_i = x_{i-1} + h f(u_i, x_i); stage cost
  h (q/2 |W - W_ref|^2 + qv/2 |V|^2 + r/2 |u - u_ref|^2); terminal
  h qf/2 |W_N - W_ref|^2 (entered as lambda_{N+1}); regularization
  gamma/2 |u - u~|^2 with u~ = u^k (Remark 1).  No input bounds.
* KKT map (eq. 9), Newton (eq. 10, dense), the upper-layer Jacobi iteration
  (eq. 15), its Gauss-Seidel forms (eqs. 18-20) and the red-black order.
* Lower layer (Sec. 4.3): the two-step elimination of eqs. 22-24 with the
  u-iteration of Sec. 5.2; each F_x solve by the elimination of v6 (eq. 25):
  F_x = [[-I, h I], [h grad_W g, h grad_V g - I]], v6 = h v7 - b6 and
  E v7 = b7 + h grad_W g b6 with E = h grad_V g - I + h^2 grad_W g; each
  F_x^T solve by the same elimination on the transpose: E^T v9 = b9 + h b8,
  v8 = h grad_W g^T v9 - b8.  E and E^T by n_lo pointwise Jacobi sweeps
  from zero (Lemma 1).
Arrays: X, Lam (N, 2 n_g) as (W, V) per stage; U (N, n_u).
"""
from __future__ import annotations

import numpy as np


class WaveProblem:
    """One wave instance (duck-typed ``inst`` attributes: dim, m, bc, horizon,
    h, act, a, b, c, kappa, gain, q, qv, r, qf, gamma, x0 [2 n_g],
    w_ref [n_g], u_ref [n_u])."""

    def __init__(self, inst):
        self.dim, self.m, self.bc = int(inst.dim), int(inst.m), str(inst.bc)
        self.N, self.h = int(inst.horizon), float(inst.h)
        self.a, self.b, self.c = float(inst.a), float(inst.b), float(inst.c)
        self.kappa, self.gain = float(inst.kappa), float(inst.gain)
        self.q, self.qv, self.r, self.qf = float(inst.q), float(inst.qv), float(inst.r), float(inst.qf)
        self.gamma = float(inst.gamma)
        self.ng = self.m ** self.dim
        self.nx = 2 * self.ng
        self.act = np.asarray(inst.act, dtype=np.int64)
        self.nu = len(self.act)
        self.L = self.laplacian()
        self.B = np.zeros((self.ng, self.nu))
        for k, p in enumerate(self.act):
            self.B[p, k] = self.gain
        self.x0 = np.asarray(inst.x0, dtype=np.float64).copy()
        self.w_ref = np.asarray(inst.w_ref, dtype=np.float64).copy()
        self.u_ref = np.asarray(inst.u_ref, dtype=np.float64).copy()

    def laplacian(self):
        """Eqs. 2-4: 3-point (5-point in 2D) differences."""
        m = self.m
        if self.bc == "neumann":
            dp = 1.0 / (m - 1)
            L1 = np.zeros((m, m))
            for j in range(m):
                L1[j, j] = -2.0
                L1[j, j - 1 if j > 0 else 1] += 1.0          # mirrored fictitious point
                L1[j, j + 1 if j < m - 1 else m - 2] += 1.0
        else:
            dp = 1.0 / (m + 1)
            L1 = -2.0 * np.eye(m) + np.eye(m, k=1) + np.eye(m, k=-1)
        L1 /= dp * dp
        if self.dim == 1:
            return L1
        I = np.eye(m)
        return np.kron(I, L1) + np.kron(L1, I)

    def split(self, x):
        return x[:self.ng], x[self.ng:]

    def g(self, x, u):
        W, V = self.split(x)
        return (self.c * (self.L @ W) - self.b * V - self.kappa * W ** 3 + self.B @ u) / self.a

    def f(self, x, u):
        """Eq. 5: [V; g]."""
        return np.concatenate([self.split(x)[1], self.g(x, u)])

    def gW(self, x):
        """grad_W g = (c L - 3 kappa diag(W^2)) / a."""
        W = self.split(x)[0]
        return (self.c * self.L - np.diag(3.0 * self.kappa * W ** 2)) / self.a

    def gV(self):
        """grad_V g = -(b / a) I (a scalar)."""
        return -self.b / self.a

    def fx(self, x, u):
        n = self.ng
        J = np.zeros((self.nx, self.nx))
        J[:n, n:] = np.eye(n)
        J[n:, :n] = self.gW(x)
        J[n:, n:] = self.gV() * np.eye(n)
        return J

    def fu(self, x, u):
        return np.vstack([np.zeros((self.ng, self.nu)), self.B / self.a])

    def cold_start(self):
        """S^0: x_i = x0, u_i = 0, lambda = 0."""
        return np.tile(self.x0, (self.N, 1)), np.zeros((self.N, self.nu)), np.zeros((self.N, self.nx))

    def stage_cost_grad_x(self, x):
        W, V = self.split(x)
        return np.concatenate([self.q * (W - self.w_ref), self.qv * V])

    def terminal_grad_x(self, x):
        W = self.split(x)[0]
        return np.concatenate([self.qf * (W - self.w_ref), np.zeros(self.ng)])


# ---------------------------------------------------------------------------
# KKT map, eq. 9
# ---------------------------------------------------------------------------
def kkt(p: WaveProblem, X, U, Lam, u_tilde=None):
    """(K1 [N, n_x], K2 [N, n_u], K3 [N, n_x]); u_tilde None: u~ = u^k."""
    h = p.h
    K1, K2, K3 = np.zeros_like(X), np.zeros_like(U), np.zeros_like(Lam)
    for i in range(p.N):
        x, u, lam = X[i], U[i], Lam[i]
        xprev = p.x0 if i == 0 else X[i - 1]
        lnext = h * p.terminal_grad_x(x) if i == p.N - 1 else Lam[i + 1]
        K1[i] = xprev - x + h * p.f(x, u)
        K2[i] = h * (p.r * (u - p.u_ref) + p.fu(x, u).T @ lam)
        if u_tilde is not None:
            K2[i] += p.gamma * (u - u_tilde[i])
        K3[i] = lnext - lam + h * (p.stage_cost_grad_x(x) + p.fx(x, u).T @ lam)
    return K1, K2, K3


def kkt_norms(K1, K2, K3):
    a = np.concatenate([np.abs(K1).ravel(), np.abs(K2).ravel(), np.abs(K3).ravel()])
    return float(a.max()), float(np.sqrt(np.sum(a * a)))


def lagrangian(p: WaveProblem, X, U, Lam):
    """The Lagrangian of eq. 8 (without the regularization term) whose
    gradients are K: sum_i h l_i + h qf/2 |W_N - W_ref|^2 + lambda_i^T
    (x_{i-1} - x_i + h f(u_i, x_i))."""
    h, J = p.h, 0.0
    for i in range(p.N):
        x, u = X[i], U[i]
        W, V = p.split(x)
        J += h * (0.5 * p.q * np.sum((W - p.w_ref) ** 2) + 0.5 * p.qv * np.sum(V ** 2)
                  + 0.5 * p.r * np.sum((u - p.u_ref) ** 2))
        xprev = p.x0 if i == 0 else X[i - 1]
        J += Lam[i] @ (xprev - x + h * p.f(x, u))
    W = p.split(X[-1])[0]
    return J + h * 0.5 * p.qf * np.sum((W - p.w_ref) ** 2)


def hessians(p: WaveProblem, x, u, lam):
    """Diagonals of grad_xx H (W block: q - 6 kappa W lambda_V / a; V block:
    qv) and grad_uu H = r (g is linear in u; grad_xu H = 0)."""
    W = p.split(x)[0]
    lV = p.split(lam)[1]
    Hxx = np.concatenate([p.q - 6.0 * p.kappa * W * lV / p.a, np.full(p.ng, p.qv)])
    return Hxx, np.full(p.nu, p.r)


def stage_block(p: WaveProblem, X, U, Lam, i, with_gamma=True):
    """D_i = grad_{s_i} K_i, rows (K1, K2, K3), columns (x, u, lambda)."""
    h, nx, nu = p.h, p.nx, p.nu
    x, u, lam = X[i], U[i], Lam[i]
    Fx, Fu = p.fx(x, u), p.fu(x, u)
    Hxx, Huu = hessians(p, x, u, lam)
    axx = h * Hxx
    if i == p.N - 1:
        axx = axx + h * np.concatenate([np.full(p.ng, p.qf), np.zeros(p.ng)])
    D = np.zeros((2 * nx + nu, 2 * nx + nu))
    D[:nx, :nx] = h * Fx - np.eye(nx)
    D[:nx, nx:nx + nu] = h * Fu
    D[nx:nx + nu, nx:nx + nu] = np.diag(h * Huu + (p.gamma if with_gamma else 0.0))
    D[nx:nx + nu, nx + nu:] = h * Fu.T
    D[nx + nu:, :nx] = np.diag(axx)
    D[nx + nu:, nx + nu:] = h * Fx.T - np.eye(nx)
    return D


def pack(p, X, U, Lam):
    return np.concatenate([np.concatenate([X[i], U[i], Lam[i]]) for i in range(p.N)])


def unpack(p, S):
    n = 2 * p.nx + p.nu
    X, U, L = np.zeros((p.N, p.nx)), np.zeros((p.N, p.nu)), np.zeros((p.N, p.nx))
    for i in range(p.N):
        s = S[i * n:(i + 1) * n]
        X[i], U[i], L[i] = s[:p.nx], s[p.nx:p.nx + p.nu], s[p.nx + p.nu:]
    return X, U, L


def kkt_matrix(p: WaveProblem, X, U, Lam, with_gamma=False):
    """The block-tridiagonal matrix of eq. 10 (M_L: identity on the state
    rows / x columns; M_U: identity on the costate rows / lambda columns)."""
    n = 2 * p.nx + p.nu
    A = np.zeros((p.N * n, p.N * n))
    for i in range(p.N):
        A[i * n:(i + 1) * n, i * n:(i + 1) * n] = stage_block(p, X, U, Lam, i, with_gamma)
        if i > 0:
            A[i * n:i * n + p.nx, (i - 1) * n:(i - 1) * n + p.nx] = np.eye(p.nx)
        if i < p.N - 1:
            A[i * n + p.nx + p.nu:(i + 1) * n, (i + 1) * n + p.nx + p.nu:(i + 2) * n] = np.eye(p.nx)
    return A


def newton_solve(p: WaveProblem, S0=None, tol=1e-10, max_iter=40):
    """Newton on K(S) = 0 with the exact Jacobian of eq. 10 (dense)."""
    X, U, L = p.cold_start() if S0 is None else (a.copy() for a in S0)
    hist = []
    for _ in range(max_iter):
        K = kkt(p, X, U, L)
        r = kkt_norms(*K)[0]
        hist.append(r)
        if r <= tol:
            break
        Kp = np.concatenate([np.concatenate([K[0][i], K[1][i], K[2][i]]) for i in range(p.N)])
        dX, dU, dL = unpack(p, np.linalg.solve(kkt_matrix(p, X, U, L), Kp))
        X, U, L = X - dX, U - dU, L - dL
    return (X, U, L), hist


# ---------------------------------------------------------------------------
# Lower layer (Sec. 4.3, eqs. 21-25; u-iteration of Sec. 5.2)
# ---------------------------------------------------------------------------
class StageLower:
    """Approximate D_i^{-1} by the lower layer, for stage i of iterate k."""

    def __init__(self, p: WaveProblem, X, U, Lam, i, n_lo, n_u_it):
        h = p.h
        x, u, lam = X[i], U[i], Lam[i]
        self.p, self.h = p, h
        self.GW = p.gW(x)                                  # grad_W g
        self.gv = p.gV()                                   # grad_V g (scalar)
        self.E = (h * self.gv - 1.0) * np.eye(p.ng) + h * h * self.GW   # eq. 25
        self.Fu = h * p.fu(x, u)                           # F_u
        Hxx, Huu = hessians(p, x, u, lam)
        self.axx = h * Hxx
        if i == p.N - 1:
            self.axx = self.axx + h * np.concatenate([np.full(p.ng, p.qf), np.zeros(p.ng)])
        self.auu = h * Huu + p.gamma
        self.n_lo, self.n_u_it = n_lo, n_u_it

    def _jacobi(self, M, b):
        """Lemma 1: v <- D^{-1}(b - (M - D) v), n_lo sweeps from v = 0."""
        d = np.diag(M)
        off = M - np.diag(d)
        v = np.zeros_like(b)
        for _ in range(self.n_lo):
            v = (b - off @ v) / d
        return v

    def fx_solve(self, b):
        """F_x v = b by eliminating v6 (eq. 25)."""
        n, h = self.p.ng, self.h
        b6, b7 = b[:n], b[n:]
        v7 = self._jacobi(self.E, b7 + h * (self.GW @ b6))
        v6 = h * v7 - b6
        return np.concatenate([v6, v7])

    def fxT_solve(self, b):
        """F_x^T v = b by the same elimination on the transpose."""
        n, h = self.p.ng, self.h
        b8, b9 = b[:n], b[n:]
        v9 = self._jacobi(self.E.T, b9 + h * b8)
        v8 = h * (self.GW.T @ v9) - b8
        return np.concatenate([v8, v9])

    def p_inv(self, b4, b5):
        """[[0, F_x], [F_x^T, A_xx]] (v4, v5) = (b4, b5): F_x v5 = b4, then
        F_x^T v4 = b5 - A_xx v5."""
        v5 = self.fx_solve(b4)
        v4 = self.fxT_solve(b5 - self.axx * v5)
        return v4, v5

    def solve(self, b1, b2, b3):
        """(dx, du, dlam) for state rows b1, costate rows b2, u rows b3."""
        v3 = np.zeros_like(b3)
        for _ in range(self.n_u_it):
            ylam, _ = self.p_inv(self.Fu @ v3 - b1, -b2)
            v3 = (b3 + self.Fu.T @ ylam) / self.auu
        v1, v2 = self.p_inv(b1 - self.Fu @ v3, b2)
        return v2, v3, v1


def _solvers(p, X, U, L, n_lo, n_u_it, exact_inner):
    if exact_inner:
        out = []
        for i in range(p.N):
            D = stage_block(p, X, U, L, i)

            def solve(b1, b2, b3, D=D):
                d = np.linalg.solve(D, np.concatenate([b1, b3, b2]))
                return d[:p.nx], d[p.nx:p.nx + p.nu], d[p.nx + p.nu:]
            out.append(solve)
        return out
    return [StageLower(p, X, U, L, i, n_lo, n_u_it).solve for i in range(p.N)]


def gs_order(N, kind):
    if kind == "jacobi":
        return None
    if kind == "forward":
        return list(range(N))
    if kind == "backward":
        return list(range(N - 1, -1, -1))
    if kind == "redblack":
        return list(range(0, N, 2)) + list(range(1, N, 2))
    raise ValueError(kind)


def iteration(p: WaveProblem, X, U, Lam, variant="jacobi", n_lo=2, n_u_it=2, exact_inner=False):
    """One upper-layer iteration: the direction D^{-1} K (jacobi, eq. 15),
    (D + L_o)^{-1} K in the given stage order (fgs / bgs / redblack, eq. 18)
    or eq. 20 (sgs), all from iterate k, then S <- S - dS (no bounds: the
    full step).  Returns (X, U, Lam) and the norms of K^k."""
    K1, K2, K3 = kkt(p, X, U, Lam)
    norms = kkt_norms(K1, K2, K3)
    solve = _solvers(p, X, U, Lam, n_lo, n_u_it, exact_inner)
    N = p.N
    dX, dU, dL = np.zeros_like(X), np.zeros_like(U), np.zeros_like(Lam)
    if variant == "sgs":
        zL = np.zeros_like(Lam)
        for i in range(N - 1, -1, -1):
            b2 = K3[i] - zL[i + 1] if i < N - 1 else K3[i]
            _, _, zL[i] = solve[i](K1[i], b2, K2[i])
        for i in range(N):
            b1 = K1[i] - dX[i - 1] if i > 0 else K1[i]
            b2 = K3[i] - zL[i + 1] if i < N - 1 else K3[i]
            dX[i], dU[i], dL[i] = solve[i](b1, b2, K2[i])
    else:
        order = gs_order(N, {"jacobi": "jacobi", "fgs": "forward", "bgs": "backward",
                             "redblack": "redblack"}[variant])
        if order is None:
            for i in range(N):
                dX[i], dU[i], dL[i] = solve[i](K1[i], K3[i], K2[i])
        else:
            seen = np.zeros(N, dtype=bool)
            for i in order:
                b1 = K1[i] - dX[i - 1] if (i > 0 and seen[i - 1]) else K1[i]
                b2 = K3[i] - dL[i + 1] if (i < N - 1 and seen[i + 1]) else K3[i]
                dX[i], dU[i], dL[i] = solve[i](b1, b2, K2[i])
                seen[i] = True
    return X - dX, U - dU, Lam - dL, norms


def solve(p: WaveProblem, variant="jacobi", S0=None, tol=1e-6, max_iter=5000, **kw):
    """Iterate until ||K^k||_inf <= tol; ((X, U, Lam), info)."""
    X, U, L = p.cold_start() if S0 is None else (a.copy() for a in S0)
    for k in range(max_iter + 1):
        r_inf, r_2 = kkt_norms(*kkt(p, X, U, L))
        if (not np.isfinite(r_inf)) or r_inf <= tol or k == max_iter:
            return (X, U, L), dict(iters=k, res_inf=r_inf, res_2=r_2, converged=r_inf <= tol,
                                   diverged=not np.isfinite(r_inf))
        X, U, L, _ = iteration(p, X, U, L, variant, **kw)


# ---------------------------------------------------------------------------
# Brute-force view of the NLP (eq. 8) for pins
# ---------------------------------------------------------------------------
def simulate(p: WaveProblem, U, tol=1e-13):
    """States of x_i = x_{i-1} + h f(u_i, x_i), each stage by Newton on x."""
    X = np.zeros((p.N, p.nx))
    x = p.x0.copy()
    for i in range(p.N):
        xp = x.copy()
        for _ in range(60):
            res = xp - x + p.h * p.f(x, U[i])
            J = p.h * p.fx(x, U[i]) - np.eye(p.nx)
            dx = np.linalg.solve(J, res)
            x = x - dx
            if np.max(np.abs(dx)) < tol * max(1.0, np.max(np.abs(x))):
                break
        X[i] = x
    return X


def reduced_cost(p: WaveProblem, U):
    """The NLP objective (eq. 8) with the states simulated."""
    X = simulate(p, U)
    J = 0.0
    for i in range(p.N):
        W, V = p.split(X[i])
        J += p.h * (0.5 * p.q * np.sum((W - p.w_ref) ** 2) + 0.5 * p.qv * np.sum(V ** 2)
                    + 0.5 * p.r * np.sum((U[i] - p.u_ref) ** 2))
    W = p.split(X[-1])[0]
    return J + p.h * 0.5 * p.qf * np.sum((W - p.w_ref) ** 2)


# ---------------------------------------------------------------------------
# The plant of the closed loop (Sec. 5.3)
# ---------------------------------------------------------------------------
def plant_step(p: WaveProblem, x, u1, dt, n_sub):
    """Advance the true system x = (W, V) by dt with the inputs held at u1:
    n_sub semi-implicit (symplectic) Euler steps of the same model,
    V <- V + tau g(W, V, u1), then W <- W + tau V with the new V (tau =
    dt / n_sub).  (Explicit Euler would amplify every undamped mode.)"""
    x = np.asarray(x, dtype=np.float64).copy()
    u1 = np.asarray(u1, dtype=np.float64)
    tau = dt / n_sub
    for _ in range(n_sub):
        W, V = x[:p.ng].copy(), x[p.ng:].copy()
        V = V + tau * p.g(np.concatenate([W, V]), u1)
        W = W + tau * V
        x = np.concatenate([W, V])
    return x


def closed_loop(inst, steps, n_sub, tol=1e-9, max_iter=20000, variant="jacobi"):
    """Receding horizon: each period solves from the plant's state (the first
    from the cold start, later ones from the previous solution shifted by one
    stage, the last repeated), applies u_1 for one stage length h and
    advances the plant.  Returns the applied inputs, the iteration counts and
    the final plant state."""
    import copy
    cur = copy.copy(inst)
    x = np.asarray(inst.x0, dtype=np.float64).copy()
    S, us, its = None, [], []
    for _ in range(steps):
        cur.x0 = x.copy()
        p = WaveProblem(cur)
        (X, U, L), info = solve(p, variant, S0=S, tol=tol, max_iter=max_iter)
        us.append(U[0].copy())
        its.append(info["iters"])
        x = plant_step(p, x, U[0], p.h, n_sub)
        S = tuple(np.vstack([A[1:], A[-1:]]) for A in (X, U, L))
    return np.array(us), np.array(its), x
