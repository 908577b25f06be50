"""FP64 CPU oracle of pinned-actuator problems: the paper's copper plate.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may import this module; it shares no code with the
CUDA path.

Problem (Sec. 5.1 and the model class of Sec. 2, eq. 1 with a = 0):
* grid: m x m points on [0, 1]^2 (dim 2) or m points on [0, 1] (dim 1).
  ``bc = "neumann"``: the points include the boundary, spacing 1 / (m - 1),
  zero-Neumann condition by mirrored fictitious points (eq. 3: w_{-1} =
  w_1, w_{m} = w_{m-2}); ``bc = "dirichlet"``: interior points, spacing
  1 / (m + 1), zero outside.
* actuators: the temperatures of the points in ``act`` are the inputs u
  (Sec. 5.1: they are controlled directly), so they are not states: the
  state x holds the other points (16 of 169 -> 153 states on the plate).
* model: w_t = Lap Phi(w) - beta (w - T_a) - gamma_r (w^4 - T_a^4),
  Phi(w) = k0 (w + k1 w^2 / 2) (k1 = 0: linear diffusion k0 Lap w), taken at
  the state points with w = x there and w = u at the actuator points; so
  f(u, x) = L_SS Phi(x) + L_SA Phi(u) - beta (x - T_a) - gamma_r (x^4 - T_a^4).
  For the plate (Table 1): rho C_p t_z w_t = k t_z Lap w - 2 Q_c - 2 Q_r gives
  k0 = k / (rho C_p), beta = 2 h_c / (rho C_p t_z), gamma_r = 2 eps sigma /
  (rho C_p t_z).
* NLP (eqs. 6-8): backward Euler, stage cost h (1/2 |x - x_ref|_Q^2 +
  1/2 |u - u_ref|_R^2 + Phi_b(u)), log barrier Phi_b(u) = -tau sum
  (ln(u - u_lo) + ln(u_hi - u)) of the input bounds (tau = 0: no barrier),
  terminal h qf / 2 |x_N - x_ref|^2 (qf = 0 on the plate), regularization
  gamma/2 |u - u~|^2 with u~ = u^k (Remark 1).
* KKT map (eq. 9), Newton (eq. 10, dense), the upper-layer Jacobi iteration
  (eq. 15) and the block Gauss-Seidel variants (eqs. 18-20), each with the
  step length of the fraction-to-the-boundary rule (eq. 11): the largest
  alpha in (0, 1] with G(u^{k+1}) >= 0.005 G(u^k) for every bound of every
  stage.  The lower layer (Sec. 4.3, eqs. 21-24) with the u fixed-point
  iteration of Sec. 5.2 (n_u_it steps from v3 = 0), P^{-1} by n_lo
  pointwise Jacobi sweeps on F_x and F_x^T (Lemma 1).
Arrays: X, Lam (N, ns) over the state points in grid order; U (N, nu).
"""
from __future__ import annotations

import numpy as np


class PinnedProblem:
    """One pinned-actuator instance (duck-typed ``inst`` attributes: dim, m,
    bc, horizon, h, act, k0, k1, beta, t_amb, gamma_r, q, r, qf, gamma, tau,
    u_lo, u_hi, x0 [ns], x_ref [ns], u_ref [nu])."""

    def __init__(self, inst):
        self.dim = int(inst.dim)
        self.m = int(inst.m)
        self.bc = str(inst.bc)
        self.N = int(inst.horizon)
        self.h = float(inst.h)
        self.k0, self.k1 = float(inst.k0), float(inst.k1)
        self.beta, self.Ta, self.gr = float(inst.beta), float(inst.t_amb), float(inst.gamma_r)
        self.q, self.r, self.qf = float(inst.q), float(inst.r), float(inst.qf)
        self.gamma, self.tau = float(inst.gamma), float(inst.tau)
        self.u_lo, self.u_hi = float(inst.u_lo), float(inst.u_hi)
        self.ng = self.m ** self.dim
        self.act = np.asarray(inst.act, dtype=np.int64)
        self.nu = len(self.act)
        is_act = np.zeros(self.ng, dtype=bool)
        is_act[self.act] = True
        self.S = np.nonzero(~is_act)[0]          # state points, grid order
        self.ns = len(self.S)
        self.L = self.laplacian()
        self.LSS = self.L[np.ix_(self.S, self.S)]
        self.LSA = self.L[np.ix_(self.S, self.act)]
        self.x0 = np.asarray(inst.x0, dtype=np.float64).copy()
        self.x_ref = np.asarray(inst.x_ref, dtype=np.float64).copy()
        self.u_ref = np.asarray(inst.u_ref, dtype=np.float64).copy()

    # eqs. 2-4: finite differences with fictitious points
    def laplacian(self):
        m = self.m
        if self.bc == "neumann":
            dp = 1.0 / (m - 1)
            L1 = np.zeros((m, m))
            for j in range(m):
                L1[j, j] = -2.0
                # a fictitious neighbour mirrors the inner one (zero normal derivative)
                left = j - 1 if j > 0 else 1
                right = j + 1 if j < m - 1 else m - 2
                L1[j, left] += 1.0
                L1[j, right] += 1.0
        else:
            dp = 1.0 / (m + 1)
            L1 = -2.0 * np.eye(m) + np.eye(m, k=1) + np.eye(m, k=-1)
        L1 /= dp * dp
        if self.dim == 1:
            return L1
        I = np.eye(m)
        return np.kron(I, L1) + np.kron(L1, I)

    def phi(self, w):
        return self.k0 * (w + 0.5 * self.k1 * w * w)

    def dphi(self, w):
        return self.k0 * (1.0 + self.k1 * w)

    @property
    def d2phi(self):
        return self.k0 * self.k1

    def f(self, x, u):
        return (self.LSS @ self.phi(x) + self.LSA @ self.phi(u) - self.beta * (x - self.Ta)
                - self.gr * (x ** 4 - self.Ta ** 4))

    def fx(self, x, u):
        """grad_x f = L_SS diag(Phi'(x)) - diag(beta + 4 gamma_r x^3)."""
        return self.LSS * self.dphi(x)[None, :] - np.diag(self.beta + 4.0 * self.gr * x ** 3)

    def fu(self, x, u):
        """grad_u f = L_SA diag(Phi'(u))."""
        return self.LSA * self.dphi(u)[None, :]

    # barrier of the input bounds (eq. 8)
    def barrier(self, u):
        if self.tau == 0.0:
            return 0.0
        return -self.tau * float(np.sum(np.log(u - self.u_lo) + np.log(self.u_hi - u)))

    def dbarrier(self, u):
        if self.tau == 0.0:
            return np.zeros_like(u)
        return -self.tau / (u - self.u_lo) + self.tau / (self.u_hi - u)

    def d2barrier(self, u):
        if self.tau == 0.0:
            return np.zeros_like(u)
        return self.tau / (u - self.u_lo) ** 2 + self.tau / (self.u_hi - u) ** 2

    def cold_start(self, u0=None):
        """S^0: x_i = x0, u_i = u0 (default: mid-range when bounded, else 0), lambda = 0."""
        if u0 is None:
            u0 = 0.5 * (self.u_lo + self.u_hi) if self.tau > 0 else 0.0
        X = np.tile(self.x0, (self.N, 1))
        U = np.full((self.N, self.nu), float(u0))
        return X, U, np.zeros((self.N, self.ns))


# ---------------------------------------------------------------------------
# KKT map, eq. 9
# ---------------------------------------------------------------------------
def kkt(p: PinnedProblem, X, U, Lam, u_tilde=None):
    """(K1 [N, ns], K2 [N, nu], K3 [N, ns]); u_tilde None: u~ = u^k."""
    h = p.h
    K1, K2, K3 = np.zeros_like(X), np.zeros_like(U), np.zeros_like(Lam)
    for i in range(p.N):
        x, u, lam = X[i], U[i], Lam[i]
        xprev = p.x0 if i == 0 else X[i - 1]
        lnext = h * p.qf * (x - p.x_ref) if i == p.N - 1 else Lam[i + 1]
        K1[i] = xprev - x + h * p.f(x, u)
        K2[i] = h * (p.r * (u - p.u_ref) + p.dbarrier(u) + p.fu(x, u).T @ lam)
        if u_tilde is not None:
            K2[i] += p.gamma * (u - u_tilde[i])
        K3[i] = lnext - lam + h * (p.q * (x - p.x_ref) + p.fx(x, u).T @ lam)
    return K1, K2, K3


def kkt_norms(K1, K2, K3):
    a = np.concatenate([np.abs(K1).ravel(), np.abs(K2).ravel(), np.abs(K3).ravel()])
    return float(a.max()), float(np.sqrt(np.sum(a * a)))


def lagrangian(p: PinnedProblem, X, U, Lam):
    """Cost of eq. 8 (barrier included, gamma-term zero at u~ = u) plus
    sum_i lambda_i^T (x_{i-1} - x_i + h f(u_i, x_i))."""
    val, h = 0.0, p.h
    for i in range(p.N):
        x, u = X[i], U[i]
        xprev = p.x0 if i == 0 else X[i - 1]
        val += h * (0.5 * p.q * np.sum((x - p.x_ref) ** 2) + 0.5 * p.r * np.sum((u - p.u_ref) ** 2)
                    + p.barrier(u))
        val += Lam[i] @ (xprev - x + h * p.f(x, u))
    return val + h * 0.5 * p.qf * np.sum((X[-1] - p.x_ref) ** 2)


# ---------------------------------------------------------------------------
# Stage blocks (eq. 17) and the dense KKT matrix (eq. 10)
# ---------------------------------------------------------------------------
def hessians(p: PinnedProblem, x, u, lam):
    """grad_xx H and grad_uu H (diagonal vectors; grad_xu H = 0 here: f is a
    sum of an x-part and a u-part)."""
    Hxx = p.q + p.d2phi * (p.LSS.T @ lam) - 12.0 * p.gr * x ** 2 * lam
    Huu = p.r + p.d2barrier(u) + p.d2phi * (p.LSA.T @ lam)
    return Hxx, Huu


def stage_block(p: PinnedProblem, X, U, Lam, i, with_gamma=True):
    """D_i = grad_{s_i} K_i, rows (K1, K2, K3), columns (x, u, lambda)."""
    h, ns, nu = p.h, p.ns, p.nu
    x, u, lam = X[i], U[i], Lam[i]
    Fx, Fu = p.fx(x, u), p.fu(x, u)
    Hxx, Huu = hessians(p, x, u, lam)
    D = np.zeros((2 * ns + nu, 2 * ns + nu))
    D[:ns, :ns] = h * Fx - np.eye(ns)
    D[:ns, ns:ns + nu] = h * Fu
    D[ns:ns + nu, ns:ns + nu] = np.diag(h * Huu + (p.gamma if with_gamma else 0.0))
    D[ns:ns + nu, ns + nu:] = h * Fu.T
    D[ns + nu:, :ns] = np.diag(h * Hxx + (h * p.qf if i == p.N - 1 else 0.0))
    D[ns + nu:, ns + nu:] = h * Fx.T - np.eye(ns)
    return D


def pack(p, X, U, Lam):
    return np.concatenate([np.concatenate([X[i], U[i], Lam[i]]) for i in range(p.N)])


def unpack(p, S):
    n = 2 * p.ns + p.nu
    X, U, L = np.zeros((p.N, p.ns)), np.zeros((p.N, p.nu)), np.zeros((p.N, p.ns))
    for i in range(p.N):
        s = S[i * n:(i + 1) * n]
        X[i], U[i], L[i] = s[:p.ns], s[p.ns:p.ns + p.nu], s[p.ns + p.nu:]
    return X, U, L


def kkt_matrix(p: PinnedProblem, X, U, Lam, with_gamma=False):
    """The block-tridiagonal matrix of eq. 10 (M_L: identity on the state
    rows / x columns; M_U: identity on the costate rows / lambda columns)."""
    n = 2 * p.ns + p.nu
    A = np.zeros((p.N * n, p.N * n))
    for i in range(p.N):
        A[i * n:(i + 1) * n, i * n:(i + 1) * n] = stage_block(p, X, U, Lam, i, with_gamma)
        if i > 0:
            A[i * n:i * n + p.ns, (i - 1) * n:(i - 1) * n + p.ns] = np.eye(p.ns)
        if i < p.N - 1:
            A[i * n + p.ns + p.nu:(i + 1) * n, (i + 1) * n + p.ns + p.nu:(i + 2) * n] = np.eye(p.ns)
    return A


# ---------------------------------------------------------------------------
# Fraction-to-the-boundary rule, eq. 11
# ---------------------------------------------------------------------------
def alpha_max(p: PinnedProblem, U, dU, frac=0.995):
    """Largest alpha in (0, 1] with G(U - alpha dU) >= (1 - frac) G(U) for
    both bounds of every input of every stage (no bounds: 1)."""
    if p.tau == 0.0:
        return 1.0
    a = 1.0
    up = dU > 0          # u decreases: the lower bound G = u - u_lo shrinks
    if np.any(up):
        a = min(a, float(np.min(frac * (U[up] - p.u_lo) / dU[up])))
    dn = dU < 0          # u increases: the upper bound G = u_hi - u shrinks
    if np.any(dn):
        a = min(a, float(np.min(frac * (p.u_hi - U[dn]) / (-dU[dn]))))
    return a


# ---------------------------------------------------------------------------
# Newton (Sec. 3.3) on the full system, dense
# ---------------------------------------------------------------------------
def newton_solve(p: PinnedProblem, S0=None, tol=1e-10, max_iter=60):
    """Newton on K(S) = 0 (the exact Jacobian of eq. 10), the step cut to the
    fraction-to-the-boundary length (eq. 11) and then halved while it does
    not lower ||K||_inf (a damped Newton: only the root is used, as the
    reference the iterations are checked against)."""
    X, U, L = p.cold_start() if S0 is None else (a.copy() for a in S0)
    hist = []
    for _ in range(max_iter):
        K = kkt(p, X, U, L)
        r = kkt_norms(*K)[0]
        hist.append(r)
        if r <= tol:
            break
        Kp = np.concatenate([np.concatenate([K[0][i], K[1][i], K[2][i]]) for i in range(p.N)])
        dS = np.linalg.solve(kkt_matrix(p, X, U, L), Kp)
        dX, dU, dL = unpack(p, dS)
        a = alpha_max(p, U, dU)
        for _ in range(40):
            Xn, Un, Ln = X - a * dX, U - a * dU, L - a * dL
            if kkt_norms(*kkt(p, Xn, Un, Ln))[0] < r:
                break
            a *= 0.5
        X, U, L = Xn, Un, Ln
    return (X, U, L), hist


# ---------------------------------------------------------------------------
# Lower layer (Sec. 4.3, eqs. 21-24; u-iteration of Sec. 5.2)
# ---------------------------------------------------------------------------
class StageLower:
    """Approximate D_i^{-1} by the lower layer, for stage i of iterate k."""

    def __init__(self, p: PinnedProblem, X, U, Lam, i, n_lo, n_u_it):
        h = p.h
        x, u, lam = X[i], U[i], Lam[i]
        self.Fx = h * p.fx(x, u) - np.eye(p.ns)          # F_x
        self.Fu = h * p.fu(x, u)                          # F_u
        Hxx, Huu = hessians(p, x, u, lam)
        self.axx = h * Hxx + (h * p.qf if i == p.N - 1 else 0.0)
        self.auu = h * Huu + p.gamma
        self.d = np.diag(self.Fx).copy()
        self.n_lo, self.n_u_it = n_lo, n_u_it

    def _jacobi(self, M, b):
        """Lemma 1: v <- D^{-1}(b - (M - D) v), n_lo sweeps from v = 0."""
        v = np.zeros_like(b)
        off = M - np.diag(self.d)
        for _ in range(self.n_lo):
            v = (b - off @ v) / self.d
        return v

    def p_inv(self, b4, b5):
        v5 = self._jacobi(self.Fx, b4)
        v4 = self._jacobi(self.Fx.T, b5 - self.axx * v5)
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
                return d[:p.ns], d[p.ns:p.ns + p.nu], d[p.ns + p.nu:]
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


def iteration(p: PinnedProblem, X, U, Lam, variant="jacobi", n_lo=2, n_u_it=2,
              exact_inner=False):
    """One upper-layer iteration: the direction D^{-1} K (jacobi, eq. 15),
    (D + L_o)^{-1} K (fgs / bgs / redblack, eq. 18 in the given stage order)
    or eq. 20 (sgs), all from iterate k, then S <- S - alpha_max dS (eq. 11).
    Returns (X, U, Lam), the norms of K^k and alpha."""
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
    a = alpha_max(p, U, dU)
    return X - a * dX, U - a * dU, Lam - a * dL, norms, a


def solve(p: PinnedProblem, variant="jacobi", S0=None, tol=1e-6, max_iter=5000, **kw):
    """Iterate until ||K^k||_inf <= tol; ((X, U, Lam), info)."""
    X, U, L = p.cold_start() if S0 is None else (a.copy() for a in S0)
    alphas = []
    for k in range(max_iter + 1):
        r_inf, r_2 = kkt_norms(*kkt(p, X, U, L))
        if (not np.isfinite(r_inf)) or r_inf <= tol or k == max_iter:
            return (X, U, L), dict(iters=k, res_inf=r_inf, res_2=r_2, converged=r_inf <= tol,
                                   diverged=not np.isfinite(r_inf), alphas=alphas)
        X, U, L, _, a = iteration(p, X, U, L, variant, **kw)
        alphas.append(a)


# ---------------------------------------------------------------------------
# Brute-force view of the NLP (eq. 8) for pins
# ---------------------------------------------------------------------------
def simulate(p: PinnedProblem, U, tol=1e-13):
    """States of x_i = x_{i-1} + h f(u_i, x_i), each stage by Newton on x."""
    X = np.zeros((p.N, p.ns))
    x = p.x0.copy()
    for i in range(p.N):
        xp = x.copy()
        for _ in range(60):
            res = xp - x + p.h * p.f(x, U[i])
            J = p.h * p.fx(x, U[i]) - np.eye(p.ns)
            dx = np.linalg.solve(J, res)
            x = x - dx
            if np.max(np.abs(dx)) < tol * max(1.0, np.max(np.abs(x))):
                break
        X[i] = x
    return X


def reduced_cost(p: PinnedProblem, U):
    """The NLP objective (eq. 8, barrier included) with the states simulated."""
    X = simulate(p, U)
    J = sum(p.h * (0.5 * p.q * np.sum((X[i] - p.x_ref) ** 2)
                   + 0.5 * p.r * np.sum((U[i] - p.u_ref) ** 2) + p.barrier(U[i]))
            for i in range(p.N))
    return J + p.h * 0.5 * p.qf * np.sum((X[-1] - p.x_ref) ** 2)


def plant_step(p: PinnedProblem, x, u1, dt, n_sub):
    """The plant (Sec. 5.3): explicit-Euler sub-steps of the same model with
    the actuator points held at u1."""
    x = np.asarray(x, dtype=np.float64).copy()
    for _ in range(n_sub):
        x = x + (dt / n_sub) * p.f(x, np.asarray(u1, dtype=np.float64))
    return x
