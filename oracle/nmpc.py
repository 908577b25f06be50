"""FP64 CPU oracle for the double-layer Jacobi method (Deng & Ohtsuka).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this module.  The
CUDA path never calls it and it never calls the CUDA path; the two share no
code.  Inputs are duck-typed instance objects with the attributes
``dim, mx, my, horizon, h, act, act_gain, q, r, qf, gamma, k0, k1, x0, ref``.

What is computed, in the paper's notation:

* Model (Sec. 2, eqs. 1 and 4): first-order heat equation
  w_t = div(k(w) grad w) + sum_a b0 u_a [cell a], k(w) = k0 (1 + k1 w), on
  interior grid cells with a Dirichlet-zero ring; the source is the d(u, w)
  term of eq. 1.  The conservative flux with face conductivity
  k((w_j + w_m)/2) equals the 3-/5-point Laplacian of the Kirchhoff
  transform Phi(w) = k0 (w + k1 w^2 / 2) because k is affine, so
  f(u, x) = Lap_h Phi(x) + b0 B u, B the 0/1 cell-selection matrix.
* NLP (Sec. 3, eq. 6): backward Euler x_i = x_{i-1} + h f(u_i, x_i); every
  cost term carries the factor h: h/2 (q |x_i - ref|^2 + r |u_i|^2) per stage
  and h/2 qf |x_N - ref|^2 at the end, entered as
  lambda_{N+1} = h qf (x_N - ref).
* Regularization (eq. 7) with u~ = u^k (Remark 1): gamma (u_i - u~_i) is zero
  in K^k; gamma I sits in the u-block of D_i.
* KKT map (Sec. 3.2, eq. 9): K_i = [x_{i-1} - x_i + h f;
  h grad_u H + gamma (u - u~); lambda_{i+1} - lambda_i + h grad_x H].
* Newton (Sec. 3.3, eq. 10) with the block elimination recursion
  D^_i = D_i - M_U D^_{i+1}^{-1} M_L; dense LU of the whole matrix (tiny).
* Upper-layer Jacobi (Sec. 4.2, eq. 15): S <- S - alpha D^{-1} K, all stages
  at once from x_{i-1} and lambda_{i+1} of iterate k.
* Jacobi-type variants (Sec. 4.2, eqs. 18-20): block Gauss-Seidel (D + L)^{-1}
  in forward (FGS), backward (BGS) or red-black stage order, and the
  symmetric sweep (SGS) of eq. 20, each with D^k, K^k of iterate k.
* Lower layer (Sec. 4.3, eqs. 21-24, and the u-iteration of Sec. 5.2):
  reordered block [[0, F_x, F_u], [F_x^T, A_xx, A_xu], [F_u^T, A_ux, A_uu]];
  v3 by ``n_u_it`` steps A_uu v3+ = b3 + [F_u^T A_ux] P^{-1}([F_u; A_xu] v3
  - [b1; b2]) from v3 = 0, then (v1, v2) = P^{-1}([b1; b2] - [F_u; A_xu] v3);
  P^{-1} solves F_x v5 = b4 then F_x^T v4 = b5 - A_xx v5, each by ``n_lo``
  pointwise Jacobi sweeps from zero (Lemma 1).
* Linear case k1 = 0: discrete LQ by the Riccati recursion (textbook closed
  form), used only to pin the root.

Arrays: X, Lam are (N, my, mx); U is (N, n_u).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# Problem data and model, Sec. 2
# ---------------------------------------------------------------------------
class Problem:
    """Grid geometry and weights of one instance, in float64."""

    def __init__(self, inst):
        self.dim = int(inst.dim)
        self.mx = int(inst.mx)
        self.my = int(inst.my)
        self.N = int(inst.horizon)
        self.h = float(inst.h)
        self.q = float(inst.q)
        self.r = float(inst.r)
        self.qf = float(inst.qf)
        self.gamma = float(inst.gamma)
        self.k0 = float(inst.k0)
        self.k1 = float(inst.k1)
        self.b0 = float(getattr(inst, "act_gain", 32.0))
        self.dx = 1.0 / (self.mx + 1)
        self.dy = 1.0 / (self.my + 1)
        self.act = np.asarray(inst.act, dtype=np.int64)
        self.nu = len(self.act)
        self.ng = self.mx * self.my
        self.shape = (self.my, self.mx)
        self.x0 = np.asarray(inst.x0, dtype=np.float64).reshape(self.shape).copy()
        self.ref = np.asarray(inst.ref, dtype=np.float64).reshape(self.shape).copy()

    # eq. 4: finite-difference Laplacian with the Dirichlet-zero ring
    def lap(self, v):
        """3-point (1D) or 5-point (2D) Laplacian of v[..., my, mx]."""
        out = (-2.0 / self.dx ** 2) * v
        out[..., :, 1:] += v[..., :, :-1] / self.dx ** 2
        out[..., :, :-1] += v[..., :, 1:] / self.dx ** 2
        if self.dim == 2:
            out += (-2.0 / self.dy ** 2) * v
            out[..., 1:, :] += v[..., :-1, :] / self.dy ** 2
            out[..., :-1, :] += v[..., 1:, :] / self.dy ** 2
        return out

    @property
    def lap_diag(self):
        d = -2.0 / self.dx ** 2
        if self.dim == 2:
            d += -2.0 / self.dy ** 2
        return d

    # k(w) = k0 (1 + k1 w) and its Kirchhoff transform Phi, Phi' = k
    def phi(self, w):
        return self.k0 * (w + 0.5 * self.k1 * w * w)

    def dphi(self, w):
        return self.k0 * (1.0 + self.k1 * w)

    @property
    def d2phi(self):
        return self.k0 * self.k1

    def B(self, u):
        """b0 B u: u[..., a] * b0 added to actuator cell a (repeated cells add)."""
        w = np.zeros(u.shape[:-1] + (self.ng,))
        for a in range(self.nu):
            w[..., self.act[a]] += self.b0 * u[..., a]
        return w.reshape(u.shape[:-1] + self.shape)

    def BT(self, y):
        """(b0 B)^T y: b0 times y at each actuator cell."""
        return self.b0 * y.reshape(y.shape[:-2] + (self.ng,))[..., self.act]

    def f(self, x, u):
        """f(u, x) = Lap Phi(x) + b0 B u (eq. 5 with the first-order model)."""
        return self.lap(self.phi(x)) + self.B(u)

    def cold_start(self):
        """S^0: x_i = x0, u_i = 0, lambda_i = 0 (no bounds, so it is feasible)."""
        X = np.broadcast_to(self.x0, (self.N,) + self.shape).copy()
        return X, np.zeros((self.N, self.nu)), np.zeros((self.N,) + self.shape)


# ---------------------------------------------------------------------------
# KKT map, Sec. 3.2, eq. 9
# ---------------------------------------------------------------------------
def kkt(p: Problem, X, U, Lam, u_tilde=None):
    """K_i(x_{i-1}, s_i, lambda_{i+1}) for every stage i.

    Returns (K1, K2, K3): state-equation rows (N, my, mx), u rows (N, nu) and
    costate rows (N, my, mx).  With ``u_tilde`` None, u~ = u^k and the
    regularization term is zero.
    """
    h = p.h
    Xprev = np.concatenate([p.x0[None], X[:-1]], axis=0)          # x_0 = x0bar
    lam_next = np.concatenate([Lam[1:], (h * p.qf * (X[-1] - p.ref))[None]], axis=0)
    mu = p.lap(Lam)                       # Lap^T lambda (Lap is symmetric)
    K1 = Xprev - X + h * p.f(X, U)
    grad_x_H = p.q * (X - p.ref) + p.dphi(X) * mu     # grad_x l + (grad_x f)^T lambda
    K3 = lam_next - Lam + h * grad_x_H
    grad_u_H = p.r * U + p.BT(Lam)                    # grad_u l + (grad_u f)^T lambda
    K2 = h * grad_u_H
    if u_tilde is not None:
        K2 = K2 + p.gamma * (U - u_tilde)
    return K1, K2, K3


def kkt_norms(K1, K2, K3):
    """(||K||_inf, ||K||_2) over all stacked rows (stopping test, Table 2)."""
    allk = np.concatenate([np.abs(K1).ravel(), np.abs(K2).ravel(), np.abs(K3).ravel()])
    return float(allk.max()), float(np.sqrt(np.sum(allk * allk)))


# ---------------------------------------------------------------------------
# Lower layer, Sec. 4.3 (eqs. 21-24) and the u-iteration of Sec. 5.2
# ---------------------------------------------------------------------------
class StageCoeffs:
    """Blocks of the reordered stage matrix (eq. 21) at iterate k, all stages.

    F_x  = h grad_x f - I = h Lap diag(Phi'(x)) - I
    F_u  = h grad_u f     = h b0 B
    A_xx = h grad_xx H (+ h qf I at stage N) = h (q + Phi'' Lap lambda) [+ h qf]
    A_uu = h grad_uu H + gamma I             = h r + gamma
    A_xu = A_ux = 0 (f is affine in u and l has no cross term).
    """

    def __init__(self, p: Problem, X, U, Lam):
        h = p.h
        self.p = p
        self.dphi = p.dphi(X)
        self.diag = h * p.lap_diag * self.dphi - 1.0     # diagonal of F_x and F_x^T
        axx = h * (p.q + p.d2phi * p.lap(Lam))
        axx[-1] += h * p.qf
        self.axx = axx
        self.auu = h * p.r + p.gamma

    def Fx_offdiag(self, v):
        """(F_x - diag F_x) v = h (Lap - diag Lap)(Phi' v)."""
        p = self.p
        return p.h * (p.lap(self.dphi * v) - p.lap_diag * self.dphi * v)

    def FxT_offdiag(self, v):
        """(F_x^T - diag F_x^T) v = h Phi' (Lap - diag Lap) v."""
        p = self.p
        return p.h * self.dphi * (p.lap(v) - p.lap_diag * v)

    def Fu(self, v3):
        return self.p.h * self.p.B(v3)

    def FuT(self, y):
        return self.p.h * self.p.BT(y)


def jacobi_solve(diag, offdiag, b, n_sweeps):
    """Pointwise Jacobi (Lemma 1): v <- D^{-1}(b - (L+U) v), n_sweeps from v=0."""
    v = np.zeros_like(b)
    for _ in range(n_sweeps):
        v = (b - offdiag(v)) / diag
    return v


def apply_P_inv(c: StageCoeffs, b4, b5, n_lo):
    """Approximate solve of [[0, F_x], [F_x^T, A_xx]] [v4; v5] = [b4; b5] (eq. 24):
    F_x v5 = b4, then F_x^T v4 = b5 - A_xx v5, each by n_lo Jacobi sweeps."""
    v5 = jacobi_solve(c.diag, c.Fx_offdiag, b4, n_lo)
    v4 = jacobi_solve(c.diag, c.FxT_offdiag, b5 - c.axx * v5, n_lo)
    return v4, v5


def lower_layer(c: StageCoeffs, b1, b2, b3, n_lo=2, n_u_it=2):
    """Approximate (Delta lambda, Delta x, Delta u) = D_i^{-1} K_i for all stages.

    b1, b2, b3: state-equation, costate and u rows of K (right-hand side of the
    reordered system, eq. 22).  Eq. 23a is solved by the u fixed-point
    iteration of Sec. 5.2 (n_u_it steps from v3 = 0), eq. 23b by one more
    P^{-1} application.
    """
    v3 = np.zeros_like(b3)
    for _ in range(n_u_it):
        # y = P^{-1}([F_u; A_xu] v3 - [b1; b2]), A_xu = 0
        y_lam, _y_x = apply_P_inv(c, c.Fu(v3) - b1, -b2, n_lo)
        # A_uu v3 = b3 + [F_u^T A_ux] y, A_ux = 0
        v3 = (b3 + c.FuT(y_lam)) / c.auu
    v1, v2 = apply_P_inv(c, b1 - c.Fu(v3), b2, n_lo)
    return v1, v2, v3


# ---------------------------------------------------------------------------
# Dense stage blocks (tiny instances), ordering s = (x, u, lambda) as in eq. 17
# ---------------------------------------------------------------------------
def lap_matrix(p: Problem):
    """Dense Laplacian (ng x ng) built column by column from ``lap``."""
    e = np.eye(p.ng).reshape((p.ng,) + p.shape)
    return p.lap(e).reshape(p.ng, p.ng).T


def b_matrix(p: Problem):
    Bm = np.zeros((p.ng, p.nu))
    for a in range(p.nu):
        Bm[p.act[a], a] += p.b0
    return Bm


def pack(p: Problem, X, U, Lam):
    return np.concatenate([np.concatenate([X[i].ravel(), U[i], Lam[i].ravel()])
                           for i in range(p.N)])


def unpack(p: Problem, S):
    n = 2 * p.ng + p.nu
    X, U, L = p.cold_start()
    for i in range(p.N):
        s = S[i * n:(i + 1) * n]
        X[i] = s[:p.ng].reshape(p.shape)
        U[i] = s[p.ng:p.ng + p.nu]
        L[i] = s[p.ng + p.nu:].reshape(p.shape)
    return X, U, L


def pack_kkt(p: Problem, K1, K2, K3):
    return np.concatenate([np.concatenate([K1[i].ravel(), K2[i], K3[i].ravel()])
                           for i in range(p.N)])


def dense_stage_blocks(p: Problem, X, U, Lam, with_gamma=True):
    """D_i = grad_{s_i} K_i (eq. 17), rows (K1, K2, K3).  With ``with_gamma``
    the u-block holds h r + gamma (the matrix of the upper-layer iteration,
    u~ frozen); without it, the exact Jacobian of K with u~ = u (Newton)."""
    Lm = lap_matrix(p)
    Bm = b_matrix(p)
    h, ng, nu = p.h, p.ng, p.nu
    blocks = []
    for i in range(p.N):
        x = X[i].ravel()
        mu = Lm @ Lam[i].ravel()
        fx = Lm * p.dphi(x)[None, :]
        Hxx = np.diag(p.q + p.d2phi * mu)
        D = np.zeros((2 * ng + nu, 2 * ng + nu))
        D[:ng, :ng] = h * fx - np.eye(ng)
        D[:ng, ng:ng + nu] = h * Bm
        D[ng:ng + nu, ng:ng + nu] = (h * p.r + (p.gamma if with_gamma else 0.0)) * np.eye(nu)
        D[ng:ng + nu, ng + nu:] = h * Bm.T
        D[ng + nu:, :ng] = h * Hxx + (h * p.qf * np.eye(ng) if i == p.N - 1 else 0.0)
        D[ng + nu:, ng + nu:] = h * fx.T - np.eye(ng)
        blocks.append(D)
    return blocks


def coupling_blocks(p: Problem):
    """M_L (state row, x column) and M_U (costate row, lambda column), eq. 10."""
    n = 2 * p.ng + p.nu
    ML = np.zeros((n, n)); ML[:p.ng, :p.ng] = np.eye(p.ng)
    MU = np.zeros((n, n)); MU[p.ng + p.nu:, p.ng + p.nu:] = np.eye(p.ng)
    return ML, MU


def dense_kkt_matrix(p: Problem, X, U, Lam, with_gamma=False):
    """The whole block-tridiagonal KKT matrix of eq. 10."""
    D = dense_stage_blocks(p, X, U, Lam, with_gamma)
    ML, MU = coupling_blocks(p)
    n = D[0].shape[0]
    A = np.zeros((p.N * n, p.N * n))
    for i in range(p.N):
        A[i * n:(i + 1) * n, i * n:(i + 1) * n] = D[i]
        if i > 0:
            A[i * n:(i + 1) * n, (i - 1) * n:i * n] = ML
        if i < p.N - 1:
            A[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = MU
    return A


def block_elimination_solve(D, ML, MU, K):
    """Solve the block-tridiagonal system of eq. 10 by the backward recursion
    D^_i = D_i - M_U D^_{i+1}^{-1} M_L (Sec. 3.3) and a forward sweep."""
    N = len(D)
    n = D[0].shape[0]
    Kb = [K[i * n:(i + 1) * n] for i in range(N)]
    Dh, rh = [None] * N, [None] * N
    Dh[N - 1], rh[N - 1] = D[N - 1], Kb[N - 1]
    for i in range(N - 2, -1, -1):
        Dh[i] = D[i] - MU @ np.linalg.solve(Dh[i + 1], ML)
        rh[i] = Kb[i] - MU @ np.linalg.solve(Dh[i + 1], rh[i + 1])
    ds = [np.linalg.solve(Dh[0], rh[0])]
    for i in range(1, N):
        ds.append(np.linalg.solve(Dh[i], rh[i] - ML @ ds[i - 1]))
    return np.concatenate(ds)


def newton_step(p: Problem, X, U, Lam, use_dense_lu=False):
    """One Newton step S <- S - (grad K)^{-1} K (Sec. 3.3, alpha = 1), with the
    exact Jacobian (u~ = u, so the regularization term drops out)."""
    K = pack_kkt(p, *kkt(p, X, U, Lam))
    if use_dense_lu:
        dS = np.linalg.solve(dense_kkt_matrix(p, X, U, Lam, with_gamma=False), K)
    else:
        ML, MU = coupling_blocks(p)
        dS = block_elimination_solve(dense_stage_blocks(p, X, U, Lam, with_gamma=False),
                                     ML, MU, K)
    return unpack(p, pack(p, X, U, Lam) - dS)


def newton_solve(p: Problem, S0=None, tol=1e-14, max_iter=30, use_dense_lu=False):
    """Newton on K(S) = 0 from S0 (cold start by default); returns (S, history)."""
    X, U, L = p.cold_start() if S0 is None else (a.copy() for a in S0)
    hist = []
    for _ in range(max_iter):
        r = kkt_norms(*kkt(p, X, U, L))[0]
        hist.append(r)
        if r <= tol:
            break
        X, U, L = newton_step(p, X, U, L, use_dense_lu)
    return (X, U, L), hist


# ---------------------------------------------------------------------------
# Upper layer, Sec. 4.2, eq. 15
# ---------------------------------------------------------------------------
def jacobi_iteration(p: Problem, X, U, Lam, n_lo=2, n_u_it=2, alpha=1.0, exact_inner=False,
                     u_tilde=None):
    """One double-layer Jacobi iteration S^{k+1} = S^k - alpha (D^k)^{-1} K^k.

    Every stage uses x_{i-1} and lambda_{i+1} of iterate k only, so all stages
    update at once.  With ``exact_inner`` each stage system is solved by a
    dense LU instead of the lower layer.  ``u_tilde`` None means u~ = u^k
    (Remark 1); an array fixes the regularization reference.  Returns
    (X, U, Lam) of iterate k+1 and (||K^k||_inf, ||K^k||_2) of the KKT map
    without the regularization term.
    """
    K1, K2, K3 = kkt(p, X, U, Lam)
    if u_tilde is not None:
        K2 = K2 + p.gamma * (U - u_tilde)
    norms = kkt_norms(K1, K2, K3)
    if exact_inner:
        D = dense_stage_blocks(p, X, U, Lam)
        n = 2 * p.ng + p.nu
        Kp = pack_kkt(p, K1, K2, K3)
        dS = np.concatenate([np.linalg.solve(D[i], Kp[i * n:(i + 1) * n]) for i in range(p.N)])
        dX, dU, dL = unpack(p, dS)
        return X - alpha * dX, U - alpha * dU, Lam - alpha * dL, norms
    c = StageCoeffs(p, X, U, Lam)
    v1, v2, v3 = lower_layer(c, K1, K3, K2, n_lo=n_lo, n_u_it=n_u_it)
    return X - alpha * v2, U - alpha * v3, Lam - alpha * v1, norms


def solve_jacobi(p: Problem, S0=None, tol=1e-6, max_iter=10000, n_lo=2, n_u_it=2,
                 alpha=1.0, exact_inner=False, record=False, u_tilde=None):
    """Iterate eq. 15 until ||K^k||_inf <= tol (Table 2's stopping rule).

    Returns ((X, U, Lam), info); the iterate returned is the first whose
    residual passed (or the last one).  info: iters, res_inf, res_2,
    converged, diverged, hist.
    """
    X, U, L = p.cold_start() if S0 is None else (a.copy() for a in S0)
    hist = []
    for k in range(max_iter + 1):
        r_inf, r_2 = kkt_norms(*kkt(p, X, U, L))
        if record:
            hist.append(r_inf)
        done = (not np.isfinite(r_inf)) or r_inf <= tol or k == max_iter
        if done:
            return (X, U, L), dict(iters=k, res_inf=r_inf, res_2=r_2,
                                   converged=bool(r_inf <= tol),
                                   diverged=not np.isfinite(r_inf), hist=hist)
        X, U, L, _ = jacobi_iteration(p, X, U, L, n_lo, n_u_it, alpha, exact_inner, u_tilde)


# ---------------------------------------------------------------------------
# Jacobi-type variants, Sec. 4.2 (eqs. 18-20)
# ---------------------------------------------------------------------------
def _stage_view(c: StageCoeffs, i: int) -> StageCoeffs:
    """The coefficients of stage i alone (arrays keep a leading axis of 1)."""
    v = object.__new__(StageCoeffs)
    v.p = c.p
    v.dphi = c.dphi[i:i + 1]
    v.diag = c.diag[i:i + 1]
    v.axx = c.axx[i:i + 1]
    v.auu = c.auu
    return v


def stage_solver(p: Problem, X, U, Lam, n_lo=2, n_u_it=2, exact_inner=False):
    """solve(i, b1, b2, b3) -> (dx, du, dlam): the approximate (D_i^k)^{-1}
    of the lower layer (or, with ``exact_inner``, a dense solve of D_i^k)
    applied to state rows b1, costate rows b2 and u rows b3 of stage i."""
    if exact_inner:
        D = dense_stage_blocks(p, X, U, Lam)
        ng, nu = p.ng, p.nu

        def solve(i, b1, b2, b3):
            d = np.linalg.solve(D[i], np.concatenate([b1.ravel(), b3, b2.ravel()]))
            return (d[:ng].reshape(p.shape), d[ng:ng + nu], d[ng + nu:].reshape(p.shape))
        return solve
    c = StageCoeffs(p, X, U, Lam)

    def solve(i, b1, b2, b3):
        v1, v2, v3 = lower_layer(_stage_view(c, i), b1[None], b2[None], b3[None], n_lo, n_u_it)
        return v2[0], v3[0], v1[0]
    return solve


def gs_order(N: int, kind: str):
    """Stage visiting order (0-based) of a block Gauss-Seidel sweep: forward
    (FGS, eq. 18), backward (BGS) or red-black (even stages, then odd)."""
    if kind == "forward":
        return list(range(N))
    if kind == "backward":
        return list(range(N - 1, -1, -1))
    if kind == "redblack":
        return list(range(0, N, 2)) + list(range(1, N, 2))
    raise ValueError(kind)


def gauss_seidel_iteration(p: Problem, X, U, Lam, order, n_lo=2, n_u_it=2, alpha=1.0,
                           exact_inner=False, u_tilde=None):
    """S^{k+1} = S^k - alpha (D^k + L_o)^{-1} K^k: block Gauss-Seidel on the
    KKT system of eq. 10 with the stages visited in ``order``; L_o holds the
    coupling blocks to stages visited earlier.  Forward order is FGS (eq. 18,
    L_o = L), backward order BGS (D^k + U).  Visiting stage i solves D_i^k
    Delta s_i = K_i^k - (M_L Delta s_{i-1} if i-1 was visited) - (M_U
    Delta s_{i+1} if i+1 was visited): M_L takes Delta x_{i-1} into the state
    rows, M_U Delta lambda_{i+1} into the costate rows.  D^k and K^k are those
    of iterate k throughout.  Returns (X, U, Lam) and the norms of K^k."""
    K1, K2, K3 = kkt(p, X, U, Lam)
    if u_tilde is not None:
        K2 = K2 + p.gamma * (U - u_tilde)
    norms = kkt_norms(*kkt(p, X, U, Lam))
    solve = stage_solver(p, X, U, Lam, n_lo, n_u_it, exact_inner)
    dX, dU, dL = np.zeros_like(X), np.zeros_like(U), np.zeros_like(Lam)
    seen = np.zeros(p.N, dtype=bool)
    for i in order:
        b1, b2 = K1[i].copy(), K3[i].copy()
        if i > 0 and seen[i - 1]:
            b1 = b1 - dX[i - 1]
        if i < p.N - 1 and seen[i + 1]:
            b2 = b2 - dL[i + 1]
        dX[i], dU[i], dL[i] = solve(i, b1, b2, K2[i])
        seen[i] = True
    return X - alpha * dX, U - alpha * dU, Lam - alpha * dL, norms


def sgs_iteration(p: Problem, X, U, Lam, n_lo=2, n_u_it=2, alpha=1.0, exact_inner=False,
                  u_tilde=None):
    """Symmetric Gauss-Seidel, eq. 20: S^{k+1} = S^k - alpha (D^k + L)^{-1}
    (K^k - U (D^k + U)^{-1} K^k): a backward sweep z = (D^k + U)^{-1} K^k,
    then a forward sweep on K^k - U z, whose costate rows of stage i lose
    z_lambda of stage i+1."""
    K1, K2, K3 = kkt(p, X, U, Lam)
    if u_tilde is not None:
        K2 = K2 + p.gamma * (U - u_tilde)
    norms = kkt_norms(*kkt(p, X, U, Lam))
    solve = stage_solver(p, X, U, Lam, n_lo, n_u_it, exact_inner)
    N = p.N
    zL = np.zeros_like(Lam)
    for i in range(N - 1, -1, -1):
        b2 = K3[i] - zL[i + 1] if i < N - 1 else K3[i]
        _, _, zL[i] = solve(i, K1[i], b2, K2[i])
    dX, dU, dL = np.zeros_like(X), np.zeros_like(U), np.zeros_like(Lam)
    for i in range(N):
        b1 = K1[i] - dX[i - 1] if i > 0 else K1[i]
        b2 = K3[i] - zL[i + 1] if i < N - 1 else K3[i]
        dX[i], dU[i], dL[i] = solve(i, b1, b2, K2[i])
    return X - alpha * dX, U - alpha * dU, Lam - alpha * dL, norms


def variant_iteration(p: Problem, X, U, Lam, variant="jacobi", **kw):
    """One iteration of an upper-layer variant: jacobi (eq. 15), fgs (eq. 18),
    bgs, sgs (eq. 20) or redblack."""
    if variant == "jacobi":
        return jacobi_iteration(p, X, U, Lam, **kw)
    if variant == "sgs":
        return sgs_iteration(p, X, U, Lam, **kw)
    kind = {"fgs": "forward", "bgs": "backward", "redblack": "redblack"}[variant]
    return gauss_seidel_iteration(p, X, U, Lam, gs_order(p.N, kind), **kw)


def solve_variant(p: Problem, variant="jacobi", S0=None, tol=1e-6, max_iter=10000, **kw):
    """Iterate a variant until ||K^k||_inf <= tol (as solve_jacobi)."""
    X, U, L = p.cold_start() if S0 is None else (a.copy() for a in S0)
    for k in range(max_iter + 1):
        r_inf, r_2 = kkt_norms(*kkt(p, X, U, L))
        if (not np.isfinite(r_inf)) or r_inf <= tol or k == max_iter:
            return (X, U, L), dict(iters=k, res_inf=r_inf, res_2=r_2,
                                   converged=bool(r_inf <= tol), diverged=not np.isfinite(r_inf))
        X, U, L, _ = variant_iteration(p, X, U, L, variant, **kw)


# ---------------------------------------------------------------------------
# Linear case k1 = 0: discrete LQ by the Riccati recursion (textbook closed form)
# ---------------------------------------------------------------------------
def riccati_lq(p: Problem):
    """Optimal controls for k1 = 0.  Dynamics x_i = Ab x_{i-1} + Bb u_i with
    Ab = (I - h k0 Lap)^{-1}, Bb = Ab h b0 B; cost
    sum_i h/2 (q |x_i - ref|^2 + r |u_i|^2) + h/2 qf |x_N - ref|^2.
    Value function after stage i: V_i(x) = 1/2 x'P_i x + p_i'x.  Returns U."""
    assert p.k1 == 0.0
    ng = p.ng
    A = p.k0 * lap_matrix(p)
    Bm = b_matrix(p)
    Ab = np.linalg.inv(np.eye(ng) - p.h * A)
    Bb = Ab @ (p.h * Bm)
    xr = p.ref.ravel()
    Q = p.q * np.eye(ng)
    R = p.r * np.eye(p.nu)
    P = p.h * p.qf * np.eye(ng)
    pv = -p.h * p.qf * xr
    gains = []
    for _ in range(p.N):
        Pt = P + p.h * Q                  # stage-i tracking cost folded into V
        pt = pv - p.h * (Q @ xr)
        Huu = Bb.T @ Pt @ Bb + p.h * R
        Kg = -np.linalg.solve(Huu, Bb.T @ Pt @ Ab)
        kg = -np.linalg.solve(Huu, Bb.T @ pt)
        gains.append((Kg, kg))
        Acl = Ab + Bb @ Kg
        P = Acl.T @ Pt @ Acl + p.h * Kg.T @ R @ Kg
        pv = Acl.T @ (Pt @ (Bb @ kg) + pt) + p.h * Kg.T @ R @ kg
        P = 0.5 * (P + P.T)
    gains.reverse()
    x = p.x0.ravel().copy()
    U = np.zeros((p.N, p.nu))
    for i in range(p.N):
        Kg, kg = gains[i]
        U[i] = Kg @ x + kg
        x = Ab @ x + Bb @ U[i]
    return U


# ---------------------------------------------------------------------------
# Direct evaluation of the NLP (eq. 6) for brute-force checks
# ---------------------------------------------------------------------------
def simulate_backward_euler(p: Problem, U, newton_tol=1e-15):
    """States of x_i = x_{i-1} + h f(u_i, x_i); each stage by Newton on x alone."""
    Lm = lap_matrix(p)
    Bm = b_matrix(p)
    x = p.x0.ravel().copy()
    X = np.zeros((p.N, p.ng))
    for i in range(p.N):
        xp = x.copy()
        for _ in range(60):
            res = xp - x + p.h * (Lm @ p.phi(x) + Bm @ U[i])
            J = p.h * Lm * p.dphi(x)[None, :] - np.eye(p.ng)
            dx = np.linalg.solve(J, res)
            x = x - dx
            if np.max(np.abs(dx)) < newton_tol:
                break
        X[i] = x
    return X


def nlp_cost(p: Problem, U):
    """Objective of eq. 6 (with the terminal term) at controls U."""
    X = simulate_backward_euler(p, U)
    xr = p.ref.ravel()
    J = sum(p.h * 0.5 * (p.q * np.sum((X[i] - xr) ** 2) + p.r * np.sum(U[i] ** 2))
            for i in range(p.N))
    return J + p.h * 0.5 * p.qf * np.sum((X[-1] - xr) ** 2)


def lagrangian(p: Problem, X, U, Lam):
    """Cost of eq. 6 plus sum_i lambda_i^T (x_{i-1} - x_i + h f(u_i, x_i))."""
    xr = p.ref
    val = 0.0
    xprev = p.x0
    for i in range(p.N):
        val += p.h * 0.5 * (p.q * np.sum((X[i] - xr) ** 2) + p.r * np.sum(U[i] ** 2))
        val += np.sum(Lam[i] * (xprev - X[i] + p.h * p.f(X[i], U[i])))
        xprev = X[i]
    return val + p.h * 0.5 * p.qf * np.sum((X[-1] - xr) ** 2)


# ---------------------------------------------------------------------------
# Closed loop (Sec. 5.3): receding horizon with an explicit-Euler plant
# ---------------------------------------------------------------------------
def plant_step(p: Problem, w, u1, dt, n_sub):
    """Advance the true system by dt with n_sub explicit-Euler sub-steps of the
    same finite-difference model under the first-stage controls u1."""
    w = np.array(w, dtype=np.float64, copy=True).reshape(p.shape)
    for _ in range(n_sub):
        w = w + (dt / n_sub) * p.f(w, np.asarray(u1, dtype=np.float64))
    return w


def closed_loop(inst, steps, n_sub, tol=1e-10, max_iter=20000):
    """Each step: solve the NMPC problem from the measured plant state (cold
    start, so the result does not depend on warm-start choices), apply u_1 for
    one stage length h, advance the plant.  Returns (U1 [steps, nu],
    W [steps + 1, ng], iterations per step)."""
    import copy
    cur = copy.copy(inst)
    w = np.asarray(inst.x0, dtype=np.float64).copy()
    U1, W, its = [], [w.copy()], []
    for _ in range(steps):
        cur.x0 = w.copy()
        p = Problem(cur)
        (X, U, L), info = solve_jacobi(p, tol=tol, max_iter=max_iter)
        U1.append(U[0].copy())
        its.append(info["iters"])
        w = plant_step(p, w, U[0], p.h, n_sub).ravel()
        W.append(w.copy())
    return np.array(U1), np.array(W), its
