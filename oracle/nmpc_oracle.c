/*
 * Plain C FP64 oracle of the double-layer Jacobi method (Deng & Ohtsuka).
 *
 * TEST INFRASTRUCTURE ONLY.  It is the same computation as oracle/nmpc.py,
 * written as scalar loops so that complete solves of the large 2D workload
 * (256 x 256 cells, N = 100 stages) finish on the host in seconds instead of
 * minutes; tests pin it element by element against oracle/nmpc.py, which
 * the paper's mathematics pins.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU legs load it; it shares no code with the CUDA path.  The
 * one parallel construct is a loop over the stages of an iteration, which
 * the upper-layer Jacobi method (eq. 15) makes independent; every stage's
 * arithmetic is sequential and in float64.
 *
 * What is computed (the notation of oracle/nmpc.py):
 *   model  (Sec. 2, eqs. 1, 4): f(u, x) = Lap Phi(x) + b0 B u, Phi(w) =
 *          k0 (w + k1 w^2 / 2), 3-/5-point Laplacian with a zero ring;
 *   KKT    (Sec. 3.2, eq. 9), every cost term scaled by h, lambda_{N+1} =
 *          h qf (x_N - ref), u~ = u^k (Remark 1);
 *   upper  (Sec. 4.2, eq. 15): S <- S - alpha D^{-1} K, all stages from k;
 *   lower  (Sec. 4.3, eqs. 21-24 and the u-iteration of Sec. 5.2): n_u_it
 *          steps v3 <- (b3 + F_u^T y_lam) / A_uu with (y_lam, y_x) =
 *          P^{-1}(F_u v3 - b1, -b2) from v3 = 0, then (v1, v2) =
 *          P^{-1}(b1 - F_u v3, b2); P^{-1}(b4, b5) solves F_x v5 = b4, then
 *          F_x^T v4 = b5 - A_xx v5, each by n_lo pointwise Jacobi sweeps
 *          from zero (Lemma 1);
 *   stop   (Table 2): ||K(S^k)||_inf <= tol;
 *   plant  (Sec. 5.3's closed loop): explicit-Euler sub-steps of the same
 *          finite-difference model.
 * Arrays: x, lam [N][my][mx], u [N][nu], row-major.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int dim, mx, my, N, nu;
  const int* act;  /* [nu] flat cell indices */
  double h, q, r, qf, gamma, k0, k1, b0;
  const double* x0;  /* [ng] */
  const double* ref; /* [ng] */
} orc_problem;

typedef struct {
  double res_inf, res_2;
  int iters, converged, diverged;
} orc_info;

static double cx_of(const orc_problem* p) { double d = 1.0 / (p->mx + 1); return 1.0 / (d * d); }
static double cy_of(const orc_problem* p) {
  if (p->dim != 2) return 0.0;
  double d = 1.0 / (p->my + 1);
  return 1.0 / (d * d);
}

/* eq. 4: out = Lap v on one stage grid (zero values outside the interior) */
static void lap(const orc_problem* p, const double* v, double* out) {
  const int mx = p->mx, my = p->my;
  const double cx = cx_of(p), cy = cy_of(p);
  for (int iy = 0; iy < my; ++iy)
    for (int ix = 0; ix < mx; ++ix) {
      const int c = iy * mx + ix;
      double s = -2.0 * cx * v[c];
      if (ix > 0) s += cx * v[c - 1];
      if (ix < mx - 1) s += cx * v[c + 1];
      if (p->dim == 2) {
        s += -2.0 * cy * v[c];
        if (iy > 0) s += cy * v[c - mx];
        if (iy < my - 1) s += cy * v[c + mx];
      }
      out[c] = s;
    }
}

static double lap_diag(const orc_problem* p) { return -2.0 * cx_of(p) - 2.0 * cy_of(p); }
static double phi(const orc_problem* p, double w) { return p->k0 * (w + 0.5 * p->k1 * w * w); }
static double dphi(const orc_problem* p, double w) { return p->k0 * (1.0 + p->k1 * w); }

/* per-stage work arrays */
typedef struct {
  double *t1, *t2, *dp, *dg, *axx, *b4, *b5, *v5, *v4, *vn, *ylam, *k1, *k3;
  double* v3;
  double* k2;
} orc_ws;

static int ws_alloc(orc_ws* w, int ng, int nu) {
  double* base = (double*)malloc(sizeof(double) * ((size_t)13 * ng + 2 * (size_t)nu));
  if (!base) return -1;
  double** f[13] = {&w->t1, &w->t2, &w->dp, &w->dg, &w->axx, &w->b4, &w->b5,
                    &w->v5, &w->v4, &w->vn, &w->ylam, &w->k1, &w->k3};
  for (int j = 0; j < 13; ++j) *f[j] = base + (size_t)j * ng;
  w->v3 = base + (size_t)13 * ng;
  w->k2 = w->v3 + nu;
  return 0;
}

static void ws_free(orc_ws* w) { free(w->t1); }

/* K_i of eq. 9 for stage i (0-based) of (X, U, L): state rows k1, u rows k2,
   costate rows k3. */
static void kkt_stage(const orc_problem* p, const double* X, const double* U, const double* L,
                      int i, orc_ws* w, double* k1, double* k2, double* k3) {
  const int ng = p->mx * p->my, nu = p->nu, N = p->N;
  const double h = p->h;
  const double* x = X + (size_t)i * ng;
  const double* lm = L + (size_t)i * ng;
  const double* u = U + (size_t)i * nu;
  const double* xprev = (i == 0) ? p->x0 : X + (size_t)(i - 1) * ng;
  /* f = Lap Phi(x) + b0 B u */
  for (int c = 0; c < ng; ++c) w->t1[c] = phi(p, x[c]);
  lap(p, w->t1, w->t2);
  for (int a = 0; a < nu; ++a) w->t2[p->act[a]] += p->b0 * u[a];
  for (int c = 0; c < ng; ++c) k1[c] = xprev[c] - x[c] + h * w->t2[c];
  /* mu = Lap^T lambda (Lap is symmetric) */
  lap(p, lm, w->t1);
  for (int c = 0; c < ng; ++c) {
    const double lam_next = (i == N - 1) ? h * p->qf * (x[c] - p->ref[c])
                                         : L[(size_t)(i + 1) * ng + c];
    k3[c] = lam_next - lm[c] + h * (p->q * (x[c] - p->ref[c]) + dphi(p, x[c]) * w->t1[c]);
  }
  for (int a = 0; a < nu; ++a) k2[a] = h * (p->r * u[a] + p->b0 * lm[p->act[a]]);
}

/* (F_x - diag F_x) v = h (Lap - diag Lap)(Phi' v) */
static void fx_off(const orc_problem* p, const orc_ws* w, const double* v, double* out,
                   double* tmp) {
  const int ng = p->mx * p->my;
  const double ld = lap_diag(p);
  for (int c = 0; c < ng; ++c) tmp[c] = w->dp[c] * v[c];
  lap(p, tmp, out);
  for (int c = 0; c < ng; ++c) out[c] = p->h * (out[c] - ld * tmp[c]);
}

/* (F_x^T - diag F_x^T) v = h Phi' (Lap - diag Lap) v */
static void fxt_off(const orc_problem* p, const orc_ws* w, const double* v, double* out) {
  const int ng = p->mx * p->my;
  const double ld = lap_diag(p);
  lap(p, v, out);
  for (int c = 0; c < ng; ++c) out[c] = p->h * w->dp[c] * (out[c] - ld * v[c]);
}

/* Lemma 1: v <- D^{-1}(b - (L + U) v), n sweeps from v = 0; result in v */
static void jacobi_fx(const orc_problem* p, orc_ws* w, const double* b, double* v, int n,
                      int transposed) {
  const int ng = p->mx * p->my;
  memset(v, 0, sizeof(double) * ng);
  for (int s = 0; s < n; ++s) {
    if (transposed) fxt_off(p, w, v, w->vn);
    else fx_off(p, w, v, w->vn, w->t2);
    for (int c = 0; c < ng; ++c) v[c] = (b[c] - w->vn[c]) / w->dg[c];
  }
}

/* eq. 24: F_x v5 = b4, then F_x^T v4 = b5 - A_xx v5 (b5 is overwritten) */
static void apply_p_inv(const orc_problem* p, orc_ws* w, double* b4, double* b5, int n_lo,
                        double* v4, double* v5) {
  const int ng = p->mx * p->my;
  jacobi_fx(p, w, b4, v5, n_lo, 0);
  for (int c = 0; c < ng; ++c) b5[c] = b5[c] - w->axx[c] * v5[c];
  jacobi_fx(p, w, b5, v4, n_lo, 1);
}

/* One stage of one upper-layer iteration: Delta s_i by the lower layer from
   K_i (k1, k2, k3 in w), written as S_i - alpha Delta s_i into (Xo, Uo, Lo). */
static void lower_layer_stage(const orc_problem* p, const double* X, const double* U,
                              const double* L, int i, int n_lo, int n_u_it, double alpha,
                              orc_ws* w, double* Xo, double* Uo, double* Lo) {
  const int ng = p->mx * p->my, nu = p->nu, N = p->N;
  const double h = p->h;
  const double* x = X + (size_t)i * ng;
  const double* lm = L + (size_t)i * ng;
  /* stage coefficients (eq. 21 blocks) */
  lap(p, lm, w->t1);
  for (int c = 0; c < ng; ++c) {
    w->dp[c] = dphi(p, x[c]);
    w->dg[c] = h * lap_diag(p) * w->dp[c] - 1.0;
    w->axx[c] = h * (p->q + p->k0 * p->k1 * w->t1[c]) + ((i == N - 1) ? h * p->qf : 0.0);
  }
  const double auu = h * p->r + p->gamma;
  /* u fixed-point iteration (Sec. 5.2), from v3 = 0 */
  for (int a = 0; a < nu; ++a) w->v3[a] = 0.0;
  for (int it = 0; it < n_u_it; ++it) {
    for (int c = 0; c < ng; ++c) {
      w->b4[c] = -w->k1[c];
      w->b5[c] = -w->k3[c];
    }
    for (int a = 0; a < nu; ++a) w->b4[p->act[a]] += h * p->b0 * w->v3[a];
    apply_p_inv(p, w, w->b4, w->b5, n_lo, w->ylam, w->v5);
    for (int a = 0; a < nu; ++a) w->v3[a] = (w->k2[a] + h * p->b0 * w->ylam[p->act[a]]) / auu;
  }
  /* eq. 23b: (v1, v2) = P^{-1}(b1 - F_u v3, b2) */
  for (int c = 0; c < ng; ++c) {
    w->b4[c] = w->k1[c];
    w->b5[c] = w->k3[c];
  }
  for (int a = 0; a < nu; ++a) w->b4[p->act[a]] -= h * p->b0 * w->v3[a];
  apply_p_inv(p, w, w->b4, w->b5, n_lo, w->v4, w->v5);
  /* eq. 15 update */
  for (int c = 0; c < ng; ++c) {
    Xo[(size_t)i * ng + c] = x[c] - alpha * w->v5[c];
    Lo[(size_t)i * ng + c] = lm[c] - alpha * w->v4[c];
  }
  for (int a = 0; a < nu; ++a) Uo[(size_t)i * nu + a] = U[(size_t)i * nu + a] - alpha * w->v3[a];
}

/* Norms of K(S) (over every stacked row) and, unless resid_only, one
   upper-layer iteration S -> (Xo, Uo, Lo).  NaN propagates into res_inf. */
static int iterate(const orc_problem* p, const double* X, const double* U, const double* L,
                   int n_lo, int n_u_it, double alpha, int resid_only, double* Xo, double* Uo,
                   double* Lo, double* res_inf, double* res_2) {
  const int ng = p->mx * p->my, nu = p->nu, N = p->N;
  double* smax = (double*)malloc(sizeof(double) * 2 * (size_t)N);
  if (!smax) return -1;
  double* ssq = smax + N;
  int fail = 0;
#pragma omp parallel
  {
    orc_ws w;
    const int ok = (ws_alloc(&w, ng, nu) == 0);
    if (!ok) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < N; ++i) {
      if (!ok) continue;
      kkt_stage(p, X, U, L, i, &w, w.k1, w.k2, w.k3);
      double m = 0.0, s = 0.0;
      int nan = 0;
      for (int c = 0; c < ng; ++c) {
        const double a = fabs(w.k1[c]), b = fabs(w.k3[c]);
        nan |= isnan(a) || isnan(b);
        m = fmax(m, fmax(a, b));
        s += a * a + b * b;
      }
      for (int j = 0; j < nu; ++j) {
        const double a = fabs(w.k2[j]);
        nan |= isnan(a);
        m = fmax(m, a);
        s += a * a;
      }
      smax[i] = nan ? NAN : m;
      ssq[i] = s;
      if (!resid_only) lower_layer_stage(p, X, U, L, i, n_lo, n_u_it, alpha, &w, Xo, Uo, Lo);
    }
    if (ok) ws_free(&w);
  }
  double m = 0.0, s = 0.0;
  int nan = 0;
  for (int i = 0; i < N; ++i) {
    nan |= isnan(smax[i]);
    m = fmax(m, smax[i]);
    s += ssq[i];
  }
  free(smax);
  *res_inf = nan ? NAN : m;
  *res_2 = sqrt(s);
  return fail ? -1 : 0;
}

/* ||K(S)||_inf and ||K(S)||_2 (eq. 9, u~ = u). */
int orc_kkt_norms(const orc_problem* p, const double* X, const double* U, const double* L,
                  double* out2) {
  return iterate(p, X, U, L, 1, 1, 1.0, 1, NULL, NULL, NULL, out2, out2 + 1);
}

/* One upper-layer iteration (eq. 15) from (X, U, L) into (Xo, Uo, Lo); out2:
   the norms of K at the input. */
int orc_jacobi_iteration(const orc_problem* p, const double* X, const double* U, const double* L,
                         int n_lo, int n_u_it, double alpha, double* Xo, double* Uo, double* Lo,
                         double* out2) {
  return iterate(p, X, U, L, n_lo, n_u_it, alpha, 0, Xo, Uo, Lo, out2, out2 + 1);
}

/* Iterate eq. 15 from the start held in (X, U, L) until ||K(S^k)||_inf <= tol
   (Table 2's stopping rule), a non-finite residual, or max_iter; the returned
   iterate S^k is left in (X, U, L). */
int orc_solve_jacobi(const orc_problem* p, double* X, double* U, double* L, double tol,
                     int max_iter, int n_lo, int n_u_it, double alpha, orc_info* info) {
  const size_t ns = (size_t)p->N * p->mx * p->my, nus = (size_t)p->N * p->nu;
  double* Xb = (double*)malloc(sizeof(double) * (2 * ns + nus));
  if (!Xb) return -1;
  double* Lb = Xb + ns;
  double* Ub = Lb + ns;
  int rc = 0;
  for (int k = 0;; ++k) {
    double r_inf = 0.0, r_2 = 0.0;
    const int done_max = (k == max_iter);
    rc = iterate(p, X, U, L, n_lo, n_u_it, alpha, done_max, Xb, Ub, Lb, &r_inf, &r_2);
    if (rc) break;
    const int bad = !isfinite(r_inf);
    if (bad || r_inf <= tol || done_max) {
      info->iters = k;
      info->res_inf = r_inf;
      info->res_2 = r_2;
      info->converged = (r_inf <= tol);
      info->diverged = bad;
      break;
    }
    memcpy(X, Xb, sizeof(double) * ns);
    memcpy(L, Lb, sizeof(double) * ns);
    memcpy(U, Ub, sizeof(double) * nus);
  }
  free(Xb);
  return rc;
}

/* Sec. 5.3's plant: w advances by dt in n_sub explicit-Euler sub-steps of the
   same model under the controls u1 (in place). */
int orc_plant_step(const orc_problem* p, double* w, const double* u1, double dt, int n_sub) {
  const int ng = p->mx * p->my;
  double* t1 = (double*)malloc(sizeof(double) * 2 * (size_t)ng);
  if (!t1) return -1;
  double* t2 = t1 + ng;
  for (int s = 0; s < n_sub; ++s) {
    for (int c = 0; c < ng; ++c) t1[c] = phi(p, w[c]);
    lap(p, t1, t2);
    for (int a = 0; a < p->nu; ++a) t2[p->act[a]] += p->b0 * u1[a];
    for (int c = 0; c < ng; ++c) w[c] = w[c] + (dt / n_sub) * t2[c];
  }
  free(t1);
  return 0;
}

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the stage loops use (set_threads <= 0: the runtime's default). */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
