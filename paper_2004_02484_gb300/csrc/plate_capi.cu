// Pinned-actuator solver (include/nmpc_plate.h): the double-layer method on
// the paper's own problem class, the heat plate of Sec. 5.1 whose actuator
// points have their temperatures set directly, with input bounds, the log
// barrier (eq. 8) and the fraction-to-the-boundary step (eq. 11).
//
// One iteration is two kernels (three with the red-black upper layer):
//   k_plate_dir  one CTA per (instance, stage) loads the stage's grid into
//     shared memory (w = x at the state points, u at the actuator points;
//     lambda at the state points, zero at the actuators), evaluates K_i
//     (eq. 9) and its norms, the stage's coefficients, and the lower layer
//     (eqs. 21-24 with the u-iteration of Sec. 5.2): n_lo pointwise Jacobi
//     sweeps on F_x and F_x^T over the state points.  It stores the
//     direction Delta s_i and the stage's largest admissible step under
//     eq. 11 (a per-instance atomic minimum).  Red-black: half 0 runs the
//     even stages; half 1 the odd ones, its right-hand side lowered by the
//     even neighbours' directions (M_L Delta x_{i-1}, M_U Delta lambda_{i+1};
//     the form of eq. 18).
//   k_plate_update  per (instance, stage): the convergence decision from
//     ||K(S^k)||_inf (the whole instance's maximum, complete once every
//     stage's k_plate_dir has run) and otherwise S^{k+1} = S^k - alpha_max
//     Delta S.
// The Laplacian of the grid, with the mirrored fictitious points of the
// zero-Neumann condition (eqs. 2-3) or the zero Dirichlet ring, and its
// transpose are host-built tables of five (column, weight) entries per
// point.  Everything is float64.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/nmpc_plate.h"

namespace plate_dev {

constexpr int ELL = 5;
constexpr int THREADS = 256;
constexpr int MAX_NU = 64;
enum { ST_RUNNING = 0, ST_CONVERGED = 1, ST_DIVERGED = 2, ST_MAX_ITER = 3 };
enum { MODE_SOLVE = 0, MODE_ONESHOT = 1 };

struct PInst {
  int dim, m, ng, ns, nu, N;
  long long s_off;  // packed x, lam: stage 1 of this instance
  long long u_off;  // packed u
  long long g_off;  // x0, x_ref, state tables
  long long a_off;  // u_ref, actuator tables
  long long t_off;  // per-point tables
  double h, k0, k1, beta, ta, gr, q, r, qf, gamma, tau, ulo, uhi;
};

struct PArgs {
  const PInst* inst;
  const int2* work;  // (instance, stage)
  int n_work, n_inst;
  const int* pt_state;  // [sum ng]: state index, or -1 - a for actuator a
  const int* act_pt;    // [sum nu]: grid point of actuator a
  const int* Lc;        // [sum ng][ELL] columns of L (unused slots: the point itself, weight 0)
  const double* Lv;
  const int* Ltc;       // the same for L^T
  const double* Ltv;
  const double* Ld;     // [sum ng] L[p][p]
  const double* x0;
  const double* xref;
  const double* uref;
  const double* xin;
  const double* uin;
  const double* lin;
  double* xout;
  double* uout;
  double* lout;
  double* dx;  // direction Delta s
  double* du;
  double* dl;
  unsigned long long* rmax;   // [2][n] bits of ||K||_inf per iteration parity
  double* rsq;                // [2][n]
  unsigned long long* acand;  // [2][n] bits of the admissible step
  int* status;
  int* iters;
  int* final_buf;
  double* fin;                // [2][n] final (||K||_inf, ||K||_2)
  int* n_active;
  int n_lo, n_u_it, rb, half, k, mode, max_iter;
  double tol;
};

__device__ __forceinline__ double phi(const PInst& I, double w) {
  return I.k0 * (w + 0.5 * I.k1 * w * w);
}
__device__ __forceinline__ double dphi(const PInst& I, double w) {
  return I.k0 * (1.0 + I.k1 * w);
}

// max that keeps a NaN once one has been seen (fmax would drop it)
__device__ __forceinline__ double nan_max(double a, double b) {
  return (a != a || b != b) ? CUDART_NAN : fmax(a, b);
}

// Block reductions of (max, sum) over THREADS threads.
__device__ void block_max_sum(double& mx, double& sq, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double om = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = (om != om || om > mx) ? om : mx;  // NaN propagates
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
  }
  if (lane == 0) {
    red[w] = mx;
    red[32 + w] = sq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < THREADS / 32; ++i) {
      mx = (red[i] != red[i] || red[i] > mx) ? red[i] : mx;
      sq += red[32 + i];
    }
  }
  __syncthreads();
}

// Sweeps of P^{-1} (eq. 24) over the state points of the stage grid:
// F_x v5 = b4, then F_x^T v4 = b5 - A_xx v5, n_lo pointwise Jacobi sweeps
// each from zero (Lemma 1).  F_x = h (L diag(Phi'(w)) - diag(beta + 4 gr x^3))
// - I on the state points; its off-diagonal part sums L[p][q] Phi'(w_q) v_q
// over the state neighbours q (v is zero at the actuator points).
struct Fields {
  double *W, *LB, *PH, *DP, *LTL, *DG, *AX, *V, *V2, *B4, *B5, *K1, *K3, *Y4, *Y5, *Z;
};

__device__ void p_inv(const PArgs& A, const PInst& I, const Fields& f, const int* pts) {
  const int ng = I.ng;
  const int* Lc = A.Lc + I.t_off * ELL;
  const double* Lv = A.Lv + I.t_off * ELL;
  const int* Ltc = A.Ltc + I.t_off * ELL;
  const double* Ltv = A.Ltv + I.t_off * ELL;
  const double* Ld = A.Ld + I.t_off;
  // F_x v5 = b4
  double* cur = f.V;
  double* nxt = f.V2;
  for (int p = threadIdx.x; p < ng; p += THREADS) cur[p] = (pts[p] >= 0) ? f.B4[p] / f.DG[p] : 0.0;
  __syncthreads();
  for (int sw = 1; sw < A.n_lo; ++sw) {
    for (int p = threadIdx.x; p < ng; p += THREADS) {
      double v = 0.0;
      if (pts[p] >= 0) {
        double off = 0.0;
#pragma unroll
        for (int e = 0; e < ELL; ++e) {
          const int c = Lc[p * ELL + e];
          off += Lv[p * ELL + e] * f.DP[c] * cur[c];
        }
        off -= Ld[p] * f.DP[p] * cur[p];
        v = (f.B4[p] - I.h * off) / f.DG[p];
      }
      nxt[p] = v;
    }
    __syncthreads();
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int p = threadIdx.x; p < ng; p += THREADS) f.Y5[p] = cur[p];
  __syncthreads();
  // F_x^T v4 = b5 - A_xx v5; off-diagonal part h Phi'(x_p) sum_q L[q][p] v_q
  for (int p = threadIdx.x; p < ng; p += THREADS)
    cur[p] = (pts[p] >= 0) ? (f.B5[p] - f.AX[p] * f.Y5[p]) / f.DG[p] : 0.0;
  __syncthreads();
  for (int sw = 1; sw < A.n_lo; ++sw) {
    for (int p = threadIdx.x; p < ng; p += THREADS) {
      double v = 0.0;
      if (pts[p] >= 0) {
        double off = 0.0;
#pragma unroll
        for (int e = 0; e < ELL; ++e) off += Ltv[p * ELL + e] * cur[Ltc[p * ELL + e]];
        off -= Ld[p] * cur[p];
        v = (f.B5[p] - f.AX[p] * f.Y5[p] - I.h * f.DP[p] * off) / f.DG[p];
      }
      nxt[p] = v;
    }
    __syncthreads();
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int p = threadIdx.x; p < ng; p += THREADS) f.Y4[p] = cur[p];
  __syncthreads();
}

__global__ void __launch_bounds__(THREADS) k_plate_dir(PArgs A) {
  const int2 it = A.work[blockIdx.x];
  const int b = it.x, s = it.y;
  if (A.rb && ((s & 1) != A.half)) return;
  if (A.mode == MODE_SOLVE && A.status[b] != ST_RUNNING) return;
  const PInst I = A.inst[b];
  const int ng = I.ng, ns = I.ns, nu = I.nu, N = I.N;
  const bool last = (s == N - 1);
  extern __shared__ double smem[];
  Fields f;
  double* q = smem;
  f.W = q; q += ng;
  f.LB = q; q += ng;
  f.PH = q; q += ng;
  f.DP = q; q += ng;
  f.LTL = q; q += ng;
  f.DG = q; q += ng;
  f.AX = q; q += ng;
  f.V = q; q += ng;
  f.V2 = q; q += ng;
  f.B4 = q; q += ng;
  f.B5 = q; q += ng;
  f.K1 = q; q += ng;
  f.K3 = q; q += ng;
  f.Y4 = q; q += ng;
  f.Y5 = q; q += ng;
  f.Z = q; q += ng;
  __shared__ double sK2[MAX_NU], sAUU[MAX_NU], sV3[MAX_NU], red[64];
  const int* pts = A.pt_state + I.t_off;
  const int* apt = A.act_pt + I.a_off;
  const int* Lc = A.Lc + I.t_off * ELL;
  const double* Lv = A.Lv + I.t_off * ELL;
  const int* Ltc = A.Ltc + I.t_off * ELL;
  const double* Ltv = A.Ltv + I.t_off * ELL;
  const double* Ld = A.Ld + I.t_off;
  const long long so = I.s_off + (long long)s * ns;
  const long long uo = I.u_off + (long long)s * nu;
  const double h = I.h;

  // the stage's grid: w = x (states) / u (actuators); lambda-bar
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    const int t = pts[p];
    double w, lb;
    if (t >= 0) {
      w = A.xin[so + t];
      lb = A.lin[so + t];
    } else {
      w = A.uin[uo + (-1 - t)];
      lb = 0.0;
    }
    f.W[p] = w;
    f.LB[p] = lb;
    f.PH[p] = phi(I, w);
    f.DP[p] = dphi(I, w);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    double acc = 0.0;
#pragma unroll
    for (int e = 0; e < ELL; ++e) acc += Ltv[p * ELL + e] * f.LB[Ltc[p * ELL + e]];
    f.LTL[p] = acc;  // (L^T lambda-bar)(p)
  }
  __syncthreads();

  // K_i (eq. 9), coefficients, norms
  double mx = 0.0, sq = 0.0;
  const double d2p = I.k0 * I.k1;
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    const int t = pts[p];
    if (t < 0) {
      f.K1[p] = f.K3[p] = 0.0;
      f.DG[p] = 1.0;
      f.AX[p] = 0.0;
      continue;
    }
    const double x = f.W[p], lam = f.LB[p], xr = A.xref[I.g_off + t];
    const double xprev = (s == 0) ? A.x0[I.g_off + t] : A.xin[so - ns + t];
    const double lnext = last ? h * I.qf * (x - xr) : A.lin[so + ns + t];
    double lph = 0.0;
#pragma unroll
    for (int e = 0; e < ELL; ++e) lph += Lv[p * ELL + e] * f.PH[Lc[p * ELL + e]];
    const double x3 = x * x * x;
    const double fp = lph - I.beta * (x - I.ta) - I.gr * (x3 * x - I.ta * I.ta * I.ta * I.ta);
    const double K1 = xprev - x + h * fp;
    const double gxT = f.DP[p] * f.LTL[p] - (I.beta + 4.0 * I.gr * x3) * lam;
    const double K3 = lnext - lam + h * (I.q * (x - xr) + gxT);
    mx = nan_max(mx, nan_max(fabs(K1), fabs(K3)));
    sq += K1 * K1 + K3 * K3;
    // red-black half 1: the right-hand side takes the even neighbours'
    // directions (state rows: M_L Delta x_{i-1}; costate rows: M_U Delta
    // lambda_{i+1}); the norms above stay those of K(S^k)
    double K1r = K1, K3r = K3;
    if (A.rb && A.half == 1) {
      if (s > 0) K1r -= A.dx[so - ns + t];
      if (!last) K3r -= A.dl[so + ns + t];
    }
    f.K1[p] = K1r;
    f.K3[p] = K3r;
    f.DG[p] = h * (Ld[p] * f.DP[p] - I.beta - 4.0 * I.gr * x3) - 1.0;
    f.AX[p] = h * (I.q + d2p * f.LTL[p] - 12.0 * I.gr * x * x * lam) + (last ? h * I.qf : 0.0);
  }
  for (int a = threadIdx.x; a < nu; a += THREADS) {
    const int pa = apt[a];
    const double u = f.W[pa];
    double db = 0.0, d2b = 0.0;
    if (I.tau > 0.0) {
      db = -I.tau / (u - I.ulo) + I.tau / (I.uhi - u);
      d2b = I.tau / ((u - I.ulo) * (u - I.ulo)) + I.tau / ((I.uhi - u) * (I.uhi - u));
    }
    const double K2 = h * (I.r * (u - A.uref[I.a_off + a]) + db + f.DP[pa] * f.LTL[pa]);
    mx = nan_max(mx, fabs(K2));
    sq += K2 * K2;
    sK2[a] = K2;
    sAUU[a] = h * (I.r + d2b + d2p * f.LTL[pa]) + I.gamma;
    sV3[a] = 0.0;
  }
  __syncthreads();
  block_max_sum(mx, sq, red);
  if (threadIdx.x == 0) {
    const int slot = (A.k & 1) * A.n_inst + b;
    atomicMax(&A.rmax[slot], (unsigned long long)__double_as_longlong(mx));
    atomicAdd(&A.rsq[slot], sq);
  }
  if (A.mode == MODE_SOLVE && A.k >= A.max_iter) return;  // norms only

  // u fixed-point iteration (Sec. 5.2): y = P^{-1}(F_u v3 - b1, -b2),
  // v3 = (b3 + F_u^T y_lambda) / A_uu, from v3 = 0
  for (int itu = 0; itu <= A.n_u_it; ++itu) {
    const bool final_pass = (itu == A.n_u_it);
    // Z = Phi'(u) v3 at the actuator points, zero elsewhere
    for (int p = threadIdx.x; p < ng; p += THREADS) f.Z[p] = 0.0;
    __syncthreads();
    for (int a = threadIdx.x; a < nu; a += THREADS) f.Z[apt[a]] = f.DP[apt[a]] * sV3[a];
    __syncthreads();
    for (int p = threadIdx.x; p < ng; p += THREADS) {
      double fu = 0.0;  // (F_u v3)(p) = h sum_a L[p][a] Phi'(u_a) v3_a
#pragma unroll
      for (int e = 0; e < ELL; ++e) fu += Lv[p * ELL + e] * f.Z[Lc[p * ELL + e]];
      fu *= h;
      if (pts[p] >= 0) {
        f.B4[p] = final_pass ? f.K1[p] - fu : fu - f.K1[p];
        f.B5[p] = final_pass ? f.K3[p] : -f.K3[p];
      } else {
        f.B4[p] = f.B5[p] = 0.0;
      }
    }
    __syncthreads();
    p_inv(A, I, f, pts);
    if (final_pass) break;
    for (int a = threadIdx.x; a < nu; a += THREADS) {
      const int pa = apt[a];
      double acc = 0.0;  // (L^T y_lambda)(a) over the state points
#pragma unroll
      for (int e = 0; e < ELL; ++e) acc += Ltv[pa * ELL + e] * f.Y4[Ltc[pa * ELL + e]];
      sV3[a] = (sK2[a] + h * f.DP[pa] * acc) / sAUU[a];
    }
    __syncthreads();
  }
  // direction (Delta x, Delta u, Delta lambda) = (v5, v3, v4); admissible step
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    const int t = pts[p];
    if (t >= 0) {
      A.dx[so + t] = f.Y5[p];
      A.dl[so + t] = f.Y4[p];
    }
  }
  double amin = 1.0;
  for (int a = threadIdx.x; a < nu; a += THREADS) {
    const double d = sV3[a], u = f.W[apt[a]];
    A.du[uo + a] = d;
    if (I.tau > 0.0) {
      if (d > 0.0) amin = fmin(amin, 0.995 * (u - I.ulo) / d);
      if (d < 0.0) amin = fmin(amin, 0.995 * (I.uhi - u) / (-d));
    }
  }
  for (int o = 16; o > 0; o >>= 1) amin = fmin(amin, __shfl_xor_sync(0xffffffffu, amin, o));
  if ((threadIdx.x & 31) == 0 && amin < 1.0)
    atomicMin(&A.acand[(A.k & 1) * A.n_inst + b], (unsigned long long)__double_as_longlong(amin));
}

// The decision of iteration k and the update S^{k+1} = S^k - alpha Delta S.
__global__ void __launch_bounds__(THREADS) k_plate_update(PArgs A) {
  const int2 it = A.work[blockIdx.x];
  const int b = it.x, s = it.y;
  const PInst I = A.inst[b];
  const int slot = (A.k & 1) * A.n_inst + b;
  bool stop = false;
  double r = 0.0;
  if (A.mode == MODE_SOLVE) {
    if (A.status[b] != ST_RUNNING) return;  // finished before this kernel
    r = __longlong_as_double((long long)A.rmax[slot]);
    stop = !(r <= 1.79e308) || r <= A.tol || A.k >= A.max_iter;
  }
  if (s == 0 && threadIdx.x == 0) {
    const int nslot = ((A.k + 1) & 1) * A.n_inst + b;
    A.rmax[nslot] = 0ull;
    A.rsq[nslot] = 0.0;
    A.acand[nslot] = (unsigned long long)__double_as_longlong(1.0);
  }
  if (stop) {
    if (s == 0 && threadIdx.x == 0) {
      A.status[b] = !(r <= 1.79e308) ? ST_DIVERGED : (r <= A.tol ? ST_CONVERGED : ST_MAX_ITER);
      A.iters[b] = A.k;
      A.final_buf[b] = A.k & 1;
      A.fin[b] = r;
      A.fin[A.n_inst + b] = sqrt(A.rsq[slot]);
      atomicSub(A.n_active, 1);
    }
    return;
  }
  const double alpha = fmin(1.0, __longlong_as_double((long long)A.acand[slot]));
  const long long so = I.s_off + (long long)s * I.ns;
  const long long uo = I.u_off + (long long)s * I.nu;
  for (int t = threadIdx.x; t < I.ns; t += THREADS) {
    A.xout[so + t] = A.xin[so + t] - alpha * A.dx[so + t];
    A.lout[so + t] = A.lin[so + t] - alpha * A.dl[so + t];
  }
  for (int a = threadIdx.x; a < I.nu; a += THREADS) A.uout[uo + a] = A.uin[uo + a] - alpha * A.du[uo + a];
}

// Start iterate into buffer 0 (mode 0 cold, 1 copy of the current state,
// 2 the current state shifted by one stage) and the control words.
__global__ void k_plate_init(const PInst* inst, int n_inst, int mode, const double* x0,
                             const double* xc, const double* uc, const double* lc, double* x,
                             double* u, double* lam, unsigned long long* rmax, double* rsq,
                             unsigned long long* acand, int* status, int* n_active) {
  const int b = blockIdx.y;
  const PInst I = inst[b];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < I.N * I.ns; e += gridDim.x * blockDim.x) {
    const int s = e / I.ns, t = e - s * I.ns;
    const int ss = (mode == 2) ? min(s + 1, I.N - 1) : s;
    const long long src = I.s_off + (long long)ss * I.ns + t;
    x[I.s_off + e] = (mode == 0) ? x0[I.g_off + t] : xc[src];
    lam[I.s_off + e] = (mode == 0) ? 0.0 : lc[src];
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < I.N * I.nu; e += gridDim.x * blockDim.x) {
    const int s = e / I.nu, a = e - s * I.nu;
    const int ss = (mode == 2) ? min(s + 1, I.N - 1) : s;
    u[I.u_off + e] = (mode == 0) ? (I.tau > 0.0 ? 0.5 * (I.ulo + I.uhi) : 0.0)
                                 : uc[I.u_off + (long long)ss * I.nu + a];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int q = 0; q < 2; ++q) {
      rmax[q * n_inst + b] = 0ull;
      rsq[q * n_inst + b] = 0.0;
      acand[q * n_inst + b] = (unsigned long long)__double_as_longlong(1.0);
    }
    status[b] = ST_RUNNING;
    if (b == 0) *n_active = n_inst;
  }
}

// The returned iterate (buffer final_buf[b]) into the current state.
__global__ void k_plate_gather(const PInst* inst, const int* final_buf, const double* x0b,
                               const double* x1b, const double* u0b, const double* u1b,
                               const double* l0b, const double* l1b, double* xc, double* uc,
                               double* lc, double* u_out) {
  const int b = blockIdx.y;
  const PInst I = inst[b];
  const int fb = final_buf[b];
  const double* xs = fb ? x1b : x0b;
  const double* us = fb ? u1b : u0b;
  const double* ls = fb ? l1b : l0b;
  for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < (long long)I.N * I.ns;
       e += gridDim.x * blockDim.x) {
    xc[I.s_off + e] = xs[I.s_off + e];
    lc[I.s_off + e] = ls[I.s_off + e];
  }
  for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < (long long)I.N * I.nu;
       e += gridDim.x * blockDim.x) {
    uc[I.u_off + e] = us[I.u_off + e];
    if (u_out) u_out[I.u_off + e] = us[I.u_off + e];
  }
}

// The plant: w (state points) += (dt / n_sub) f(w, u1), n_sub times, with the
// actuator points at the first-stage inputs u1 of the current state; dt < 0
// takes each instance's own stage length h.
__global__ void __launch_bounds__(THREADS) k_plate_plant(PArgs A, double* w, const double* uc,
                                                         double dt, int n_sub) {
  const int b = blockIdx.x;
  const PInst I = A.inst[b];
  extern __shared__ double smem[];
  double* W = smem;
  double* PH = W + I.ng;
  const int* pts = A.pt_state + I.t_off;
  const int* Lc = A.Lc + I.t_off * ELL;
  const double* Lv = A.Lv + I.t_off * ELL;
  for (int p = threadIdx.x; p < I.ng; p += THREADS) {
    const int t = pts[p];
    W[p] = (t >= 0) ? w[I.g_off + t] : uc[I.u_off + (-1 - t)];
  }
  __syncthreads();
  const double tau = (dt < 0.0 ? I.h : dt) / n_sub;
  for (int k = 0; k < n_sub; ++k) {
    for (int p = threadIdx.x; p < I.ng; p += THREADS) PH[p] = phi(I, W[p]);
    __syncthreads();
    double nw[4];
    int cnt = 0;
    for (int p = threadIdx.x; p < I.ng; p += THREADS, ++cnt) {
      double v = W[p];
      if (pts[p] >= 0) {
        double lph = 0.0;
#pragma unroll
        for (int e = 0; e < ELL; ++e) lph += Lv[p * ELL + e] * PH[Lc[p * ELL + e]];
        const double x = v, x4 = x * x * x * x;
        v = x + tau * (lph - I.beta * (x - I.ta) - I.gr * (x4 - I.ta * I.ta * I.ta * I.ta));
      }
      nw[cnt] = v;
    }
    __syncthreads();
    cnt = 0;
    for (int p = threadIdx.x; p < I.ng; p += THREADS, ++cnt) W[p] = nw[cnt];
    __syncthreads();
  }
  for (int p = threadIdx.x; p < I.ng; p += THREADS) {
    const int t = pts[p];
    if (t >= 0) w[I.g_off + t] = W[p];
  }
}

}  // namespace plate_dev

using plate_dev::PInst;
using plate_dev::PArgs;

struct nmpc_plate {
  int n = 0;
  nmpc_plate_opts opts{};
  std::vector<PInst> inst_h;
  long long n_s = 0, n_x = 0, n_u = 0, n_a = 0, n_pts = 0;  // sum ns, N ns, N nu, nu, ng
  int ng_max = 0, max_N = 0;
  // device
  PInst* inst_d = nullptr;
  int2* work_d = nullptr;
  int n_work = 0;
  int *pt_state = nullptr, *act_pt = nullptr, *Lc = nullptr, *Ltc = nullptr;
  double *Lv = nullptr, *Ltv = nullptr, *Ld = nullptr;
  double *x0 = nullptr, *xref = nullptr, *uref = nullptr;
  double* xb[3] = {nullptr, nullptr, nullptr};
  double* ub[3] = {nullptr, nullptr, nullptr};
  double* lb[3] = {nullptr, nullptr, nullptr};
  double *dx = nullptr, *du = nullptr, *dl = nullptr;
  unsigned long long *rmax = nullptr, *acand = nullptr;
  double *rsq = nullptr, *fin = nullptr;
  int *status = nullptr, *iters = nullptr, *final_buf = nullptr, *n_active = nullptr;
  bool has_state = false;
  size_t smem = 0;
};

namespace {

#define PCK(call)                                                          \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      fprintf(stderr, "nmpc_plate: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      return NMPC_ERR_CUDA;                                                \
    }                                                                      \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
}

template <typename T>
cudaError_t upload(T* d, const std::vector<T>& v) {
  if (v.empty()) return cudaSuccess;
  return cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void free_plate(nmpc_plate* h) {
  void* ptrs[] = {h->inst_d, h->work_d, h->pt_state, h->act_pt, h->Lc, h->Ltc, h->Lv, h->Ltv,
                  h->Ld, h->x0, h->xref, h->uref, h->xb[0], h->xb[1], h->xb[2], h->ub[0],
                  h->ub[1], h->ub[2], h->lb[0], h->lb[1], h->lb[2], h->dx, h->du, h->dl,
                  h->rmax, h->acand, h->rsq, h->fin, h->status, h->iters, h->final_buf,
                  h->n_active};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

int validate(const nmpc_plate_desc& d) {
  if ((d.dim != 1 && d.dim != 2) || d.horizon < 1 || d.n_u < 1 || !d.act_cell) return NMPC_ERR_BAD_ARG;
  if (d.bc != 0 && d.bc != 1) return NMPC_ERR_BAD_ARG;
  if (d.m < (d.bc == 0 ? 3 : 1)) return NMPC_ERR_BAD_ARG;
  const long long ng = d.dim == 2 ? (long long)d.m * d.m : d.m;
  if (ng > NMPC_PLATE_MAX_POINTS || d.n_u > plate_dev::MAX_NU) return NMPC_ERR_UNSUPPORTED;
  if (d.n_u >= ng) return NMPC_ERR_BAD_ARG;
  std::vector<char> seen(ng, 0);
  for (int a = 0; a < d.n_u; ++a) {
    if (d.act_cell[a] < 0 || d.act_cell[a] >= ng || seen[d.act_cell[a]]) return NMPC_ERR_BAD_ARG;
    seen[d.act_cell[a]] = 1;
  }
  if (!(d.h > 0) || !(d.k0 > 0) || !std::isfinite(d.k1) || !(d.beta >= 0) || !(d.gamma_r >= 0) ||
      !std::isfinite(d.t_amb) || !(d.q >= 0) || !(d.r > 0) || !(d.qf >= 0) || !(d.gamma >= 0) ||
      !(d.tau >= 0))
    return NMPC_ERR_BAD_ARG;
  if (d.tau > 0 && !(d.u_lo < d.u_hi)) return NMPC_ERR_BAD_ARG;
  return NMPC_OK;
}

// Row p of the grid Laplacian as (column, weight) pairs: zero Neumann by
// mirrored fictitious points (a missing neighbour is replaced by the inner
// one, so that neighbour's weight doubles), zero Dirichlet by dropping
// neighbours outside.
void laplacian_rows(const nmpc_plate_desc& d, std::vector<std::vector<std::pair<int, double>>>& rows) {
  const int m = d.m, dim = d.dim;
  const long long ng = dim == 2 ? (long long)m * m : m;
  const double dp = d.bc == 0 ? 1.0 / (m - 1) : 1.0 / (m + 1);
  const double w = 1.0 / (dp * dp);
  rows.assign(ng, {});
  auto add = [&](int p, int c, double v) {
    for (auto& e : rows[p])
      if (e.first == c) {
        e.second += v;
        return;
      }
    rows[p].push_back({c, v});
  };
  for (int p = 0; p < ng; ++p) {
    const int ix = p % m, iy = p / m;
    add(p, p, -2.0 * dim * w);
    for (int axis = 0; axis < dim; ++axis) {
      const int i = axis == 0 ? ix : iy;
      for (int dir = -1; dir <= 1; dir += 2) {
        int j = i + dir;
        if (j < 0 || j >= m) {
          if (d.bc == 1) continue;   // Dirichlet: zero outside
          j = i - dir;               // Neumann: the mirrored point
        }
        const int c = axis == 0 ? iy * m + j : j * m + ix;
        add(p, c, w);
      }
    }
  }
}

PArgs make_args(nmpc_plate* h, int rd) {
  PArgs A{};
  A.inst = h->inst_d;
  A.work = h->work_d;
  A.n_work = h->n_work;
  A.n_inst = h->n;
  A.pt_state = h->pt_state;
  A.act_pt = h->act_pt;
  A.Lc = h->Lc;
  A.Lv = h->Lv;
  A.Ltc = h->Ltc;
  A.Ltv = h->Ltv;
  A.Ld = h->Ld;
  A.x0 = h->x0;
  A.xref = h->xref;
  A.uref = h->uref;
  A.xin = h->xb[rd];
  A.uin = h->ub[rd];
  A.lin = h->lb[rd];
  A.xout = h->xb[rd ^ 1];
  A.uout = h->ub[rd ^ 1];
  A.lout = h->lb[rd ^ 1];
  A.dx = h->dx;
  A.du = h->du;
  A.dl = h->dl;
  A.rmax = h->rmax;
  A.rsq = h->rsq;
  A.acand = h->acand;
  A.status = h->status;
  A.iters = h->iters;
  A.final_buf = h->final_buf;
  A.fin = h->fin;
  A.n_active = h->n_active;
  A.n_lo = h->opts.n_lo;
  A.n_u_it = h->opts.n_u_it;
  A.rb = (h->opts.variant == NMPC_VARIANT_REDBLACK) ? 1 : 0;
  A.max_iter = h->opts.max_iter;
  A.tol = h->opts.tol;
  return A;
}

// One iteration k: the direction kernels (one or two halves), then the update.
cudaError_t launch_iteration(nmpc_plate* h, PArgs A, cudaStream_t st) {
  const int halves = A.rb ? 2 : 1;
  for (int half = 0; half < halves; ++half) {
    A.half = half;
    plate_dev::k_plate_dir<<<h->n_work, plate_dev::THREADS, h->smem, st>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  plate_dev::k_plate_update<<<h->n_work, plate_dev::THREADS, 0, st>>>(A);
  return cudaGetLastError();
}

dim3 inst_grid(const nmpc_plate* h) { return dim3(8, (unsigned)h->n); }

}  // namespace

extern "C" {

void nmpc_plate_default_opts(nmpc_plate_opts* o) {
  if (!o) return;
  o->tol = 1e-6;
  o->max_iter = 5000;
  o->n_lo = 2;
  o->n_u_it = 2;
  o->variant = NMPC_VARIANT_JACOBI;
  o->check_every = 16;
}

int nmpc_plate_setup(const nmpc_plate_desc* descs, int n, const nmpc_plate_opts* opts,
                     nmpc_plate** out) {
  if (!descs || n < 1 || !out) return NMPC_ERR_BAD_ARG;
  *out = nullptr;
  nmpc_plate_opts o;
  nmpc_plate_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol >= 0) || o.max_iter < 0 || o.n_lo < 1 || o.n_u_it < 0 || o.check_every < 1 ||
      (o.variant != NMPC_VARIANT_JACOBI && o.variant != NMPC_VARIANT_REDBLACK))
    return NMPC_ERR_BAD_ARG;
  for (int b = 0; b < n; ++b) {
    const int rc = validate(descs[b]);
    if (rc != NMPC_OK) return rc;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return NMPC_ERR_NO_DEVICE;
  nmpc_plate* h = new (std::nothrow) nmpc_plate();
  if (!h) return NMPC_ERR_CUDA;
  h->n = n;
  h->opts = o;
  std::vector<int> pt_state, act_pt, Lc, Ltc;
  std::vector<double> Lv, Ltv, Ld;
  std::vector<int2> work;
  for (int b = 0; b < n; ++b) {
    const nmpc_plate_desc& d = descs[b];
    PInst I{};
    I.dim = d.dim;
    I.m = d.m;
    I.ng = d.dim == 2 ? d.m * d.m : d.m;
    I.nu = d.n_u;
    I.ns = I.ng - I.nu;
    I.N = d.horizon;
    I.s_off = h->n_x;
    I.u_off = h->n_u;
    I.g_off = h->n_s;
    I.a_off = h->n_a;
    I.t_off = h->n_pts;
    I.h = d.h;
    I.k0 = d.k0;
    I.k1 = d.k1;
    I.beta = d.beta;
    I.ta = d.t_amb;
    I.gr = d.gamma_r;
    I.q = d.q;
    I.r = d.r;
    I.qf = d.qf;
    I.gamma = d.gamma;
    I.tau = d.tau;
    I.ulo = d.u_lo;
    I.uhi = d.u_hi;
    // point -> state index (grid order of the non-actuator points) or -1 - a
    std::vector<int> state_of(I.ng, -1);
    for (int a = 0; a < d.n_u; ++a) state_of[d.act_cell[a]] = -1 - a;
    int t = 0;
    std::vector<char> is_act(I.ng, 0);
    for (int a = 0; a < d.n_u; ++a) is_act[d.act_cell[a]] = 1;
    for (int p = 0; p < I.ng; ++p)
      if (!is_act[p]) state_of[p] = t++;
    for (int p = 0; p < I.ng; ++p) pt_state.push_back(state_of[p]);
    for (int a = 0; a < d.n_u; ++a) act_pt.push_back(d.act_cell[a]);
    std::vector<std::vector<std::pair<int, double>>> rows, trows(I.ng);
    laplacian_rows(d, rows);
    for (int p = 0; p < I.ng; ++p)
      for (auto& e : rows[p]) trows[e.first].push_back({p, e.second});
    for (int p = 0; p < I.ng; ++p) {
      double diag = 0.0;
      for (int e = 0; e < plate_dev::ELL; ++e) {
        const bool on = e < (int)rows[p].size();
        Lc.push_back(on ? rows[p][e].first : p);
        Lv.push_back(on ? rows[p][e].second : 0.0);
        if (on && rows[p][e].first == p) diag = rows[p][e].second;
        const bool ton = e < (int)trows[p].size();
        Ltc.push_back(ton ? trows[p][e].first : p);
        Ltv.push_back(ton ? trows[p][e].second : 0.0);
      }
      Ld.push_back(diag);
    }
    for (int s = 0; s < I.N; ++s) work.push_back(make_int2(b, s));
    h->n_x += (long long)I.N * I.ns;
    h->n_u += (long long)I.N * I.nu;
    h->n_s += I.ns;
    h->n_a += I.nu;
    h->n_pts += I.ng;
    h->ng_max = std::max(h->ng_max, I.ng);
    h->max_N = std::max(h->max_N, I.N);
    h->inst_h.push_back(I);
  }
  h->n_work = (int)work.size();
  h->smem = (size_t)16 * h->ng_max * sizeof(double);
  bool ok = true;
  auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
  A(dalloc(&h->inst_d, n));
  A(dalloc(&h->work_d, work.size()));
  A(dalloc(&h->pt_state, pt_state.size()));
  A(dalloc(&h->act_pt, act_pt.size()));
  A(dalloc(&h->Lc, Lc.size()));
  A(dalloc(&h->Ltc, Ltc.size()));
  A(dalloc(&h->Lv, Lv.size()));
  A(dalloc(&h->Ltv, Ltv.size()));
  A(dalloc(&h->Ld, Ld.size()));
  A(dalloc(&h->x0, h->n_s));
  A(dalloc(&h->xref, h->n_s));
  A(dalloc(&h->uref, h->n_a));
  for (int q = 0; q < 3; ++q) {
    A(dalloc(&h->xb[q], h->n_x));
    A(dalloc(&h->ub[q], h->n_u));
    A(dalloc(&h->lb[q], h->n_x));
  }
  A(dalloc(&h->dx, h->n_x));
  A(dalloc(&h->du, h->n_u));
  A(dalloc(&h->dl, h->n_x));
  A(dalloc(&h->rmax, 2 * n));
  A(dalloc(&h->acand, 2 * n));
  A(dalloc(&h->rsq, 2 * n));
  A(dalloc(&h->fin, 2 * n));
  A(dalloc(&h->status, n));
  A(dalloc(&h->iters, n));
  A(dalloc(&h->final_buf, n));
  A(dalloc(&h->n_active, 1));
  if (ok) {
    A(upload(h->inst_d, h->inst_h));
    A(upload(h->work_d, work));
    A(upload(h->pt_state, pt_state));
    A(upload(h->act_pt, act_pt));
    A(upload(h->Lc, Lc));
    A(upload(h->Ltc, Ltc));
    A(upload(h->Lv, Lv));
    A(upload(h->Ltv, Ltv));
    A(upload(h->Ld, Ld));
  }
  if (ok && h->smem > 48 * 1024)
    A(cudaFuncSetAttribute(plate_dev::k_plate_dir, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)h->smem));
  if (!ok) {
    free_plate(h);
    delete h;
    return NMPC_ERR_CUDA;
  }
  *out = h;
  return NMPC_OK;
}

int nmpc_plate_sizes(const nmpc_plate* h, int64_t* out) {
  if (!h || !out) return NMPC_ERR_BAD_ARG;
  out[0] = h->n_s;
  out[1] = h->n_x;
  out[2] = h->n_u;
  out[3] = h->n_a;
  return NMPC_OK;
}

int nmpc_plate_solve(nmpc_plate* h, const double* x0, const double* x_ref, const double* u_ref,
                     int init, double* u_out, nmpc_stats* stats, void* stream) {
  if (!h || !x0 || !x_ref || !u_ref) return NMPC_ERR_BAD_ARG;
  if (init != NMPC_INIT_COLD && init != NMPC_INIT_WARM && init != NMPC_INIT_SHIFT)
    return NMPC_ERR_BAD_ARG;
  if (init != NMPC_INIT_COLD && !h->has_state) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  PCK(cudaMemcpyAsync(h->x0, x0, h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PCK(cudaMemcpyAsync(h->xref, x_ref, h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PCK(cudaMemcpyAsync(h->uref, u_ref, h->n_a * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const int mode = init == NMPC_INIT_COLD ? 0 : (init == NMPC_INIT_WARM ? 1 : 2);
  plate_dev::k_plate_init<<<inst_grid(h), 256, 0, st>>>(h->inst_d, h->n, mode, h->x0, h->xb[2],
                                                        h->ub[2], h->lb[2], h->xb[0], h->ub[0],
                                                        h->lb[0], h->rmax, h->rsq, h->acand,
                                                        h->status, h->n_active);
  PCK(cudaGetLastError());
  int active = h->n;
  for (int k = 0; k <= h->opts.max_iter;) {
    for (int c = 0; c < h->opts.check_every && k <= h->opts.max_iter; ++c, ++k) {
      PArgs A = make_args(h, k & 1);
      A.k = k;
      A.mode = plate_dev::MODE_SOLVE;
      PCK(launch_iteration(h, A, st));
    }
    PCK(cudaMemcpyAsync(&active, h->n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    if (active == 0) break;
  }
  plate_dev::k_plate_gather<<<inst_grid(h), 256, 0, st>>>(h->inst_d, h->final_buf, h->xb[0],
                                                          h->xb[1], h->ub[0], h->ub[1], h->lb[0],
                                                          h->lb[1], h->xb[2], h->ub[2], h->lb[2],
                                                          u_out);
  PCK(cudaGetLastError());
  h->has_state = true;
  std::vector<int> status(h->n), iters(h->n);
  std::vector<double> fin(2 * h->n);
  PCK(cudaMemcpyAsync(status.data(), h->status, h->n * sizeof(int), cudaMemcpyDeviceToHost, st));
  PCK(cudaMemcpyAsync(iters.data(), h->iters, h->n * sizeof(int), cudaMemcpyDeviceToHost, st));
  PCK(cudaMemcpyAsync(fin.data(), h->fin, 2 * h->n * sizeof(double), cudaMemcpyDeviceToHost, st));
  PCK(cudaStreamSynchronize(st));
  int rc = NMPC_OK;
  for (int b = 0; b < h->n; ++b) {
    if (stats) {
      stats[b].status = status[b];
      stats[b].iters = iters[b];
      stats[b].res_inf = fin[b];
      stats[b].res_2 = fin[h->n + b];
    }
    if (rc == NMPC_OK) {
      if (status[b] == plate_dev::ST_DIVERGED) rc = NMPC_ERR_DIVERGED;
      else if (status[b] != plate_dev::ST_CONVERGED) rc = NMPC_ERR_NOT_CONVERGED;
    }
  }
  return rc;
}

int nmpc_plate_iterate(nmpc_plate* h, const double* x0, const double* x_ref, const double* u_ref,
                       const double* x_in, const double* u_in, const double* lam_in,
                       double* x_out, double* u_out, double* lam_out, int n_iter, double* out,
                       void* stream) {
  if (!h || !x0 || !x_ref || !u_ref || !x_in || !u_in || !lam_in || !x_out || !u_out || !lam_out ||
      n_iter < 1)
    return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  PCK(cudaMemcpyAsync(h->x0, x0, h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PCK(cudaMemcpyAsync(h->xref, x_ref, h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PCK(cudaMemcpyAsync(h->uref, u_ref, h->n_a * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PCK(cudaMemcpyAsync(h->xb[0], x_in, h->n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PCK(cudaMemcpyAsync(h->ub[0], u_in, h->n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PCK(cudaMemcpyAsync(h->lb[0], lam_in, h->n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double a1 = 1.0;
  unsigned long long a1b;
  std::memcpy(&a1b, &a1, sizeof(a1b));
  std::vector<unsigned long long> aone(2 * h->n, a1b);
  for (int it = 0; it < n_iter; ++it) {
    PCK(cudaMemsetAsync(h->rmax, 0, 2 * h->n * sizeof(unsigned long long), st));
    PCK(cudaMemsetAsync(h->rsq, 0, 2 * h->n * sizeof(double), st));
    PCK(cudaMemcpyAsync(h->acand, aone.data(), aone.size() * sizeof(unsigned long long),
                        cudaMemcpyHostToDevice, st));
    PArgs A = make_args(h, it & 1);
    A.k = 0;  // slot 0 of the control words
    A.mode = plate_dev::MODE_ONESHOT;
    // the slot of k = 0 is read; the update's reset of slot 1 is harmless
    A.xin = h->xb[it & 1];
    A.uin = h->ub[it & 1];
    A.lin = h->lb[it & 1];
    A.xout = h->xb[(it + 1) & 1];
    A.uout = h->ub[(it + 1) & 1];
    A.lout = h->lb[(it + 1) & 1];
    PCK(launch_iteration(h, A, st));
    PCK(cudaStreamSynchronize(st));  // the host vectors above outlive the copies
  }
  const int fb = n_iter & 1;
  PCK(cudaMemcpyAsync(x_out, h->xb[fb], h->n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PCK(cudaMemcpyAsync(u_out, h->ub[fb], h->n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
  PCK(cudaMemcpyAsync(lam_out, h->lb[fb], h->n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (out) {
    std::vector<unsigned long long> rm(h->n), ac(h->n);
    std::vector<double> rs(h->n);
    PCK(cudaMemcpyAsync(rm.data(), h->rmax, h->n * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, st));
    PCK(cudaMemcpyAsync(rs.data(), h->rsq, h->n * sizeof(double), cudaMemcpyDeviceToHost, st));
    PCK(cudaMemcpyAsync(ac.data(), h->acand, h->n * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    for (int b = 0; b < h->n; ++b) {
      double r, a;
      std::memcpy(&r, &rm[b], sizeof(r));
      std::memcpy(&a, &ac[b], sizeof(a));
      out[3 * b] = r;
      out[3 * b + 1] = std::sqrt(rs[b]);
      out[3 * b + 2] = std::min(1.0, a);
    }
  }
  return NMPC_OK;
}

int nmpc_plate_get_state(nmpc_plate* h, double* x, double* u, double* lam, void* stream) {
  if (!h) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (x) PCK(cudaMemcpyAsync(x, h->xb[2], h->n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (u) PCK(cudaMemcpyAsync(u, h->ub[2], h->n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (lam) PCK(cudaMemcpyAsync(lam, h->lb[2], h->n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return NMPC_OK;
}

namespace {
int plant(nmpc_plate* h, double* w, double dt, int n_sub, void* stream) {
  PArgs A = make_args(h, 0);
  plate_dev::k_plate_plant<<<h->n, plate_dev::THREADS, 2 * h->ng_max * sizeof(double),
                             (cudaStream_t)stream>>>(A, w, h->ub[2], dt, n_sub);
  PCK(cudaGetLastError());
  return NMPC_OK;
}
}  // namespace

int nmpc_plate_plant_step(nmpc_plate* h, double* w, double dt, int n_sub, void* stream) {
  if (!h || !w || !(dt >= 0) || n_sub < 1 || !h->has_state) return NMPC_ERR_BAD_ARG;
  return plant(h, w, dt, n_sub, stream);
}

int nmpc_plate_closed_loop(nmpc_plate* h, double* w, const double* x_ref, const double* u_ref,
                           int steps, int n_sub, double* u_hist, int* iters_hist,
                           double* res_hist, void* stream) {
  if (!h || !w || !x_ref || !u_ref || steps < 1 || n_sub < 1) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<nmpc_stats> stats(h->n);
  int rc_all = NMPC_OK;
  for (int t = 0; t < steps; ++t) {
    const int init = (t == 0 && !h->has_state) ? NMPC_INIT_COLD : NMPC_INIT_SHIFT;
    const int rc = nmpc_plate_solve(h, w, x_ref, u_ref, init, nullptr, stats.data(), stream);
    if (rc == NMPC_ERR_BAD_ARG || rc == NMPC_ERR_CUDA) return rc;
    if (rc != NMPC_OK && rc_all == NMPC_OK) rc_all = rc;
    for (int b = 0; b < h->n; ++b) {
      if (iters_hist) iters_hist[(size_t)t * h->n + b] = stats[b].iters;
      if (res_hist) res_hist[(size_t)t * h->n + b] = stats[b].res_inf;
    }
    if (u_hist) {
      // u_1 of every instance (stage 1 of the packed control trajectory)
      for (int b = 0; b < h->n; ++b) {
        const PInst& I = h->inst_h[b];
        PCK(cudaMemcpyAsync(u_hist + (size_t)t * h->n_a + I.a_off, h->ub[2] + I.u_off,
                            I.nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
      }
    }
    const int prc = plant(h, w, -1.0, n_sub, stream);  // each instance's own h
    if (prc != NMPC_OK) return prc;
  }
  return rc_all;
}

void nmpc_plate_destroy(nmpc_plate* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  free_plate(h);
  delete h;
}

}  // extern "C"
