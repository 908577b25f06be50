// Device code of the double-layer Jacobi NMPC solver (sm_103a).
//
// One CTA processes one (instance, stage) work item of one upper-layer
// iteration (eq. 15): every stage of every instance is updated at once from
// iterate k, so the whole grid is one iteration.  Inside a work item:
//   phase A (float64): the stage's KKT rows K_i (eq. 9) from x_{i-1}, s_i,
//     lambda_{i+1}; the coefficient fields Phi'(x) and A_xx of the reordered
//     stage block (eq. 21); the residual norms (max |K|, sum K^2);
//   phase B (T = float or double): the lower layer (Sec. 4.3, eqs. 22-24 and
//     the u fixed-point iteration of Sec. 5.2) by pointwise Jacobi sweeps over
//     the stage grid held in shared memory (or a global scratch slab when the
//     stage does not fit);
//   phase C (float64): S_i <- S_i - alpha Delta s_i into the other buffer.
// Convergence bookkeeping (per-instance status, iteration counter, norms) is
// kept on the device so that a chunk of iterations can be replayed as a CUDA
// graph without host involvement.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace nmpc_dev {

struct InstDev {
  int dim, mx, my, ng;
  int N, nu, act_off, pad;
  long long s_off;  // offset of stage 1 in packed x / lam
  long long u_off;  // offset in packed u
  long long g_off;  // offset in packed x0 / ref
  double h, q, r, qf, gamma, k0, k1, b0, cx, cy;
};

enum { MODE_SOLVE = 0, MODE_ONESHOT = 1 };
enum { ST_RUNNING = 0, ST_CONVERGED = 1, ST_DIVERGED = 2, ST_MAX_ITER = 3 };
enum { NUM_WORK_ARRAYS = 8 };

struct IterArgs {
  const InstDev* inst;
  const int2* work;  // (instance, 0-based stage)
  int n_work;
  int n_inst;
  const int* act;
  const double* x0;
  const double* ref;
  // state buffers: solve mode reads [k & 1] and writes [(k + 1) & 1];
  // one-shot mode reads [0] and writes [1]
  const double* xin[2];
  const double* uin[2];
  const double* lin[2];
  double* xout[2];
  double* uout[2];
  double* lout[2];
  // control (solve mode)
  int* iter_k;
  int* block_done;
  unsigned long long* res_inf;  // [3][n_inst] bit patterns of non-negative doubles
  double* res_sq;               // [3][n_inst]
  unsigned long long* res_first;// [n_inst] ||K(S^0)||_inf
  int* status;
  int* iters;
  int* final_buf;
  double* fin_inf;
  double* fin_2;
  int* n_active;
  double tol, div_limit, alpha;
  int max_iter, n_lo, n_u_it;
  int resid_only;  // one-shot: residual norms only
  // lower-layer work arrays: shared memory (scratch == nullptr) or a global
  // slab of scratch_stride bytes per CTA
  char* scratch;
  long long scratch_stride;
  int ng_max;
};

__device__ __forceinline__ double phi_k(double w, double k0, double k1) {
  return k0 * (w + 0.5 * k1 * w * w);
}

__device__ __forceinline__ double sanitize_abs(double v) {
  double a = fabs(v);
  return (a <= 1.79e308) ? a : CUDART_INF;  // NaN and Inf count as +Inf
}

// Sum of the four (or two) stencil neighbours, each weighted by its axis
// coefficient; cells outside the interior grid are zero (Dirichlet ring).
template <typename V, typename Getter>
__device__ __forceinline__ V nbr_sum(int c, int ix, int iy, int mx, int my, V cx, V cy,
                                     Getter g) {
  V sx = V(0), sy = V(0);
  if (ix > 0) sx += g(c - 1);
  if (ix < mx - 1) sx += g(c + 1);
  if (iy > 0) sy += g(c - mx);
  if (iy < my - 1) sy += g(c + mx);
  return cx * sx + cy * sy;
}

template <typename T>
__device__ __forceinline__ T act_sum(int c, int nu, const int* act_s, const T* v) {
  T s = T(0);
  for (int a = 0; a < nu; ++a)
    if (act_s[a] == c) s += v[a];
  return s;
}

struct BlockRed {
  double mx[32];
  double sq[32];
};

__device__ __forceinline__ void block_reduce_store(double vmax, double vsq, BlockRed* red,
                                                   double* out_max, double* out_sq) {
  for (int o = 16; o > 0; o >>= 1) {
    vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    vsq += __shfl_xor_sync(0xffffffffu, vsq, o);
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red->mx[wid] = vmax;
    red->sq[wid] = vsq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0, s = 0.0;
    int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) {
      m = fmax(m, red->mx[w]);
      s += red->sq[w];
    }
    *out_max = m;
    *out_sq = s;
  }
}

// Shared-memory layout of one work item: small per-stage arrays first, then
// (in shared-memory mode) the NUM_WORK_ARRAYS work arrays of ng_max T each.
template <typename T>
struct SmallShared {
  BlockRed red;
  double red_out[2];
  double u[64];
  T b3[64];
  T v3[64];
  int act[64];
  int skip;
};

template <typename T>
__device__ void process_item(const IterArgs& A, int b, int s, int k, int rd, bool resid_only,
                             SmallShared<T>& sm, T* wk) {
  const InstDev I = A.inst[b];
  const int ng = I.ng, mx = I.mx, my = I.my, nu = I.nu, N = I.N;
  const long long so = I.s_off + (long long)s * ng;
  const double* __restrict__ X = A.xin[rd];
  const double* __restrict__ L = A.lin[rd];
  const double* __restrict__ Uin = A.uin[rd];
  const double* __restrict__ x0 = A.x0 + I.g_off;
  const double* __restrict__ ref = A.ref + I.g_off;
  const double h = I.h, cx = I.cx, cy = I.cy, k0 = I.k0, k1 = I.k1, b0 = I.b0;
  const double dcoef = 2.0 * (cx + cy);
  const bool last = (s == N - 1);

  T* b1 = wk;
  T* b2 = wk + ng;
  T* dp = wk + 2 * ng;
  T* ax = wk + 3 * ng;
  T* va = wk + 4 * ng;
  T* vb = wk + 5 * ng;
  T* wa = wk + 6 * ng;
  T* wb = wk + 7 * ng;

  for (int a = threadIdx.x; a < nu; a += blockDim.x) {
    sm.act[a] = A.act[I.act_off + a];
    sm.u[a] = Uin[I.u_off + (long long)s * nu + a];
  }
  __syncthreads();

  // ---- phase A: K_i (eq. 9) in float64, coefficient fields, norms ----
  double vmax = 0.0, vsq = 0.0;
  for (int c = threadIdx.x; c < ng; c += blockDim.x) {
    const int ix = c % mx, iy = c / mx;
    const double x = X[so + c];
    const double lam = L[so + c];
    const double xp = (s == 0) ? x0[c] : X[so - ng + c];
    const double ln = last ? h * I.qf * (x - ref[c]) : L[so + ng + c];
    const double* Xs = X + so;
    const double* Ls = L + so;
    const double nphi = nbr_sum<double>(c, ix, iy, mx, my, cx, cy,
                                        [&](int m) { return phi_k(Xs[m], k0, k1); });
    const double lphi = nphi - dcoef * phi_k(x, k0, k1);
    const double nlam = nbr_sum<double>(c, ix, iy, mx, my, cx, cy, [&](int m) { return Ls[m]; });
    const double mu = nlam - dcoef * lam;  // (Lap lambda)_c
    const double src = b0 * act_sum<double>(c, nu, sm.act, sm.u);
    const double dphi = k0 * (1.0 + k1 * x);
    const double K1 = xp - x + h * (lphi + src);
    const double K3 = ln - lam + h * (I.q * (x - ref[c]) + dphi * mu);
    double a1 = sanitize_abs(K1), a3 = sanitize_abs(K3);
    vmax = fmax(vmax, fmax(a1, a3));
    vsq += K1 * K1 + K3 * K3;
    if (!resid_only) {
      b1[c] = (T)K1;
      b2[c] = (T)K3;
      dp[c] = (T)dphi;
      ax[c] = (T)(h * (I.q + k0 * k1 * mu) + (last ? h * I.qf : 0.0));
    }
  }
  for (int a = threadIdx.x; a < nu; a += blockDim.x) {
    const double K2 = h * (I.r * sm.u[a] + b0 * L[so + sm.act[a]]);
    vmax = fmax(vmax, sanitize_abs(K2));
    vsq += K2 * K2;
    sm.b3[a] = (T)K2;
    sm.v3[a] = T(0);
  }
  block_reduce_store(vmax, vsq, &sm.red, &sm.red_out[0], &sm.red_out[1]);
  if (threadIdx.x == 0) {
    const int slot = (k % 3) * A.n_inst + b;
    atomicMax(&A.res_inf[slot], (unsigned long long)__double_as_longlong(sm.red_out[0]));
    atomicAdd(&A.res_sq[slot], sm.red_out[1]);
    if (k == 0 && A.res_first)
      atomicMax(&A.res_first[b], (unsigned long long)__double_as_longlong(sm.red_out[0]));
  }
  if (resid_only) {
    __syncthreads();
    return;
  }
  __syncthreads();

  // ---- phase B: lower layer in T ----
  const T th = (T)h, tcx = (T)cx, tcy = (T)cy, tb0 = (T)b0;
  const T tdc = (T)dcoef;
  const T auu = (T)(h * I.r + I.gamma);
  const int n_lo = A.n_lo;
  T* y5 = va;  // final buffers of the two Jacobi solves (set below)
  T* y4 = wa;
  for (int it = 0; it <= A.n_u_it; ++it) {
    // Y(v3) = P^{-1}(F_u v3 - b1, -b2): F_x v5 = c4 by n_lo sweeps from zero
    T* cur = va;
    T* nxt = vb;
    for (int c = threadIdx.x; c < ng; c += blockDim.x) {
      const T c4 = -b1[c] + th * tb0 * act_sum<T>(c, nu, sm.act, sm.v3);
      const T d = -T(1) - th * tdc * dp[c];
      cur[c] = c4 / d;
    }
    __syncthreads();
    for (int sw = 1; sw < n_lo; ++sw) {
      for (int c = threadIdx.x; c < ng; c += blockDim.x) {
        const int ix = c % mx, iy = c / mx;
        const T c4 = -b1[c] + th * tb0 * act_sum<T>(c, nu, sm.act, sm.v3);
        const T d = -T(1) - th * tdc * dp[c];
        const T off = th * nbr_sum<T>(c, ix, iy, mx, my, tcx, tcy,
                                      [&](int m) { return dp[m] * cur[m]; });
        nxt[c] = (c4 - off) / d;
      }
      __syncthreads();
      T* t = cur; cur = nxt; nxt = t;
    }
    y5 = cur;
    // F_x^T v4 = -b2 - A_xx v5 by n_lo sweeps from zero
    T* wc = (y5 == va) ? wa : wa;  // wa/wb are free
    T* wn = wb;
    for (int c = threadIdx.x; c < ng; c += blockDim.x) {
      const T e = -b2[c] - ax[c] * y5[c];
      const T d = -T(1) - th * tdc * dp[c];
      wc[c] = e / d;
    }
    __syncthreads();
    for (int sw = 1; sw < n_lo; ++sw) {
      for (int c = threadIdx.x; c < ng; c += blockDim.x) {
        const int ix = c % mx, iy = c / mx;
        const T e = -b2[c] - ax[c] * y5[c];
        const T d = -T(1) - th * tdc * dp[c];
        const T off = th * dp[c] * nbr_sum<T>(c, ix, iy, mx, my, tcx, tcy,
                                              [&](int m) { return wc[m]; });
        wn[c] = (e - off) / d;
      }
      __syncthreads();
      T* t = wc; wc = wn; wn = t;
    }
    y4 = wc;
    if (it < A.n_u_it) {
      // A_uu v3 = b3 + F_u^T y_lambda (A_ux = 0)
      __syncthreads();
      for (int a = threadIdx.x; a < nu; a += blockDim.x)
        sm.v3[a] = (sm.b3[a] + th * tb0 * y4[sm.act[a]]) / auu;
      __syncthreads();
    }
  }
  // back-solve (eq. 23b): (v1, v2) = P^{-1}(b1 - F_u v3, b2) = -Y(v3)

  // ---- phase C: S_i <- S_i - alpha Delta s_i (float64) ----
  const double alpha = A.alpha;
  double* Xo = A.xout[rd ^ 1];
  double* Lo = A.lout[rd ^ 1];
  double* Uo = A.uout[rd ^ 1];
  for (int c = threadIdx.x; c < ng; c += blockDim.x) {
    Xo[so + c] = X[so + c] + alpha * (double)y5[c];
    Lo[so + c] = L[so + c] + alpha * (double)y4[c];
  }
  for (int a = threadIdx.x; a < nu; a += blockDim.x)
    Uo[I.u_off + (long long)s * nu + a] = sm.u[a] - alpha * (double)sm.v3[a];
  __syncthreads();
}

template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_iterate(IterArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallShared<T>& sm = *reinterpret_cast<SmallShared<T>*>(smem_raw);
  T* wk;
  if (A.scratch == nullptr) {
    size_t off = (sizeof(SmallShared<T>) + 15) & ~size_t(15);
    wk = reinterpret_cast<T*>(smem_raw + off);
  } else {
    wk = reinterpret_cast<T*>(A.scratch + (long long)blockIdx.x * A.scratch_stride);
  }
  const int k = (MODE == MODE_SOLVE) ? *(volatile int*)A.iter_k : 0;

  for (int w = blockIdx.x; w < A.n_work; w += gridDim.x) {
    const int2 item = A.work[w];
    const int b = item.x, s = item.y;
    bool resid_only = (MODE == MODE_ONESHOT) ? (A.resid_only != 0) : false;
    if (MODE == MODE_SOLVE) {
      if (threadIdx.x == 0) {
        int skip = 0;
        if (k > A.max_iter || A.status[b] != ST_RUNNING) {
          skip = 1;
        } else if (k > 0) {
          const int pslot = ((k - 1) % 3) * A.n_inst + b;
          const double r = __longlong_as_double((long long)A.res_inf[pslot]);
          const double r0 = __longlong_as_double((long long)A.res_first[b]);
          int st = ST_RUNNING;
          if (r <= A.tol) st = ST_CONVERGED;
          else if (!(r <= 1.79e308) || r > A.div_limit * fmax(r0, 1e-300)) st = ST_DIVERGED;
          if (st != ST_RUNNING) {
            skip = 1;
            if (s == 0) {
              A.status[b] = st;
              A.iters[b] = k - 1;
              A.final_buf[b] = (k - 1) & 1;
              A.fin_inf[b] = r;
              A.fin_2[b] = sqrt(A.res_sq[pslot]);
              atomicSub(A.n_active, 1);
            }
          }
        }
        if (!skip && s == 0) {
          const int nslot = ((k + 1) % 3) * A.n_inst + b;
          A.res_inf[nslot] = 0ull;
          A.res_sq[nslot] = 0.0;
        }
        sm.skip = skip;
      }
      __syncthreads();
      if (sm.skip) {
        __syncthreads();
        continue;
      }
      resid_only = (k == A.max_iter);
    }
    process_item<T>(A, b, s, k, (MODE == MODE_SOLVE) ? (k & 1) : 0, resid_only, sm, wk);
  }

  if (MODE == MODE_SOLVE) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const int d = atomicAdd(A.block_done, 1);
      if (d == (int)gridDim.x - 1) {
        *A.block_done = 0;
        *A.iter_k = k + 1;
        __threadfence();
      }
    }
  }
}

// Reset the per-instance control and write S^0 (cold start) into buffer 0.
__global__ void k_init_control(IterArgs A, int cold) {
  const int b = blockIdx.y;
  if (b >= A.n_inst) return;
  const InstDev I = A.inst[b];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int q = 0; q < 3; ++q) {
      A.res_inf[q * A.n_inst + b] = 0ull;
      A.res_sq[q * A.n_inst + b] = 0.0;
    }
    A.res_first[b] = 0ull;
    A.status[b] = ST_RUNNING;
    A.iters[b] = 0;
    A.final_buf[b] = 0;
    A.fin_inf[b] = 0.0;
    A.fin_2[b] = 0.0;
    if (b == 0) {
      *A.n_active = A.n_inst;
      *A.iter_k = 0;
      *A.block_done = 0;
    }
  }
  if (!cold) return;
  const long long n = (long long)I.N * I.ng;
  double* X = A.xout[0];
  double* L = A.lout[0];
  double* U = A.uout[0];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    X[I.s_off + e] = A.x0[I.g_off + (e % I.ng)];
    L[I.s_off + e] = 0.0;
  }
  const long long nu_all = (long long)I.N * I.nu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nu_all;
       e += (long long)gridDim.x * blockDim.x)
    U[I.u_off + e] = 0.0;
}

// After the iteration chunks: settle instances still running at max_iter,
// gather every instance's returned iterate into the "current" buffers and
// u_out.  src[0]/src[1] are the ping-pong buffers.
struct FinalArgs {
  const InstDev* inst;
  int n_inst;
  const double* xs[2];
  const double* us[2];
  const double* ls[2];
  double* xc;
  double* uc;
  double* lc;
  double* u_out;
  int* status;
  int* iters;
  int* final_buf;
  double* fin_inf;
  double* fin_2;
  const unsigned long long* res_inf;
  const double* res_sq;
  double tol;
  int max_iter;
};

__global__ void k_finalize_status(FinalArgs F) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= F.n_inst) return;
  if (F.status[b] == ST_RUNNING) {
    const int slot = (F.max_iter % 3) * F.n_inst + b;
    const double r = __longlong_as_double((long long)F.res_inf[slot]);
    F.status[b] = (r <= F.tol) ? ST_CONVERGED : ((r <= 1.79e308) ? ST_MAX_ITER : ST_DIVERGED);
    F.iters[b] = F.max_iter;
    F.final_buf[b] = F.max_iter & 1;
    F.fin_inf[b] = r;
    F.fin_2[b] = sqrt(F.res_sq[slot]);
  }
}

__global__ void k_gather_final(FinalArgs F) {
  const int b = blockIdx.y;
  if (b >= F.n_inst) return;
  const InstDev I = F.inst[b];
  const int fb = F.final_buf[b];
  const long long n = (long long)I.N * I.ng;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    F.xc[I.s_off + e] = F.xs[fb][I.s_off + e];
    F.lc[I.s_off + e] = F.ls[fb][I.s_off + e];
  }
  const long long nu_all = (long long)I.N * I.nu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nu_all;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = F.us[fb][I.u_off + e];
    F.uc[I.u_off + e] = v;
    if (F.u_out) F.u_out[I.u_off + e] = v;
  }
}

// weights override: (q, r, qf) per instance from a device array
__global__ void k_set_weights(InstDev* inst, int n_inst, const double* w) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_inst) return;
  inst[b].q = w[3 * b + 0];
  inst[b].r = w[3 * b + 1];
  inst[b].qf = w[3 * b + 2];
}

}  // namespace nmpc_dev
