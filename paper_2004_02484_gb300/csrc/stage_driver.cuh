// The upper-layer driver shared by the stage-per-CTA solvers (the pinned-
// actuator plate and the second-order wave): per iteration k the problem's
// direction kernel(s) publish ||K(S^k)||_inf, ||K(S^k)||_2^2 and the largest
// admissible step (eq. 11) per instance and store Delta S; k_update then
// takes the convergence decision (Table 2's rule ||K||_inf <= tol) and forms
// S^{k+1} = S^k - alpha Delta S.  Start iterates (cold, warm, shifted by one
// stage), the returned iterate and the host loops of a solve and of a fixed
// number of iterations live here too.
//
// Arrays are packed per instance: x, lambda [sum N nx] stage-major, u
// [sum N nu] stage-major, x0 [sum nx].  Control words come in two slots,
// one per iteration parity, so that iteration k+1's direction kernels can
// accumulate while iteration k's decision is still being read.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/nmpc.h"

namespace stage_drv {

enum { ST_RUNNING = 0, ST_CONVERGED = 1, ST_DIVERGED = 2, ST_MAX_ITER = 3 };
enum { MODE_SOLVE = 0, MODE_ONESHOT = 1 };

struct Layout {
  int N, nx, nu;     // stages, state entries per stage, inputs per stage
  long long s_off;   // packed x, lambda: stage 1 of this instance
  long long u_off;   // packed u
  long long g_off;   // packed x0
  double u_cold;     // the cold start's input
};

struct Ctl {
  const Layout* lay;
  const int2* work;            // (instance, stage), one CTA each
  unsigned long long* rmax;    // [2][n] bits of ||K||_inf (non-negative doubles order as integers)
  double* rsq;                 // [2][n] ||K||_2^2
  unsigned long long* acand;   // [2][n] bits of the admissible step
  int* status;
  int* iters;
  int* final_buf;
  double* fin;                 // [2][n] final (||K||_inf, ||K||_2)
  int* n_active;
  int n_inst, k, mode, max_iter;
  double tol;
};

struct Iter {
  const double* xin;
  const double* uin;
  const double* lin;
  double* xout;
  double* uout;
  double* lout;
  double* dx;  // direction Delta S
  double* du;
  double* dl;
};

// max that keeps a NaN once one has been seen (fmax would drop it)
__device__ __forceinline__ double nan_max(double a, double b) {
  return (a != a || b != b) ? CUDART_NAN : fmax(a, b);
}

// Block reduction of (max, sum) over nthreads threads (a multiple of 32);
// thread 0 holds the result.  red: 64 doubles of shared memory.
__device__ inline void block_max_sum(double& mx, double& sq, double* red, int nthreads) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    mx = nan_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
  }
  if (lane == 0) {
    red[w] = mx;
    red[32 + w] = sq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < nthreads / 32; ++i) {
      mx = nan_max(mx, red[i]);
      sq += red[32 + i];
    }
  }
  __syncthreads();
}

// A direction CTA of instance b has nothing to do (the instance has stopped).
__device__ __forceinline__ bool finished(const Ctl& C, int b) {
  return C.mode == MODE_SOLVE && C.status[b] != ST_RUNNING;
}

// Thread 0's block norms into the instance's slot of iteration k; true when
// the iteration only evaluates the norms (the last one a solve allows).
__device__ __forceinline__ bool publish_norms(const Ctl& C, int b, double mx, double sq) {
  if (threadIdx.x == 0) {
    const int slot = (C.k & 1) * C.n_inst + b;
    atomicMax(&C.rmax[slot], (unsigned long long)__double_as_longlong(mx));
    atomicAdd(&C.rsq[slot], sq);
  }
  return C.mode == MODE_SOLVE && C.k >= C.max_iter;
}

// A warp's smallest admissible step (amin in (0, 1]) into the instance's slot.
__device__ __forceinline__ void publish_step(const Ctl& C, int b, double amin) {
  for (int o = 16; o > 0; o >>= 1) amin = fmin(amin, __shfl_xor_sync(0xffffffffu, amin, o));
  if ((threadIdx.x & 31) == 0 && amin < 1.0)
    atomicMin(&C.acand[(C.k & 1) * C.n_inst + b], (unsigned long long)__double_as_longlong(amin));
}

// The decision of iteration k and S^{k+1} = S^k - alpha Delta S, one CTA
// per (instance, stage).
// (static: each translation unit that includes this header has its own copy)
static __global__ void __launch_bounds__(256) k_update(Ctl C, Iter S) {
  const int2 it = C.work[blockIdx.x];
  const int b = it.x, s = it.y;
  const Layout L = C.lay[b];
  const int slot = (C.k & 1) * C.n_inst + b;
  bool stop = false;
  double r = 0.0;
  if (C.mode == MODE_SOLVE) {
    if (C.status[b] != ST_RUNNING) return;  // finished before this kernel
    r = __longlong_as_double((long long)C.rmax[slot]);
    stop = !(r <= 1.79e308) || r <= C.tol || C.k >= C.max_iter;
  }
  if (s == 0 && threadIdx.x == 0) {
    const int nslot = ((C.k + 1) & 1) * C.n_inst + b;
    C.rmax[nslot] = 0ull;
    C.rsq[nslot] = 0.0;
    C.acand[nslot] = (unsigned long long)__double_as_longlong(1.0);
  }
  if (stop) {
    if (s == 0 && threadIdx.x == 0) {
      C.status[b] = !(r <= 1.79e308) ? ST_DIVERGED : (r <= C.tol ? ST_CONVERGED : ST_MAX_ITER);
      C.iters[b] = C.k;
      C.final_buf[b] = C.k & 1;
      C.fin[b] = r;
      C.fin[C.n_inst + b] = sqrt(C.rsq[slot]);
      atomicSub(C.n_active, 1);
    }
    return;
  }
  const double alpha = fmin(1.0, __longlong_as_double((long long)C.acand[slot]));
  const long long so = L.s_off + (long long)s * L.nx;
  const long long uo = L.u_off + (long long)s * L.nu;
  for (int t = threadIdx.x; t < L.nx; t += blockDim.x) {
    S.xout[so + t] = S.xin[so + t] - alpha * S.dx[so + t];
    S.lout[so + t] = S.lin[so + t] - alpha * S.dl[so + t];
  }
  for (int a = threadIdx.x; a < L.nu; a += blockDim.x)
    S.uout[uo + a] = S.uin[uo + a] - alpha * S.du[uo + a];
}

// Start iterate into buffer 0 (mode 0 cold, 1 a copy of the current state,
// 2 the current state shifted by one stage, the last repeated) and the
// control words.  Grid (x, instances).
static __global__ void k_init(const Layout* lay, int n_inst, int mode, const double* x0,
                              const double* xc, const double* uc, const double* lc, double* x,
                              double* u, double* lam, unsigned long long* rmax, double* rsq,
                              unsigned long long* acand, int* status, int* n_active) {
  const int b = blockIdx.y;
  const Layout L = lay[b];
  const long long nxs = (long long)L.N * L.nx, nus = (long long)L.N * L.nu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nxs;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / L.nx), t = (int)(e - (long long)s * L.nx);
    const int ss = (mode == 2) ? min(s + 1, L.N - 1) : s;
    const long long src = L.s_off + (long long)ss * L.nx + t;
    x[L.s_off + e] = (mode == 0) ? x0[L.g_off + t] : xc[src];
    lam[L.s_off + e] = (mode == 0) ? 0.0 : lc[src];
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nus;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / L.nu), a = (int)(e - (long long)s * L.nu);
    const int ss = (mode == 2) ? min(s + 1, L.N - 1) : s;
    u[L.u_off + e] = (mode == 0) ? L.u_cold : uc[L.u_off + (long long)ss * L.nu + a];
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
static __global__ void k_gather(const Layout* lay, const int* final_buf, const double* x0b,
                                const double* x1b, const double* u0b, const double* u1b,
                                const double* l0b, const double* l1b, double* xc, double* uc,
                                double* lc, double* u_out) {
  const int b = blockIdx.y;
  const Layout L = lay[b];
  const int fb = final_buf[b];
  const double* xs = fb ? x1b : x0b;
  const double* us = fb ? u1b : u0b;
  const double* ls = fb ? l1b : l0b;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)L.N * L.nx;
       e += (long long)gridDim.x * blockDim.x) {
    xc[L.s_off + e] = xs[L.s_off + e];
    lc[L.s_off + e] = ls[L.s_off + e];
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)L.N * L.nu;
       e += (long long)gridDim.x * blockDim.x) {
    uc[L.u_off + e] = us[L.u_off + e];
    if (u_out) u_out[L.u_off + e] = us[L.u_off + e];
  }
}

#define SDRV_CHECK(call)                                                    \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      fprintf(stderr, "nmpc: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      return NMPC_ERR_CUDA;                                                 \
    }                                                                       \
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

// Device state of the driver: three iterate buffers (two ping-pong, one
// current state), the direction, the control words and the instance layout.
struct Driver {
  int n = 0;
  std::vector<Layout> lay_h;
  long long n_g = 0, n_x = 0, n_u = 0;  // sum nx (x0), sum N nx, sum N nu
  Layout* lay = nullptr;
  int2* work = nullptr;
  int n_work = 0;
  double* x0 = nullptr;  // the solve's start state [n_g]
  double* xb[3] = {nullptr, nullptr, nullptr};
  double* ub[3] = {nullptr, nullptr, nullptr};
  double* lb[3] = {nullptr, nullptr, nullptr};
  double *dx = nullptr, *du = nullptr, *dl = nullptr;
  unsigned long long *rmax = nullptr, *acand = nullptr;
  double *rsq = nullptr, *fin = nullptr;
  int *status = nullptr, *iters = nullptr, *final_buf = nullptr, *n_active = nullptr;
  bool has_state = false;
};

// Offsets from lay_h[b].{N, nx, nu}; one work item per (instance, stage).
inline cudaError_t driver_alloc(Driver& d) {
  d.n = (int)d.lay_h.size();
  d.n_g = d.n_x = d.n_u = 0;
  std::vector<int2> work;
  for (int b = 0; b < d.n; ++b) {
    Layout& L = d.lay_h[b];
    L.s_off = d.n_x;
    L.u_off = d.n_u;
    L.g_off = d.n_g;
    d.n_x += (long long)L.N * L.nx;
    d.n_u += (long long)L.N * L.nu;
    d.n_g += L.nx;
    for (int s = 0; s < L.N; ++s) work.push_back(make_int2(b, s));
  }
  d.n_work = (int)work.size();
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(dalloc(&d.lay, d.n));
  A(dalloc(&d.work, work.size()));
  A(dalloc(&d.x0, d.n_g));
  for (int q = 0; q < 3; ++q) {
    A(dalloc(&d.xb[q], d.n_x));
    A(dalloc(&d.ub[q], d.n_u));
    A(dalloc(&d.lb[q], d.n_x));
  }
  A(dalloc(&d.dx, d.n_x));
  A(dalloc(&d.du, d.n_u));
  A(dalloc(&d.dl, d.n_x));
  A(dalloc(&d.rmax, 2 * d.n));
  A(dalloc(&d.acand, 2 * d.n));
  A(dalloc(&d.rsq, 2 * d.n));
  A(dalloc(&d.fin, 2 * d.n));
  A(dalloc(&d.status, d.n));
  A(dalloc(&d.iters, d.n));
  A(dalloc(&d.final_buf, d.n));
  A(dalloc(&d.n_active, 1));
  A(upload(d.lay, d.lay_h));
  A(upload(d.work, work));
  return e;
}

inline void driver_free(Driver& d) {
  void* ptrs[] = {d.lay, d.work, d.x0, d.xb[0], d.xb[1], d.xb[2], d.ub[0], d.ub[1], d.ub[2],
                  d.lb[0], d.lb[1], d.lb[2], d.dx, d.du, d.dl, d.rmax, d.acand, d.rsq, d.fin,
                  d.status, d.iters, d.final_buf, d.n_active};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

inline Ctl make_ctl(const Driver& d, int k, int mode, int max_iter, double tol) {
  Ctl C{};
  C.lay = d.lay;
  C.work = d.work;
  C.rmax = d.rmax;
  C.rsq = d.rsq;
  C.acand = d.acand;
  C.status = d.status;
  C.iters = d.iters;
  C.final_buf = d.final_buf;
  C.fin = d.fin;
  C.n_active = d.n_active;
  C.n_inst = d.n;
  C.k = k;
  C.mode = mode;
  C.max_iter = max_iter;
  C.tol = tol;
  return C;
}

inline Iter make_iter(const Driver& d, int rd) {
  Iter S{};
  S.xin = d.xb[rd];
  S.uin = d.ub[rd];
  S.lin = d.lb[rd];
  S.xout = d.xb[rd ^ 1];
  S.uout = d.ub[rd ^ 1];
  S.lout = d.lb[rd ^ 1];
  S.dx = d.dx;
  S.du = d.du;
  S.dl = d.dl;
  return S;
}

inline dim3 inst_grid(const Driver& d) { return dim3(8, (unsigned)d.n); }

// One iteration: the problem's direction kernel(s), dir(C, S) -> cudaError_t,
// then the update.
template <class Dir>
cudaError_t launch_iteration(const Driver& d, const Ctl& C, const Iter& S, Dir& dir,
                             cudaStream_t st) {
  cudaError_t e = dir(C, S);
  if (e != cudaSuccess) return e;
  k_update<<<d.n_work, 256, 0, st>>>(C, S);
  return cudaGetLastError();
}

// A solve from d.x0 (already on the device): init NMPC_INIT_*; host polls of
// the running count every check_every iterations.  Fills stats (host, [n])
// and u_out (device or NULL); returns NMPC_OK or the first of NOT_CONVERGED /
// DIVERGED met.
template <class Dir>
int solve(Driver& d, int init, int max_iter, double tol, int check_every, Dir& dir, double* u_out,
          nmpc_stats* stats, cudaStream_t st) {
  if (init != NMPC_INIT_COLD && init != NMPC_INIT_WARM && init != NMPC_INIT_SHIFT)
    return NMPC_ERR_BAD_ARG;
  if (init != NMPC_INIT_COLD && !d.has_state) return NMPC_ERR_BAD_ARG;
  const int mode = init == NMPC_INIT_COLD ? 0 : (init == NMPC_INIT_WARM ? 1 : 2);
  k_init<<<inst_grid(d), 256, 0, st>>>(d.lay, d.n, mode, d.x0, d.xb[2], d.ub[2], d.lb[2], d.xb[0],
                                       d.ub[0], d.lb[0], d.rmax, d.rsq, d.acand, d.status,
                                       d.n_active);
  SDRV_CHECK(cudaGetLastError());
  int active = d.n;
  for (int k = 0; k <= max_iter;) {
    for (int c = 0; c < check_every && k <= max_iter; ++c, ++k)
      SDRV_CHECK(launch_iteration(d, make_ctl(d, k, MODE_SOLVE, max_iter, tol), make_iter(d, k & 1),
                                  dir, st));
    SDRV_CHECK(cudaMemcpyAsync(&active, d.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    SDRV_CHECK(cudaStreamSynchronize(st));
    if (active == 0) break;
  }
  k_gather<<<inst_grid(d), 256, 0, st>>>(d.lay, d.final_buf, d.xb[0], d.xb[1], d.ub[0], d.ub[1],
                                         d.lb[0], d.lb[1], d.xb[2], d.ub[2], d.lb[2], u_out);
  SDRV_CHECK(cudaGetLastError());
  d.has_state = true;
  std::vector<int> status(d.n), iters(d.n);
  std::vector<double> fin(2 * d.n);
  SDRV_CHECK(cudaMemcpyAsync(status.data(), d.status, d.n * sizeof(int), cudaMemcpyDeviceToHost, st));
  SDRV_CHECK(cudaMemcpyAsync(iters.data(), d.iters, d.n * sizeof(int), cudaMemcpyDeviceToHost, st));
  SDRV_CHECK(cudaMemcpyAsync(fin.data(), d.fin, 2 * d.n * sizeof(double), cudaMemcpyDeviceToHost, st));
  SDRV_CHECK(cudaStreamSynchronize(st));
  int rc = NMPC_OK;
  for (int b = 0; b < d.n; ++b) {
    if (stats) {
      stats[b].status = status[b];
      stats[b].iters = iters[b];
      stats[b].res_inf = fin[b];
      stats[b].res_2 = fin[d.n + b];
      stats[b].f64_iters = iters[b] + 1;  // every residual is evaluated in float64
    }
    if (rc == NMPC_OK) {
      if (status[b] == ST_DIVERGED) rc = NMPC_ERR_DIVERGED;
      else if (status[b] != ST_CONVERGED) rc = NMPC_ERR_NOT_CONVERGED;
    }
  }
  return rc;
}

// n_iter iterations from (x_in, u_in, lam_in) (device, packed) into the
// output arrays, no convergence test; out: NULL or host [n][3] = (||K||_inf,
// ||K||_2, alpha) of the last iteration.
template <class Dir>
int iterate(Driver& d, const double* x_in, const double* u_in, const double* lam_in, double* x_out,
            double* u_out, double* lam_out, int n_iter, double* out, Dir& dir, cudaStream_t st) {
  SDRV_CHECK(cudaMemcpyAsync(d.xb[0], x_in, d.n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDRV_CHECK(cudaMemcpyAsync(d.ub[0], u_in, d.n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDRV_CHECK(cudaMemcpyAsync(d.lb[0], lam_in, d.n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double one = 1.0;
  unsigned long long one_bits;
  std::memcpy(&one_bits, &one, sizeof(one_bits));
  std::vector<unsigned long long> aone(2 * d.n, one_bits);
  for (int it = 0; it < n_iter; ++it) {
    // slot 0 of the control words serves every iteration
    SDRV_CHECK(cudaMemsetAsync(d.rmax, 0, 2 * d.n * sizeof(unsigned long long), st));
    SDRV_CHECK(cudaMemsetAsync(d.rsq, 0, 2 * d.n * sizeof(double), st));
    SDRV_CHECK(cudaMemcpyAsync(d.acand, aone.data(), aone.size() * sizeof(unsigned long long),
                               cudaMemcpyHostToDevice, st));
    SDRV_CHECK(launch_iteration(d, make_ctl(d, 0, MODE_ONESHOT, 0, 0.0), make_iter(d, it & 1), dir,
                                st));
    SDRV_CHECK(cudaStreamSynchronize(st));  // aone outlives the copy
  }
  const int fb = n_iter & 1;
  SDRV_CHECK(cudaMemcpyAsync(x_out, d.xb[fb], d.n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDRV_CHECK(cudaMemcpyAsync(u_out, d.ub[fb], d.n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDRV_CHECK(cudaMemcpyAsync(lam_out, d.lb[fb], d.n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (out) {
    std::vector<unsigned long long> rm(d.n), ac(d.n);
    std::vector<double> rs(d.n);
    SDRV_CHECK(cudaMemcpyAsync(rm.data(), d.rmax, d.n * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, st));
    SDRV_CHECK(cudaMemcpyAsync(rs.data(), d.rsq, d.n * sizeof(double), cudaMemcpyDeviceToHost, st));
    SDRV_CHECK(cudaMemcpyAsync(ac.data(), d.acand, d.n * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, st));
    SDRV_CHECK(cudaStreamSynchronize(st));
    for (int b = 0; b < d.n; ++b) {
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

inline int get_state(const Driver& d, double* x, double* u, double* lam, cudaStream_t st) {
  if (x) SDRV_CHECK(cudaMemcpyAsync(x, d.xb[2], d.n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (u) SDRV_CHECK(cudaMemcpyAsync(u, d.ub[2], d.n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (lam) SDRV_CHECK(cudaMemcpyAsync(lam, d.lb[2], d.n_x * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return NMPC_OK;
}

// Row p of the grid Laplacian (dim 1 or 2, m points per axis) as (column,
// weight) pairs: zero Neumann by mirrored fictitious points (a missing
// neighbour is replaced by the inner one, so that neighbour's weight
// doubles; the points include the boundary, spacing 1/(m-1)), zero Dirichlet
// by dropping neighbours outside (interior points, spacing 1/(m+1)).
inline void laplacian_rows(int dim, int m, int bc,
                           std::vector<std::vector<std::pair<int, double>>>& rows) {
  const int ng = dim == 2 ? m * m : m;
  const double dp = bc == 0 ? 1.0 / (m - 1) : 1.0 / (m + 1);
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
          if (bc == 1) continue;  // Dirichlet: zero outside
          j = i - dir;            // Neumann: the mirrored point
        }
        add(p, axis == 0 ? iy * m + j : j * m + ix, w);
      }
    }
  }
}

// ELL tables (ELL entries per point; unused slots: the point itself with
// weight 0) of L and L^T, and the diagonal of L, appended to the vectors.
constexpr int ELL = 5;
inline void append_ell(int dim, int m, int bc, std::vector<int>& Lc, std::vector<double>& Lv,
                       std::vector<int>& Ltc, std::vector<double>& Ltv, std::vector<double>& Ld) {
  std::vector<std::vector<std::pair<int, double>>> rows;
  laplacian_rows(dim, m, bc, rows);
  const int ng = (int)rows.size();
  std::vector<std::vector<std::pair<int, double>>> trows(ng);
  for (int p = 0; p < ng; ++p)
    for (auto& e : rows[p]) trows[e.first].push_back({p, e.second});
  for (int p = 0; p < ng; ++p) {
    double diag = 0.0;
    for (int e = 0; e < ELL; ++e) {
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
}

}  // namespace stage_drv
