// Second-order-in-time solver (include/nmpc_wave.h): the double-layer method
// on a w_tt + b w_t = c Lap w - kappa w^3 + point forces (Sec. 2, eq. 1 with
// a != 0), state x = (W, V = dW/dt) (eq. 5).
//
// One iteration is two kernels (three with the red-black upper layer):
//   k_wave_dir  one CTA per (instance, stage) loads the stage's W, V,
//     lambda_W, lambda_V into shared memory, evaluates K_i (eq. 9) and its
//     norms, the stage's coefficients, and the lower layer (eqs. 21-24 with
//     the u-iteration of Sec. 5.2) whose F_x and F_x^T solves eliminate v6
//     (eq. 25): E v7 = b7 + h grad_W g b6 and E^T v9 = b9 + h b8 by n_lo
//     pointwise Jacobi sweeps, v6 = h v7 - b6, v8 = h grad_W g^T v9 - b8.
//     It stores the direction Delta s_i.  Red-black: half 0 runs the even
//     stages, half 1 the odd ones with the even neighbours' directions in
//     its right-hand side (eq. 18's form).
//   k_update (stage_driver.cuh)  the convergence decision and S^{k+1} =
//     S^k - Delta S (no bounds: the full step).
// grad_W g = (c L - 3 kappa diag(W^2)) / a and grad_V g = -(b / a) I, so E
// has the stencil of L scaled by h^2 c / a off the diagonal.  The Laplacian
// and its transpose are host-built tables of five (column, weight) entries
// per point.  Everything is float64.
#include <new>

#include "../../include/nmpc_wave.h"
#include "stage_driver.cuh"

namespace wave_dev {

using stage_drv::Ctl;
using stage_drv::ELL;
using stage_drv::Iter;
using stage_drv::Layout;
constexpr int THREADS = 256;
constexpr int MAX_NU = 64;
// shared-memory fields of n_g values in k_wave_dir: float64 grid values and
// costates, the lower layer's fields in its type T
constexpr int F64_FIELDS = 4, T_FIELDS = 18;
constexpr int NG_PER_THREAD = (NMPC_WAVE_MAX_POINTS + THREADS - 1) / THREADS;  // the plant's points

struct WInst {
  int dim, m, ng, nu, N;
  long long w_off;  // w_ref
  long long a_off;  // u_ref, actuator table
  long long t_off;  // per-point tables
  double h, a, b, c, kappa, gain, q, qv, r, qf, gamma;
};

struct WArgs {
  const WInst* inst;
  const int* act_of;  // [sum ng]: actuator index at the point, or -1
  const int* act_pt;  // [sum nu]: grid point of actuator a
  const int* Lc;      // [sum ng][ELL] columns of L (unused slots: the point itself, weight 0)
  const double* Lv;
  const int* Ltc;     // the same for L^T
  const double* Ltv;
  const double* Ld;   // [sum ng] L[p][p]
  const float* Lvf;   // float32 copies of Lv, Ltv, Ld (mixed precision)
  const float* Ltvf;
  const float* Ldf;
  const double* x0;
  const double* wref;
  const double* uref;
  int n_lo, n_u_it, rb, half;
};

// The lower layer runs in T: float64, or float32 in mixed precision (the
// residual, the coefficients and the update stay float64, so the fixed point
// is the float64 root); WT holds W in T for the lower layer's products.
template <typename T>
struct Fields {
  double *W, *V, *LW, *LV;
  T *WT, *ED, *AXW, *K1W, *K1V, *K3W, *K3V;
  T *B6, *B7, *B8, *B9, *T_, *C0, *C1, *Y6, *Y7, *Y8, *Y9;
};

template <typename V>
struct Stencil {
  const int *Lc, *Ltc;
  const V *Lv, *Ltv, *Ld;
  __device__ V lap(const V* v, int p) const {  // (L v)(p)
    V acc = V(0);
#pragma unroll
    for (int e = 0; e < ELL; ++e) acc += Lv[p * ELL + e] * v[Lc[p * ELL + e]];
    return acc;
  }
  __device__ V lapT(const V* v, int p) const {  // (L^T v)(p)
    V acc = V(0);
#pragma unroll
    for (int e = 0; e < ELL; ++e) acc += Ltv[p * ELL + e] * v[Ltc[p * ELL + e]];
    return acc;
  }
};

// The stencil tables in type V.
template <typename V>
__device__ __forceinline__ const V* tab(const double* d, const float* f);
template <>
__device__ __forceinline__ const double* tab<double>(const double* d, const float*) { return d; }
template <>
__device__ __forceinline__ const float* tab<float>(const double*, const float* f) { return f; }

// n_lo Jacobi sweeps from zero on E v = T (transposed: E^T), result in the
// returned buffer (C0 or C1).  E = diag ED + (h^2 c / a)(L - diag L).
template <typename T>
__device__ T* jacobi_E(const WArgs& A, const WInst& I, const Stencil<T>& L, const Fields<T>& f,
                       bool transposed) {
  const int ng = I.ng;
  const T s = (T)(I.h * I.h * I.c / I.a);
  T* cur = f.C0;
  T* nxt = f.C1;
  for (int p = threadIdx.x; p < ng; p += THREADS) cur[p] = f.T_[p] / f.ED[p];
  __syncthreads();
  for (int sw = 1; sw < A.n_lo; ++sw) {
    for (int p = threadIdx.x; p < ng; p += THREADS) {
      const T lv = transposed ? L.lapT(cur, p) : L.lap(cur, p);
      nxt[p] = (f.T_[p] - s * (lv - L.Ld[p] * cur[p])) / f.ED[p];
    }
    __syncthreads();
    T* t = cur;
    cur = nxt;
    nxt = t;
  }
  return cur;
}

// P^{-1} (eq. 24): F_x (Y6, Y7) = (B6, B7), then F_x^T (Y8, Y9) = (B8, B9) -
// A_xx (Y6, Y7), both by the v6 elimination (eq. 25).  B8 is overwritten.
template <typename T>
__device__ void p_inv(const WArgs& A, const WInst& I, const Stencil<T>& L, const Fields<T>& f) {
  const int ng = I.ng;
  const T h = (T)I.h, ia = (T)(1.0 / I.a), axv = (T)(I.h * I.qv), c = (T)I.c;
  const T k3 = (T)(3.0 * I.kappa);
  // E v7 = b7 + h grad_W g b6
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    const T gw = (c * L.lap(f.B6, p) - k3 * f.WT[p] * f.WT[p] * f.B6[p]) * ia;
    f.T_[p] = f.B7[p] + h * gw;
  }
  __syncthreads();
  const T* v7 = jacobi_E<T>(A, I, L, f, false);
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    f.Y7[p] = v7[p];
    f.Y6[p] = h * v7[p] - f.B6[p];
  }
  __syncthreads();
  // (b8, b9) = (B8, B9) - A_xx (Y6, Y7); E^T v9 = b9 + h b8
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    const T b8 = f.B8[p] - f.AXW[p] * f.Y6[p];
    f.B8[p] = b8;
    f.T_[p] = (f.B9[p] - axv * f.Y7[p]) + h * b8;
  }
  __syncthreads();
  const T* v9 = jacobi_E<T>(A, I, L, f, true);
  for (int p = threadIdx.x; p < ng; p += THREADS) f.Y9[p] = v9[p];
  __syncthreads();
  // v8 = h grad_W g^T v9 - b8
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    const T gwt = (c * L.lapT(f.Y9, p) - k3 * f.WT[p] * f.WT[p] * f.Y9[p]) * ia;
    f.Y8[p] = h * gwt - f.B8[p];
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(THREADS) k_wave_dir(WArgs A, Ctl C, Iter S) {
  const int2 it = C.work[blockIdx.x];
  const int b = it.x, s = it.y;
  if (A.rb && ((s & 1) != A.half)) return;
  if (stage_drv::finished(C, b)) return;
  const WInst I = A.inst[b];
  const Layout Ly = C.lay[b];
  const int ng = I.ng, nu = I.nu, nx = 2 * ng;
  const bool last = (s == I.N - 1);
  extern __shared__ double smem[];
  Fields<T> f;
  {
    double** fd[F64_FIELDS] = {&f.W, &f.V, &f.LW, &f.LV};
    for (int q = 0; q < F64_FIELDS; ++q) *fd[q] = smem + (size_t)q * ng;
    T* base = reinterpret_cast<T*>(smem + (size_t)F64_FIELDS * ng);
    T** ft[T_FIELDS] = {&f.WT, &f.ED, &f.AXW, &f.K1W, &f.K1V, &f.K3W, &f.K3V, &f.B6, &f.B7,
                        &f.B8, &f.B9, &f.T_,  &f.C0,  &f.C1,  &f.Y6,  &f.Y7,  &f.Y8, &f.Y9};
    for (int q = 0; q < T_FIELDS; ++q) *ft[q] = base + (size_t)q * ng;
  }
  __shared__ double sU[MAX_NU], red[64];
  __shared__ T sK2[MAX_NU], sV3[MAX_NU];
  // the residual's stencil (float64) and the lower layer's (T)
  Stencil<double> L{A.Lc + I.t_off * ELL, A.Ltc + I.t_off * ELL, A.Lv + I.t_off * ELL,
                    A.Ltv + I.t_off * ELL, A.Ld + I.t_off};
  Stencil<T> LT{A.Lc + I.t_off * ELL, A.Ltc + I.t_off * ELL,
                tab<T>(A.Lv, A.Lvf) + I.t_off * ELL, tab<T>(A.Ltv, A.Ltvf) + I.t_off * ELL,
                tab<T>(A.Ld, A.Ldf) + I.t_off};
  const int* act_of = A.act_of + I.t_off;
  const int* apt = A.act_pt + I.a_off;
  const long long so = Ly.s_off + (long long)s * nx;
  const long long uo = Ly.u_off + (long long)s * nu;
  const double h = I.h, ia = 1.0 / I.a;

  for (int p = threadIdx.x; p < ng; p += THREADS) {
    f.W[p] = S.xin[so + p];
    f.V[p] = S.xin[so + ng + p];
    f.LW[p] = S.lin[so + p];
    f.LV[p] = S.lin[so + ng + p];
  }
  for (int a = threadIdx.x; a < nu; a += THREADS) sU[a] = S.uin[uo + a];
  __syncthreads();

  // K_i (eq. 9), coefficients, norms
  double mx = 0.0, sq = 0.0;
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    const double w = f.W[p], v = f.V[p], lw = f.LW[p], lv = f.LV[p];
    const double wr = A.wref[I.w_off + p];
    const int ap = act_of[p];
    const double force = ap >= 0 ? I.gain * sU[ap] : 0.0;
    const double g = (I.c * L.lap(f.W, p) - I.b * v - I.kappa * w * w * w + force) * ia;
    const double wprev = (s == 0) ? A.x0[Ly.g_off + p] : S.xin[so - nx + p];
    const double vprev = (s == 0) ? A.x0[Ly.g_off + ng + p] : S.xin[so - nx + ng + p];
    const double lwn = last ? h * I.qf * (w - wr) : S.lin[so + nx + p];
    const double lvn = last ? 0.0 : S.lin[so + nx + ng + p];
    const double ltv = L.lapT(f.LV, p);  // (L^T lambda_V)(p)
    const double K1W = wprev - w + h * v;
    const double K1V = vprev - v + h * g;
    const double K3W = lwn - lw + h * (I.q * (w - wr) + (I.c * ltv - 3.0 * I.kappa * w * w * lv) * ia);
    const double K3V = lvn - lv + h * (I.qv * v + lw - I.b * ia * lv);
    mx = stage_drv::nan_max(mx, stage_drv::nan_max(stage_drv::nan_max(fabs(K1W), fabs(K1V)),
                                                   stage_drv::nan_max(fabs(K3W), fabs(K3V))));
    sq += K1W * K1W + K1V * K1V + K3W * K3W + K3V * K3V;
    // red-black half 1: the right-hand side takes the even neighbours'
    // directions (state rows: M_L Delta x_{i-1}; costate rows: M_U Delta
    // lambda_{i+1}); the norms above stay those of K(S^k)
    double k1w = K1W, k1v = K1V, k3w = K3W, k3v = K3V;
    if (A.rb && A.half == 1) {
      if (s > 0) {
        k1w -= S.dx[so - nx + p];
        k1v -= S.dx[so - nx + ng + p];
      }
      if (!last) {
        k3w -= S.dl[so + nx + p];
        k3v -= S.dl[so + nx + ng + p];
      }
    }
    f.K1W[p] = (T)k1w;
    f.K1V[p] = (T)k1v;
    f.K3W[p] = (T)k3w;
    f.K3V[p] = (T)k3v;
    f.WT[p] = (T)w;
    // E's diagonal: h grad_V g - 1 + h^2 grad_W g at (p, p)
    f.ED[p] = (T)(-(1.0 + h * I.b * ia) + h * h * (I.c * L.Ld[p] - 3.0 * I.kappa * w * w) * ia);
    f.AXW[p] = (T)(h * (I.q - 6.0 * I.kappa * w * lv * ia) + (last ? h * I.qf : 0.0));
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nu; a += THREADS) {
    const double K2 = h * (I.r * (sU[a] - A.uref[I.a_off + a]) + I.gain * ia * f.LV[apt[a]]);
    mx = stage_drv::nan_max(mx, fabs(K2));
    sq += K2 * K2;
    sK2[a] = (T)K2;
    sV3[a] = T(0);
  }
  __syncthreads();
  stage_drv::block_max_sum(mx, sq, red, THREADS);
  if (stage_drv::publish_norms(C, b, mx, sq)) return;  // norms only

  // u fixed-point iteration (Sec. 5.2): y = P^{-1}(F_u v3 - b1, -b2),
  // v3 = (b3 + F_u^T y_lambda) / A_uu from v3 = 0, then the final
  // P^{-1}(b1 - F_u v3, b2).  F_u = [0; h B / a]; A_uu = h r + gamma.
  const T fu = (T)(h * I.gain * ia), auu = (T)(h * I.r + I.gamma);
  for (int itu = 0; itu <= A.n_u_it; ++itu) {
    const bool final_pass = (itu == A.n_u_it);
    for (int p = threadIdx.x; p < ng; p += THREADS) {
      const int ap = act_of[p];
      const T fuv = ap >= 0 ? fu * sV3[ap] : T(0);
      f.B6[p] = final_pass ? f.K1W[p] : -f.K1W[p];
      f.B7[p] = final_pass ? f.K1V[p] - fuv : fuv - f.K1V[p];
      f.B8[p] = final_pass ? f.K3W[p] : -f.K3W[p];
      f.B9[p] = final_pass ? f.K3V[p] : -f.K3V[p];
    }
    __syncthreads();
    p_inv<T>(A, I, LT, f);
    if (final_pass) break;
    for (int a = threadIdx.x; a < nu; a += THREADS) sV3[a] = (sK2[a] + fu * f.Y9[apt[a]]) / auu;
    __syncthreads();
  }
  // direction (Delta x, Delta u, Delta lambda) = (v5, v3, v4)
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    S.dx[so + p] = (double)f.Y6[p];
    S.dx[so + ng + p] = (double)f.Y7[p];
    S.dl[so + p] = (double)f.Y8[p];
    S.dl[so + ng + p] = (double)f.Y9[p];
  }
  for (int a = threadIdx.x; a < nu; a += THREADS) S.du[uo + a] = (double)sV3[a];
}

// The plant (Sec. 5.3): the true system x = (W, V) (device [sum 2 n_g], in
// place) advances by n_sub symplectic Euler steps of tau = dt / n_sub (dt < 0:
// each instance's own stage length h) with the inputs at the first-stage
// values u1 of the current state: V <- V + tau g(W, V, u1), then W <- W + tau
// V.  One CTA per instance; W, V and the forces in shared memory.
__global__ void __launch_bounds__(THREADS) k_wave_plant(WArgs A, const Layout* lay, double* x,
                                                        const double* uc, double dt, int n_sub) {
  const int b = blockIdx.x;
  const WInst I = A.inst[b];
  const Layout Ly = lay[b];
  const int ng = I.ng;
  extern __shared__ double smem[];
  double* W = smem;
  double* V = W + ng;
  double* F = V + ng;
  Stencil<double> L{A.Lc + I.t_off * ELL, A.Ltc + I.t_off * ELL, A.Lv + I.t_off * ELL,
                    A.Ltv + I.t_off * ELL, A.Ld + I.t_off};
  const int* act_of = A.act_of + I.t_off;
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    W[p] = x[Ly.g_off + p];
    V[p] = x[Ly.g_off + ng + p];
    const int ap = act_of[p];
    F[p] = ap >= 0 ? I.gain * uc[Ly.u_off + ap] : 0.0;
  }
  __syncthreads();
  const double tau = (dt < 0.0 ? I.h : dt) / n_sub, ia = 1.0 / I.a;
  for (int k = 0; k < n_sub; ++k) {
    double vn[NG_PER_THREAD];
    int cnt = 0;
    for (int p = threadIdx.x; p < ng; p += THREADS, ++cnt) {
      const double w = W[p];
      const double g = (I.c * L.lap(W, p) - I.b * V[p] - I.kappa * w * w * w + F[p]) * ia;
      vn[cnt] = V[p] + tau * g;
    }
    __syncthreads();
    cnt = 0;
    for (int p = threadIdx.x; p < ng; p += THREADS, ++cnt) {
      V[p] = vn[cnt];
      W[p] += tau * vn[cnt];
    }
    __syncthreads();
  }
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    x[Ly.g_off + p] = W[p];
    x[Ly.g_off + ng + p] = V[p];
  }
}

}  // namespace wave_dev

using wave_dev::WArgs;
using wave_dev::WInst;

struct nmpc_wave {
  nmpc_wave_opts opts{};
  std::vector<WInst> inst_h;
  stage_drv::Driver drv;
  long long n_a = 0, n_w = 0;  // sum n_u, sum n_g
  int ng_max = 0;
  WInst* inst_d = nullptr;
  int *act_of = nullptr, *act_pt = nullptr, *Lc = nullptr, *Ltc = nullptr;
  double *Lv = nullptr, *Ltv = nullptr, *Ld = nullptr;
  float *Lvf = nullptr, *Ltvf = nullptr, *Ldf = nullptr;
  double *wref = nullptr, *uref = nullptr;
  size_t smem = 0;
};

namespace {

void free_wave(nmpc_wave* h) {
  stage_drv::driver_free(h->drv);
  void* ptrs[] = {h->inst_d, h->act_of, h->act_pt, h->Lc, h->Ltc, h->Lv, h->Ltv, h->Ld, h->Lvf,
                  h->Ltvf, h->Ldf, h->wref, h->uref};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

int validate(const nmpc_wave_desc& d) {
  if ((d.dim != 1 && d.dim != 2) || d.horizon < 1 || d.n_u < 1 || !d.act_cell) return NMPC_ERR_BAD_ARG;
  if (d.bc != 0 && d.bc != 1) return NMPC_ERR_BAD_ARG;
  if (d.m < (d.bc == 0 ? 3 : 1)) return NMPC_ERR_BAD_ARG;
  const long long ng = d.dim == 2 ? (long long)d.m * d.m : d.m;
  if (ng > NMPC_WAVE_MAX_POINTS || d.n_u > wave_dev::MAX_NU) return NMPC_ERR_UNSUPPORTED;
  std::vector<char> seen(ng, 0);
  for (int a = 0; a < d.n_u; ++a) {
    if (d.act_cell[a] < 0 || d.act_cell[a] >= ng || seen[d.act_cell[a]]) return NMPC_ERR_BAD_ARG;
    seen[d.act_cell[a]] = 1;
  }
  if (!(d.h > 0) || !(d.a > 0) || !std::isfinite(d.b) || !std::isfinite(d.c) ||
      !std::isfinite(d.kappa) || !std::isfinite(d.gain) || !(d.q >= 0) || !(d.qv >= 0) ||
      !(d.r > 0) || !(d.qf >= 0) || !(d.gamma >= 0))
    return NMPC_ERR_BAD_ARG;
  return NMPC_OK;
}

WArgs make_args(const nmpc_wave* h) {
  WArgs A{};
  A.inst = h->inst_d;
  A.act_of = h->act_of;
  A.act_pt = h->act_pt;
  A.Lc = h->Lc;
  A.Lv = h->Lv;
  A.Ltc = h->Ltc;
  A.Ltv = h->Ltv;
  A.Ld = h->Ld;
  A.Lvf = h->Lvf;
  A.Ltvf = h->Ltvf;
  A.Ldf = h->Ldf;
  A.x0 = h->drv.x0;
  A.wref = h->wref;
  A.uref = h->uref;
  A.n_lo = h->opts.n_lo;
  A.n_u_it = h->opts.n_u_it;
  A.rb = (h->opts.variant == NMPC_VARIANT_REDBLACK) ? 1 : 0;
  return A;
}

struct WaveDir {
  const nmpc_wave* h;
  cudaStream_t st;
  cudaError_t operator()(const stage_drv::Ctl& C, const stage_drv::Iter& S) const {
    WArgs A = make_args(h);
    for (int half = 0; half < (A.rb ? 2 : 1); ++half) {
      A.half = half;
      if (h->opts.precision == NMPC_MIXED)
        wave_dev::k_wave_dir<float><<<h->drv.n_work, wave_dev::THREADS, h->smem, st>>>(A, C, S);
      else
        wave_dev::k_wave_dir<double><<<h->drv.n_work, wave_dev::THREADS, h->smem, st>>>(A, C, S);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
};

int copy_problem(nmpc_wave* h, const double* x0, const double* w_ref, const double* u_ref,
                 cudaStream_t st) {
  SDRV_CHECK(cudaMemcpyAsync(h->drv.x0, x0, h->drv.n_g * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDRV_CHECK(cudaMemcpyAsync(h->wref, w_ref, h->n_w * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDRV_CHECK(cudaMemcpyAsync(h->uref, u_ref, h->n_a * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return NMPC_OK;
}

}  // namespace

extern "C" {

void nmpc_wave_default_opts(nmpc_wave_opts* o) {
  if (!o) return;
  o->tol = 1e-6;
  o->max_iter = 5000;
  o->n_lo = 2;
  o->n_u_it = 2;
  o->variant = NMPC_VARIANT_JACOBI;
  o->check_every = 16;
  o->precision = NMPC_FP64;
}

int nmpc_wave_setup(const nmpc_wave_desc* descs, int n, const nmpc_wave_opts* opts, nmpc_wave** out) {
  if (!descs || n < 1 || !out) return NMPC_ERR_BAD_ARG;
  *out = nullptr;
  nmpc_wave_opts o;
  nmpc_wave_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol >= 0) || o.max_iter < 0 || o.n_lo < 1 || o.n_u_it < 0 || o.check_every < 1 ||
      (o.variant != NMPC_VARIANT_JACOBI && o.variant != NMPC_VARIANT_REDBLACK) ||
      (o.precision != NMPC_FP64 && o.precision != NMPC_MIXED))
    return NMPC_ERR_BAD_ARG;
  for (int b = 0; b < n; ++b) {
    const int rc = validate(descs[b]);
    if (rc != NMPC_OK) return rc;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return NMPC_ERR_NO_DEVICE;
  nmpc_wave* h = new (std::nothrow) nmpc_wave();
  if (!h) return NMPC_ERR_CUDA;
  h->opts = o;
  std::vector<int> act_of, act_pt, Lc, Ltc;
  std::vector<double> Lv, Ltv, Ld;
  long long n_pts = 0;
  for (int b = 0; b < n; ++b) {
    const nmpc_wave_desc& d = descs[b];
    WInst I{};
    I.dim = d.dim;
    I.m = d.m;
    I.ng = d.dim == 2 ? d.m * d.m : d.m;
    I.nu = d.n_u;
    I.N = d.horizon;
    I.w_off = h->n_w;
    I.a_off = h->n_a;
    I.t_off = n_pts;
    I.h = d.h;
    I.a = d.a;
    I.b = d.b;
    I.c = d.c;
    I.kappa = d.kappa;
    I.gain = d.gain;
    I.q = d.q;
    I.qv = d.qv;
    I.r = d.r;
    I.qf = d.qf;
    I.gamma = d.gamma;
    std::vector<int> ao(I.ng, -1);
    for (int a = 0; a < d.n_u; ++a) ao[d.act_cell[a]] = a;
    act_of.insert(act_of.end(), ao.begin(), ao.end());
    for (int a = 0; a < d.n_u; ++a) act_pt.push_back(d.act_cell[a]);
    stage_drv::append_ell(d.dim, d.m, d.bc == 0 ? 0 : 1, Lc, Lv, Ltc, Ltv, Ld);
    stage_drv::Layout L{};
    L.N = I.N;
    L.nx = 2 * I.ng;
    L.nu = I.nu;
    L.u_cold = 0.0;
    h->drv.lay_h.push_back(L);
    h->n_a += I.nu;
    h->n_w += I.ng;
    n_pts += I.ng;
    h->ng_max = std::max(h->ng_max, I.ng);
    h->inst_h.push_back(I);
  }
  const size_t tsz = o.precision == NMPC_MIXED ? sizeof(float) : sizeof(double);
  h->smem = (size_t)h->ng_max * (wave_dev::F64_FIELDS * sizeof(double) + wave_dev::T_FIELDS * tsz);
  cudaError_t e = stage_drv::driver_alloc(h->drv);
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(stage_drv::dalloc(&h->inst_d, n));
  A(stage_drv::dalloc(&h->act_of, act_of.size()));
  A(stage_drv::dalloc(&h->act_pt, act_pt.size()));
  A(stage_drv::dalloc(&h->Lc, Lc.size()));
  A(stage_drv::dalloc(&h->Ltc, Ltc.size()));
  A(stage_drv::dalloc(&h->Lv, Lv.size()));
  A(stage_drv::dalloc(&h->Ltv, Ltv.size()));
  A(stage_drv::dalloc(&h->Ld, Ld.size()));
  A(stage_drv::dalloc(&h->wref, h->n_w));
  A(stage_drv::dalloc(&h->uref, h->n_a));
  A(stage_drv::upload(h->inst_d, h->inst_h));
  A(stage_drv::upload(h->act_of, act_of));
  A(stage_drv::upload(h->act_pt, act_pt));
  A(stage_drv::upload(h->Lc, Lc));
  A(stage_drv::upload(h->Ltc, Ltc));
  A(stage_drv::upload(h->Lv, Lv));
  A(stage_drv::upload(h->Ltv, Ltv));
  A(stage_drv::upload(h->Ld, Ld));
  {
    const std::vector<float> Lvf(Lv.begin(), Lv.end()), Ltvf(Ltv.begin(), Ltv.end()),
        Ldf(Ld.begin(), Ld.end());
    A(stage_drv::dalloc(&h->Lvf, Lvf.size()));
    A(stage_drv::dalloc(&h->Ltvf, Ltvf.size()));
    A(stage_drv::dalloc(&h->Ldf, Ldf.size()));
    A(stage_drv::upload(h->Lvf, Lvf));
    A(stage_drv::upload(h->Ltvf, Ltvf));
    A(stage_drv::upload(h->Ldf, Ldf));
  }
  if (h->smem > 48 * 1024) {
    A(cudaFuncSetAttribute(wave_dev::k_wave_dir<double>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem));
    A(cudaFuncSetAttribute(wave_dev::k_wave_dir<float>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem));
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "nmpc_wave_setup: %s\n", cudaGetErrorString(e));
    free_wave(h);
    delete h;
    return NMPC_ERR_CUDA;
  }
  *out = h;
  return NMPC_OK;
}

int nmpc_wave_sizes(const nmpc_wave* h, int64_t* out) {
  if (!h || !out) return NMPC_ERR_BAD_ARG;
  out[0] = h->drv.n_g;
  out[1] = h->drv.n_x;
  out[2] = h->drv.n_u;
  out[3] = h->n_a;
  out[4] = h->n_w;
  return NMPC_OK;
}

int nmpc_wave_solve(nmpc_wave* h, const double* x0, const double* w_ref, const double* u_ref,
                    int init, double* u_out, nmpc_stats* stats, void* stream) {
  if (!h || !x0 || !w_ref || !u_ref) return NMPC_ERR_BAD_ARG;
  if (init != NMPC_INIT_COLD && init != NMPC_INIT_WARM && init != NMPC_INIT_SHIFT)
    return NMPC_ERR_BAD_ARG;
  if (init != NMPC_INIT_COLD && !h->drv.has_state) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = copy_problem(h, x0, w_ref, u_ref, st);
  if (rc != NMPC_OK) return rc;
  WaveDir dir{h, st};
  return stage_drv::solve(h->drv, init, h->opts.max_iter, h->opts.tol, h->opts.check_every, dir,
                          u_out, stats, st);
}

int nmpc_wave_iterate(nmpc_wave* h, const double* x0, const double* w_ref, const double* u_ref,
                      const double* x_in, const double* u_in, const double* lam_in, double* x_out,
                      double* u_out, double* lam_out, int n_iter, double* out, void* stream) {
  if (!h || !x0 || !w_ref || !u_ref || !x_in || !u_in || !lam_in || !x_out || !u_out || !lam_out ||
      n_iter < 1)
    return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = copy_problem(h, x0, w_ref, u_ref, st);
  if (rc != NMPC_OK) return rc;
  WaveDir dir{h, st};
  return stage_drv::iterate(h->drv, x_in, u_in, lam_in, x_out, u_out, lam_out, n_iter, out, dir, st);
}

int nmpc_wave_get_state(nmpc_wave* h, double* x, double* u, double* lam, void* stream) {
  if (!h) return NMPC_ERR_BAD_ARG;
  return stage_drv::get_state(h->drv, x, u, lam, (cudaStream_t)stream);
}

namespace {
int plant(nmpc_wave* h, double* x, double dt, int n_sub, void* stream) {
  wave_dev::k_wave_plant<<<h->drv.n, wave_dev::THREADS, 3 * h->ng_max * sizeof(double),
                           (cudaStream_t)stream>>>(make_args(h), h->drv.lay, x, h->drv.ub[2], dt,
                                                   n_sub);
  SDRV_CHECK(cudaGetLastError());
  return NMPC_OK;
}
}  // namespace

int nmpc_wave_plant_step(nmpc_wave* h, double* x, double dt, int n_sub, void* stream) {
  if (!h || !x || !(dt >= 0) || n_sub < 1 || !h->drv.has_state) return NMPC_ERR_BAD_ARG;
  return plant(h, x, dt, n_sub, stream);
}

int nmpc_wave_closed_loop(nmpc_wave* h, double* x, const double* w_ref, const double* u_ref,
                          int steps, int n_sub, double* u_hist, int* iters_hist, double* res_hist,
                          void* stream) {
  if (!h || !x || !w_ref || !u_ref || steps < 1 || n_sub < 1) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = h->drv.n;
  std::vector<nmpc_stats> stats(n);
  int rc_all = NMPC_OK;
  for (int t = 0; t < steps; ++t) {
    const int init = (t == 0 && !h->drv.has_state) ? NMPC_INIT_COLD : NMPC_INIT_SHIFT;
    const int rc = nmpc_wave_solve(h, x, w_ref, u_ref, init, nullptr, stats.data(), stream);
    if (rc == NMPC_ERR_BAD_ARG || rc == NMPC_ERR_CUDA) return rc;
    if (rc != NMPC_OK && rc_all == NMPC_OK) rc_all = rc;
    for (int b = 0; b < n; ++b) {
      if (iters_hist) iters_hist[(size_t)t * n + b] = stats[b].iters;
      if (res_hist) res_hist[(size_t)t * n + b] = stats[b].res_inf;
    }
    if (u_hist) {
      // u_1 of every instance (stage 1 of the packed control trajectory)
      for (int b = 0; b < n; ++b) {
        const WInst& I = h->inst_h[b];
        SDRV_CHECK(cudaMemcpyAsync(u_hist + (size_t)t * h->n_a + I.a_off,
                                   h->drv.ub[2] + h->drv.lay_h[b].u_off, I.nu * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
      }
    }
    const int prc = plant(h, x, -1.0, n_sub, stream);  // each instance's own h
    if (prc != NMPC_OK) return prc;
  }
  return rc_all;
}

void nmpc_wave_destroy(nmpc_wave* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  free_wave(h);
  delete h;
}

}  // extern "C"
