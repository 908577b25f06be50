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
//   k_update (stage_driver.cuh)  per (instance, stage): the convergence
//     decision from ||K(S^k)||_inf (the whole instance's maximum, complete
//     once every stage's k_plate_dir has run) and otherwise S^{k+1} = S^k -
//     alpha_max Delta S.
// The Laplacian of the grid, with the mirrored fictitious points of the
// zero-Neumann condition (eqs. 2-3) or the zero Dirichlet ring, and its
// transpose are host-built tables of five (column, weight) entries per
// point.  Everything is float64.
#include <new>

#include "../../include/nmpc_plate.h"
#include "stage_driver.cuh"

namespace plate_dev {

using stage_drv::ELL;
using stage_drv::Ctl;
using stage_drv::Iter;
using stage_drv::Layout;
constexpr int THREADS = 256;
constexpr int MAX_NU = 64;

// Per instance: the grid and the model (packed x, u offsets are the
// driver's Layout; x0 and x_ref share its g_off).
struct PInst {
  int dim, m, ng, ns, nu, N;
  long long a_off;  // u_ref, actuator tables
  long long t_off;  // per-point tables
  double h, k0, k1, beta, ta, gr, q, r, qf, gamma, tau, ulo, uhi;
};

struct PArgs {
  const PInst* inst;
  const int* pt_state;  // [sum ng]: state index, or -1 - a for actuator a
  const int* act_pt;    // [sum nu]: grid point of actuator a
  const int* Lc;        // [sum ng][ELL] columns of L (unused slots: the point itself, weight 0)
  const double* Lv;
  const int* Ltc;       // the same for L^T
  const double* Ltv;
  const double* Ld;     // [sum ng] L[p][p]
  const float* Lvf;     // float32 copies of Lv, Ltv, Ld (mixed precision)
  const float* Ltvf;
  const float* Ldf;
  const double* x0;
  const double* xref;
  const double* uref;
  int n_lo, n_u_it, rb, half;
};

// The stencil tables in the lower layer's type T.
template <typename T>
__device__ __forceinline__ const T* tab(const double* d, const float* f);
template <>
__device__ __forceinline__ const double* tab<double>(const double* d, const float*) { return d; }
template <>
__device__ __forceinline__ const float* tab<float>(const double*, const float* f) { return f; }

__device__ __forceinline__ double phi(const PInst& I, double w) {
  return I.k0 * (w + 0.5 * I.k1 * w * w);
}
__device__ __forceinline__ double dphi(const PInst& I, double w) {
  return I.k0 * (1.0 + I.k1 * w);
}

// Sweeps of P^{-1} (eq. 24) over the state points of the stage grid:
// F_x v5 = b4, then F_x^T v4 = b5 - A_xx v5, n_lo pointwise Jacobi sweeps
// each from zero (Lemma 1).  F_x = h (L diag(Phi'(w)) - diag(beta + 4 gr x^3))
// - I on the state points; its off-diagonal part sums L[p][q] Phi'(w_q) v_q
// over the state neighbours q (v is zero at the actuator points).  The
// lower layer runs in T (float64, or float32 in mixed precision: the
// residual, the coefficients and the update stay float64, so the fixed
// point is the float64 root); the grid values and costates stay float64.
template <typename T>
struct Fields {
  double *W, *LB, *PH, *LTL;
  T *DP, *DG, *AX, *V, *V2, *B4, *B5, *K1, *K3, *Y4, *Y5, *Z;
};
constexpr int F64_FIELDS = 4, T_FIELDS = 12;  // shared memory: n_g values each

template <typename T>
__device__ void p_inv(const PArgs& A, const PInst& I, const Fields<T>& f, const int* pts) {
  const int ng = I.ng;
  const int* Lc = A.Lc + I.t_off * ELL;
  const T* Lv = tab<T>(A.Lv, A.Lvf) + I.t_off * ELL;
  const int* Ltc = A.Ltc + I.t_off * ELL;
  const T* Ltv = tab<T>(A.Ltv, A.Ltvf) + I.t_off * ELL;
  const T* Ld = tab<T>(A.Ld, A.Ldf) + I.t_off;
  const T h = (T)I.h;
  // F_x v5 = b4
  T* cur = f.V;
  T* nxt = f.V2;
  for (int p = threadIdx.x; p < ng; p += THREADS) cur[p] = (pts[p] >= 0) ? f.B4[p] / f.DG[p] : T(0);
  __syncthreads();
  for (int sw = 1; sw < A.n_lo; ++sw) {
    for (int p = threadIdx.x; p < ng; p += THREADS) {
      T v = T(0);
      if (pts[p] >= 0) {
        T off = T(0);
#pragma unroll
        for (int e = 0; e < ELL; ++e) {
          const int c = Lc[p * ELL + e];
          off += Lv[p * ELL + e] * f.DP[c] * cur[c];
        }
        off -= Ld[p] * f.DP[p] * cur[p];
        v = (f.B4[p] - h * off) / f.DG[p];
      }
      nxt[p] = v;
    }
    __syncthreads();
    T* t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int p = threadIdx.x; p < ng; p += THREADS) f.Y5[p] = cur[p];
  __syncthreads();
  // F_x^T v4 = b5 - A_xx v5; off-diagonal part h Phi'(x_p) sum_q L[q][p] v_q
  for (int p = threadIdx.x; p < ng; p += THREADS)
    cur[p] = (pts[p] >= 0) ? (f.B5[p] - f.AX[p] * f.Y5[p]) / f.DG[p] : T(0);
  __syncthreads();
  for (int sw = 1; sw < A.n_lo; ++sw) {
    for (int p = threadIdx.x; p < ng; p += THREADS) {
      T v = T(0);
      if (pts[p] >= 0) {
        T off = T(0);
#pragma unroll
        for (int e = 0; e < ELL; ++e) off += Ltv[p * ELL + e] * cur[Ltc[p * ELL + e]];
        off -= Ld[p] * cur[p];
        v = (f.B5[p] - f.AX[p] * f.Y5[p] - h * f.DP[p] * off) / f.DG[p];
      }
      nxt[p] = v;
    }
    __syncthreads();
    T* t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int p = threadIdx.x; p < ng; p += THREADS) f.Y4[p] = cur[p];
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(THREADS) k_plate_dir(PArgs A, Ctl C, Iter S) {
  const int2 it = C.work[blockIdx.x];
  const int b = it.x, s = it.y;
  if (A.rb && ((s & 1) != A.half)) return;
  if (stage_drv::finished(C, b)) return;
  const PInst I = A.inst[b];
  const Layout Ly = C.lay[b];
  const int ng = I.ng, ns = I.ns, nu = I.nu, N = I.N;
  const bool last = (s == N - 1);
  extern __shared__ double smem[];
  Fields<T> f;
  double* q = smem;
  f.W = q; q += ng;
  f.LB = q; q += ng;
  f.PH = q; q += ng;
  f.LTL = q; q += ng;
  T* qt = reinterpret_cast<T*>(q);
  f.DP = qt; qt += ng;
  f.DG = qt; qt += ng;
  f.AX = qt; qt += ng;
  f.V = qt; qt += ng;
  f.V2 = qt; qt += ng;
  f.B4 = qt; qt += ng;
  f.B5 = qt; qt += ng;
  f.K1 = qt; qt += ng;
  f.K3 = qt; qt += ng;
  f.Y4 = qt; qt += ng;
  f.Y5 = qt; qt += ng;
  f.Z = qt; qt += ng;
  __shared__ double red[64];
  __shared__ T sK2[MAX_NU], sAUU[MAX_NU], sV3[MAX_NU];
  const int* pts = A.pt_state + I.t_off;
  const int* apt = A.act_pt + I.a_off;
  const int* Lc = A.Lc + I.t_off * ELL;
  const double* Lv = A.Lv + I.t_off * ELL;
  const int* Ltc = A.Ltc + I.t_off * ELL;
  const double* Ltv = A.Ltv + I.t_off * ELL;
  const double* Ld = A.Ld + I.t_off;
  const T* LvT = tab<T>(A.Lv, A.Lvf) + I.t_off * ELL;
  const T* LtvT = tab<T>(A.Ltv, A.Ltvf) + I.t_off * ELL;
  const long long so = Ly.s_off + (long long)s * ns;
  const long long uo = Ly.u_off + (long long)s * nu;
  const double h = I.h;

  // the stage's grid: w = x (states) / u (actuators); lambda-bar
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    const int t = pts[p];
    double w, lb;
    if (t >= 0) {
      w = S.xin[so + t];
      lb = S.lin[so + t];
    } else {
      w = S.uin[uo + (-1 - t)];
      lb = 0.0;
    }
    f.W[p] = w;
    f.LB[p] = lb;
    f.PH[p] = phi(I, w);
    f.DP[p] = (T)dphi(I, w);
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
      f.K1[p] = f.K3[p] = T(0);
      f.DG[p] = T(1);
      f.AX[p] = T(0);
      continue;
    }
    const double x = f.W[p], lam = f.LB[p], xr = A.xref[Ly.g_off + t];
    const double xprev = (s == 0) ? A.x0[Ly.g_off + t] : S.xin[so - ns + t];
    const double lnext = last ? h * I.qf * (x - xr) : S.lin[so + ns + t];
    double lph = 0.0;
#pragma unroll
    for (int e = 0; e < ELL; ++e) lph += Lv[p * ELL + e] * f.PH[Lc[p * ELL + e]];
    const double x3 = x * x * x;
    const double fp = lph - I.beta * (x - I.ta) - I.gr * (x3 * x - I.ta * I.ta * I.ta * I.ta);
    const double K1 = xprev - x + h * fp;
    const double dpx = dphi(I, x);
    const double gxT = dpx * f.LTL[p] - (I.beta + 4.0 * I.gr * x3) * lam;
    const double K3 = lnext - lam + h * (I.q * (x - xr) + gxT);
    mx = stage_drv::nan_max(mx, stage_drv::nan_max(fabs(K1), fabs(K3)));
    sq += K1 * K1 + K3 * K3;
    // red-black half 1: the right-hand side takes the even neighbours'
    // directions (state rows: M_L Delta x_{i-1}; costate rows: M_U Delta
    // lambda_{i+1}); the norms above stay those of K(S^k)
    double K1r = K1, K3r = K3;
    if (A.rb && A.half == 1) {
      if (s > 0) K1r -= S.dx[so - ns + t];
      if (!last) K3r -= S.dl[so + ns + t];
    }
    f.K1[p] = (T)K1r;
    f.K3[p] = (T)K3r;
    f.DG[p] = (T)(h * (Ld[p] * dpx - I.beta - 4.0 * I.gr * x3) - 1.0);
    f.AX[p] = (T)(h * (I.q + d2p * f.LTL[p] - 12.0 * I.gr * x * x * lam) + (last ? h * I.qf : 0.0));
  }
  for (int a = threadIdx.x; a < nu; a += THREADS) {
    const int pa = apt[a];
    const double u = f.W[pa];
    double db = 0.0, d2b = 0.0;
    if (I.tau > 0.0) {
      db = -I.tau / (u - I.ulo) + I.tau / (I.uhi - u);
      d2b = I.tau / ((u - I.ulo) * (u - I.ulo)) + I.tau / ((I.uhi - u) * (I.uhi - u));
    }
    const double K2 = h * (I.r * (u - A.uref[I.a_off + a]) + db + dphi(I, u) * f.LTL[pa]);
    mx = stage_drv::nan_max(mx, fabs(K2));
    sq += K2 * K2;
    sK2[a] = (T)K2;
    sAUU[a] = (T)(h * (I.r + d2b + d2p * f.LTL[pa]) + I.gamma);
    sV3[a] = T(0);
  }
  __syncthreads();
  stage_drv::block_max_sum(mx, sq, red, THREADS);
  if (stage_drv::publish_norms(C, b, mx, sq)) return;  // norms only

  // u fixed-point iteration (Sec. 5.2): y = P^{-1}(F_u v3 - b1, -b2),
  // v3 = (b3 + F_u^T y_lambda) / A_uu, from v3 = 0
  const T hT = (T)h;
  for (int itu = 0; itu <= A.n_u_it; ++itu) {
    const bool final_pass = (itu == A.n_u_it);
    // Z = Phi'(u) v3 at the actuator points, zero elsewhere
    for (int p = threadIdx.x; p < ng; p += THREADS) f.Z[p] = T(0);
    __syncthreads();
    for (int a = threadIdx.x; a < nu; a += THREADS) f.Z[apt[a]] = f.DP[apt[a]] * sV3[a];
    __syncthreads();
    for (int p = threadIdx.x; p < ng; p += THREADS) {
      T fu = T(0);  // (F_u v3)(p) = h sum_a L[p][a] Phi'(u_a) v3_a
#pragma unroll
      for (int e = 0; e < ELL; ++e) fu += LvT[p * ELL + e] * f.Z[Lc[p * ELL + e]];
      fu *= hT;
      if (pts[p] >= 0) {
        f.B4[p] = final_pass ? f.K1[p] - fu : fu - f.K1[p];
        f.B5[p] = final_pass ? f.K3[p] : -f.K3[p];
      } else {
        f.B4[p] = f.B5[p] = T(0);
      }
    }
    __syncthreads();
    p_inv<T>(A, I, f, pts);
    if (final_pass) break;
    for (int a = threadIdx.x; a < nu; a += THREADS) {
      const int pa = apt[a];
      T acc = T(0);  // (L^T y_lambda)(a) over the state points
#pragma unroll
      for (int e = 0; e < ELL; ++e) acc += LtvT[pa * ELL + e] * f.Y4[Ltc[pa * ELL + e]];
      sV3[a] = (sK2[a] + hT * f.DP[pa] * acc) / sAUU[a];
    }
    __syncthreads();
  }
  // direction (Delta x, Delta u, Delta lambda) = (v5, v3, v4); admissible step
  for (int p = threadIdx.x; p < ng; p += THREADS) {
    const int t = pts[p];
    if (t >= 0) {
      S.dx[so + t] = (double)f.Y5[p];
      S.dl[so + t] = (double)f.Y4[p];
    }
  }
  double amin = 1.0;
  for (int a = threadIdx.x; a < nu; a += THREADS) {
    const double d = (double)sV3[a], u = f.W[apt[a]];
    S.du[uo + a] = d;
    if (I.tau > 0.0) {
      if (d > 0.0) amin = fmin(amin, 0.995 * (u - I.ulo) / d);
      if (d < 0.0) amin = fmin(amin, 0.995 * (I.uhi - u) / (-d));
    }
  }
  stage_drv::publish_step(C, b, amin);
}

// The plant: w (state points) += (dt / n_sub) f(w, u1), n_sub times, with the
// actuator points at the first-stage inputs u1 of the current state; dt < 0
// takes each instance's own stage length h.
__global__ void __launch_bounds__(THREADS) k_plate_plant(PArgs A, const Layout* lay, double* w,
                                                         const double* uc, double dt, int n_sub) {
  const int b = blockIdx.x;
  const PInst I = A.inst[b];
  const Layout Ly = lay[b];
  extern __shared__ double smem[];
  double* W = smem;
  double* PH = W + I.ng;
  const int* pts = A.pt_state + I.t_off;
  const int* Lc = A.Lc + I.t_off * ELL;
  const double* Lv = A.Lv + I.t_off * ELL;
  for (int p = threadIdx.x; p < I.ng; p += THREADS) {
    const int t = pts[p];
    W[p] = (t >= 0) ? w[Ly.g_off + t] : uc[Ly.u_off + (-1 - t)];
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
    if (t >= 0) w[Ly.g_off + t] = W[p];
  }
}

}  // namespace plate_dev

using plate_dev::PInst;
using plate_dev::PArgs;

struct nmpc_plate {
  nmpc_plate_opts opts{};
  std::vector<PInst> inst_h;
  stage_drv::Driver drv;     // iterates, direction, control words, layout
  long long n_a = 0;         // sum n_u
  int ng_max = 0;
  PInst* inst_d = nullptr;
  int *pt_state = nullptr, *act_pt = nullptr, *Lc = nullptr, *Ltc = nullptr;
  double *Lv = nullptr, *Ltv = nullptr, *Ld = nullptr;
  float *Lvf = nullptr, *Ltvf = nullptr, *Ldf = nullptr;
  double *xref = nullptr, *uref = nullptr;
  size_t smem = 0;
};

namespace {

void free_plate(nmpc_plate* h) {
  stage_drv::driver_free(h->drv);
  void* ptrs[] = {h->inst_d, h->pt_state, h->act_pt, h->Lc, h->Ltc, h->Lv, h->Ltv, h->Ld, h->Lvf,
                  h->Ltvf, h->Ldf, h->xref, h->uref};
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

PArgs make_args(const nmpc_plate* h) {
  PArgs A{};
  A.inst = h->inst_d;
  A.pt_state = h->pt_state;
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
  A.xref = h->xref;
  A.uref = h->uref;
  A.n_lo = h->opts.n_lo;
  A.n_u_it = h->opts.n_u_it;
  A.rb = (h->opts.variant == NMPC_VARIANT_REDBLACK) ? 1 : 0;
  return A;
}

// The direction kernels of one iteration: one launch, or the two red-black
// halves.
struct PlateDir {
  const nmpc_plate* h;
  cudaStream_t st;
  cudaError_t operator()(const stage_drv::Ctl& C, const stage_drv::Iter& S) const {
    PArgs A = make_args(h);
    for (int half = 0; half < (A.rb ? 2 : 1); ++half) {
      A.half = half;
      if (h->opts.precision == NMPC_MIXED)
        plate_dev::k_plate_dir<float><<<h->drv.n_work, plate_dev::THREADS, h->smem, st>>>(A, C, S);
      else
        plate_dev::k_plate_dir<double><<<h->drv.n_work, plate_dev::THREADS, h->smem, st>>>(A, C, S);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
};

int copy_problem(nmpc_plate* h, const double* x0, const double* x_ref, const double* u_ref,
                 cudaStream_t st) {
  SDRV_CHECK(cudaMemcpyAsync(h->drv.x0, x0, h->drv.n_g * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDRV_CHECK(cudaMemcpyAsync(h->xref, x_ref, h->drv.n_g * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SDRV_CHECK(cudaMemcpyAsync(h->uref, u_ref, h->n_a * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return NMPC_OK;
}

int plant(nmpc_plate* h, double* w, double dt, int n_sub, void* stream) {
  plate_dev::k_plate_plant<<<h->drv.n, plate_dev::THREADS, 2 * h->ng_max * sizeof(double),
                             (cudaStream_t)stream>>>(make_args(h), h->drv.lay, w, h->drv.ub[2], dt,
                                                     n_sub);
  SDRV_CHECK(cudaGetLastError());
  return NMPC_OK;
}

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
  o->precision = NMPC_FP64;
}

int nmpc_plate_setup(const nmpc_plate_desc* descs, int n, const nmpc_plate_opts* opts,
                     nmpc_plate** out) {
  if (!descs || n < 1 || !out) return NMPC_ERR_BAD_ARG;
  *out = nullptr;
  nmpc_plate_opts o;
  nmpc_plate_default_opts(&o);
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
  nmpc_plate* h = new (std::nothrow) nmpc_plate();
  if (!h) return NMPC_ERR_CUDA;
  h->opts = o;
  std::vector<int> pt_state, act_pt, Lc, Ltc;
  std::vector<double> Lv, Ltv, Ld;
  long long n_pts = 0;
  for (int b = 0; b < n; ++b) {
    const nmpc_plate_desc& d = descs[b];
    PInst I{};
    I.dim = d.dim;
    I.m = d.m;
    I.ng = d.dim == 2 ? d.m * d.m : d.m;
    I.nu = d.n_u;
    I.ns = I.ng - I.nu;
    I.N = d.horizon;
    I.a_off = h->n_a;
    I.t_off = n_pts;
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
    std::vector<int> state_of(I.ng, 0);
    std::vector<char> is_act(I.ng, 0);
    for (int a = 0; a < d.n_u; ++a) {
      state_of[d.act_cell[a]] = -1 - a;
      is_act[d.act_cell[a]] = 1;
    }
    int t = 0;
    for (int p = 0; p < I.ng; ++p)
      if (!is_act[p]) state_of[p] = t++;
    for (int p = 0; p < I.ng; ++p) pt_state.push_back(state_of[p]);
    for (int a = 0; a < d.n_u; ++a) act_pt.push_back(d.act_cell[a]);
    stage_drv::append_ell(d.dim, d.m, d.bc == 0 ? 0 : 1, Lc, Lv, Ltc, Ltv, Ld);
    stage_drv::Layout L{};
    L.N = I.N;
    L.nx = I.ns;
    L.nu = I.nu;
    L.u_cold = d.tau > 0.0 ? 0.5 * (d.u_lo + d.u_hi) : 0.0;
    h->drv.lay_h.push_back(L);
    h->n_a += I.nu;
    n_pts += I.ng;
    h->ng_max = std::max(h->ng_max, I.ng);
    h->inst_h.push_back(I);
  }
  const size_t tsz = o.precision == NMPC_MIXED ? sizeof(float) : sizeof(double);
  h->smem = (size_t)h->ng_max * (plate_dev::F64_FIELDS * sizeof(double) + plate_dev::T_FIELDS * tsz);
  cudaError_t e = stage_drv::driver_alloc(h->drv);
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(stage_drv::dalloc(&h->inst_d, n));
  A(stage_drv::dalloc(&h->pt_state, pt_state.size()));
  A(stage_drv::dalloc(&h->act_pt, act_pt.size()));
  A(stage_drv::dalloc(&h->Lc, Lc.size()));
  A(stage_drv::dalloc(&h->Ltc, Ltc.size()));
  A(stage_drv::dalloc(&h->Lv, Lv.size()));
  A(stage_drv::dalloc(&h->Ltv, Ltv.size()));
  A(stage_drv::dalloc(&h->Ld, Ld.size()));
  A(stage_drv::dalloc(&h->xref, h->drv.n_g));
  A(stage_drv::dalloc(&h->uref, h->n_a));
  A(stage_drv::upload(h->inst_d, h->inst_h));
  A(stage_drv::upload(h->pt_state, pt_state));
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
    A(cudaFuncSetAttribute(plate_dev::k_plate_dir<double>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem));
    A(cudaFuncSetAttribute(plate_dev::k_plate_dir<float>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem));
  }
  if (e != cudaSuccess) {
    fprintf(stderr, "nmpc_plate_setup: %s\n", cudaGetErrorString(e));
    free_plate(h);
    delete h;
    return NMPC_ERR_CUDA;
  }
  *out = h;
  return NMPC_OK;
}

int nmpc_plate_sizes(const nmpc_plate* h, int64_t* out) {
  if (!h || !out) return NMPC_ERR_BAD_ARG;
  out[0] = h->drv.n_g;
  out[1] = h->drv.n_x;
  out[2] = h->drv.n_u;
  out[3] = h->n_a;
  return NMPC_OK;
}

int nmpc_plate_solve(nmpc_plate* h, const double* x0, const double* x_ref, const double* u_ref,
                     int init, double* u_out, nmpc_stats* stats, void* stream) {
  if (!h || !x0 || !x_ref || !u_ref) return NMPC_ERR_BAD_ARG;
  if (init != NMPC_INIT_COLD && init != NMPC_INIT_WARM && init != NMPC_INIT_SHIFT)
    return NMPC_ERR_BAD_ARG;
  if (init != NMPC_INIT_COLD && !h->drv.has_state) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = copy_problem(h, x0, x_ref, u_ref, st);
  if (rc != NMPC_OK) return rc;
  PlateDir dir{h, st};
  return stage_drv::solve(h->drv, init, h->opts.max_iter, h->opts.tol, h->opts.check_every, dir,
                          u_out, stats, st);
}

int nmpc_plate_iterate(nmpc_plate* h, const double* x0, const double* x_ref, const double* u_ref,
                       const double* x_in, const double* u_in, const double* lam_in,
                       double* x_out, double* u_out, double* lam_out, int n_iter, double* out,
                       void* stream) {
  if (!h || !x0 || !x_ref || !u_ref || !x_in || !u_in || !lam_in || !x_out || !u_out || !lam_out ||
      n_iter < 1)
    return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = copy_problem(h, x0, x_ref, u_ref, st);
  if (rc != NMPC_OK) return rc;
  PlateDir dir{h, st};
  return stage_drv::iterate(h->drv, x_in, u_in, lam_in, x_out, u_out, lam_out, n_iter, out, dir, st);
}

int nmpc_plate_get_state(nmpc_plate* h, double* x, double* u, double* lam, void* stream) {
  if (!h) return NMPC_ERR_BAD_ARG;
  return stage_drv::get_state(h->drv, x, u, lam, (cudaStream_t)stream);
}

int nmpc_plate_plant_step(nmpc_plate* h, double* w, double dt, int n_sub, void* stream) {
  if (!h || !w || !(dt >= 0) || n_sub < 1 || !h->drv.has_state) return NMPC_ERR_BAD_ARG;
  return plant(h, w, dt, n_sub, stream);
}

int nmpc_plate_closed_loop(nmpc_plate* h, double* w, const double* x_ref, const double* u_ref,
                           int steps, int n_sub, double* u_hist, int* iters_hist,
                           double* res_hist, void* stream) {
  if (!h || !w || !x_ref || !u_ref || steps < 1 || n_sub < 1) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = h->drv.n;
  std::vector<nmpc_stats> stats(n);
  int rc_all = NMPC_OK;
  for (int t = 0; t < steps; ++t) {
    const int init = (t == 0 && !h->drv.has_state) ? NMPC_INIT_COLD : NMPC_INIT_SHIFT;
    const int rc = nmpc_plate_solve(h, w, x_ref, u_ref, init, nullptr, stats.data(), stream);
    if (rc == NMPC_ERR_BAD_ARG || rc == NMPC_ERR_CUDA) return rc;
    if (rc != NMPC_OK && rc_all == NMPC_OK) rc_all = rc;
    for (int b = 0; b < n; ++b) {
      if (iters_hist) iters_hist[(size_t)t * n + b] = stats[b].iters;
      if (res_hist) res_hist[(size_t)t * n + b] = stats[b].res_inf;
    }
    if (u_hist) {
      // u_1 of every instance (stage 1 of the packed control trajectory)
      for (int b = 0; b < n; ++b) {
        const PInst& I = h->inst_h[b];
        SDRV_CHECK(cudaMemcpyAsync(u_hist + (size_t)t * h->n_a + I.a_off,
                                   h->drv.ub[2] + h->drv.lay_h[b].u_off, I.nu * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
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
