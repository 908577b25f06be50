// Device code of the double-layer Jacobi NMPC solver (sm_103a).
//
// One thread-block cluster of C CTAs processes one (instance, stage) work
// item of one upper-layer iteration (eq. 15); every stage of every instance
// is updated at once from iterate k, so one launch is one iteration.  The
// stage grid is split into C slabs (rows in 2D, segments in 1D); stencil
// neighbours in another CTA's slab are read from its shared memory through
// the cluster's distributed shared memory.  Inside a work item:
//   P1/P2 residual: the stage's KKT rows K_i (eq. 9) from x_{i-1}, s_i,
//     lambda_{i+1}, the coefficient fields Phi'(x), A_xx and 1/diag(F_x) of
//     the reordered stage block (eq. 21), and the residual norms.  Two forms:
//       full  - everything in float64 (the certifying residual);
//       split - the O(1) differences x_{i-1} - x_i and lambda_{i+1} -
//               lambda_i in float64, the O(h) stencil terms in float32.
//   P3 lower layer (T = float or double): Sec. 4.3 (eqs. 22-24) with the u
//     fixed-point iteration of Sec. 5.2, by pointwise Jacobi sweeps over the
//     slab; the first sweep from zero is D^{-1} c and is folded into the
//     second sweep's neighbour reads.
//   P4 update: S_i <- S_i - alpha Delta s_i in float64 into the other buffer.
// Convergence bookkeeping (per-instance status, residual history, the switch
// from split to full residuals, the iteration counter) stays on the device so
// that chunks of iterations replay as a CUDA graph with no host arguments.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace nmpc_dev {

namespace cg = cooperative_groups;

constexpr int RES_SLOTS = 16;    // rolling residual history per instance
constexpr int NUM_WORK_ARRAYS = 11;
constexpr int NUM_STAGE_ARRAYS = 5;  // float64 staging of x_i, lambda_i, x_{i-1}, lambda_{i+1}, ref
constexpr int MAX_NU = 64;

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
  unsigned long long* res_inf;   // [RES_SLOTS][n_inst], bits of non-negative doubles
  unsigned long long* res_err;   // [RES_SLOTS][n_inst] bound on a split residual's rounding error
  double* res_sq;                // [RES_SLOTS][n_inst]
  unsigned long long* res_first; // [n_inst] ||K(S^0)||_inf
  int* status;
  int* iters;
  int* final_buf;
  double* fin_inf;
  double* fin_2;
  int* full_from;  // [n_inst] first iteration evaluated with the float64 residual
  int* full0;      // [n_inst] 1: iteration 0 also uses it (warm starts)
  int* n_active;
  double tol, div_limit, alpha;
  double split_min;  // below max(tol, split_min) iterations use the float64 residual
  int max_iter, n_lo, n_u_it;
  int resid_only;  // one-shot: residual norms only (float64)
  int full_all;    // every residual in float64 (FP64 precision)
  int csize;       // CTAs per work item (cluster size)
  int stage;       // float64 slab inputs staged in shared memory (1) or read in place
  int local_u;     // u-iteration through the actuators' local responses (1) or full sweeps
  int box_r;       // half-width of a local-response box, 2 (n_lo - 1)
  int slab_max;    // length of each padded slab array (halo rows and pads included)
  // lower-layer work arrays: shared memory (scratch == nullptr) or a global
  // slab of scratch_stride bytes per CTA
  char* scratch;
  long long scratch_stride;
};

struct Cl {
  int C, rank;
  __device__ __forceinline__ void sync() const {
    if (C > 1) cg::this_cluster().sync();
    else __syncthreads();
  }
  template <typename T>
  __device__ __forceinline__ T* map(T* p, int r) const {
    return cg::this_cluster().map_shared_rank(p, r);
  }
};

// Quotient q / d for 0 <= q < 2^22, d >= 1, inv = 1.0f / d: the float
// estimate is off by at most one and is corrected.
__device__ __forceinline__ int fdiv(int q, int d, float inv) {
  const int j = __float2int_rz(__int2float_rz(q) * inv);
  const int r = q - j * d;
  return j + (r >= d ? 1 : 0) - (r < 0 ? 1 : 0);
}

// A cluster rank's slab in the padded layout of its shared work arrays.  The
// stage grid is split into whole rows (2D) or segments (1D), `per` rows or
// cells per rank (the last non-empty rank may hold fewer, later ranks none).
// 2D: slab cell (row j, column i) sits at p = (j + 1) W + i + 1, W = mx + 2;
// padded rows 0 and rows + 1 hold the neighbouring ranks' boundary rows (the
// halo) or zeros at the grid's Dirichlet ring, padded columns 0 and mx + 1
// are zero.  1D: cell q sits at p = q + 1; positions 0 and n + 1 are halo or
// zero.  Stencils then read their neighbours with no bounds tests, and a rank
// that writes a boundary value also stores it into the neighbour's halo.
struct Geo {
  int dim;
  int mx, per;   // grid row length; rows (2D) / cells (1D) per rank
  int cols;      // 2D: mx; 1D: n
  int n;         // cells of this rank
  int rows;      // 2D: rows of this rank; 1D: 1
  int W;         // 2D: padded row stride mx + 2; 1D: 0
  int lo;        // first grid cell of the slab
  int r0;        // first grid row (2D) / cell (1D) of the slab
  int edge;      // cells of the first (last) row: 2D mx, 1D 1
  int up_off;    // shift into rank - 1's layout: its bottom halo row
  int dn_off;    // shift back into rank + 1's layout: its top halo row
  int plen;      // padded positions in use
  bool up, dn;   // rank - 1 / rank + 1 hold cells (halo exchange partners)
  float inv_cols, inv_W;
  __device__ __forceinline__ int pidx(int q) const {
    return (dim == 2) ? W + 1 + q + 2 * fdiv(q, cols, inv_cols) : q + 1;
  }
};

__device__ __forceinline__ Geo geo_of(const InstDev& I, int C, int rank) {
  Geo g;
  const bool d2 = (I.dim == 2);
  g.dim = I.dim;
  g.mx = I.mx;
  const int nun = d2 ? I.my : I.mx;
  g.per = (nun + C - 1) / C;
  const int a = min(rank * g.per, nun), b = min(a + g.per, nun);
  g.r0 = a;
  g.rows = d2 ? b - a : 1;
  g.n = d2 ? (b - a) * I.mx : b - a;
  g.cols = d2 ? I.mx : g.n;
  g.W = d2 ? I.mx + 2 : 0;
  g.lo = d2 ? a * I.mx : a;
  g.edge = d2 ? I.mx : 1;
  g.up_off = d2 ? g.per * g.W : g.per;
  g.dn_off = d2 ? (b - a) * g.W : (b - a);
  g.plen = d2 ? (b - a + 2) * g.W : (b - a) + 2;
  g.up = (rank > 0) && (b > a);
  g.dn = (b < nun) && (b > a);
  g.inv_cols = 1.0f / (float)max(g.cols, 1);
  g.inv_W = 1.0f / (float)max(g.W, 1);
  return g;
}

// Padded position of grid cell c in the slab of the rank that owns it.
__device__ __forceinline__ int owner_of(int c, const Geo& g, int& p) {
  if (g.dim == 2) {
    const int row = c / g.mx, col = c - row * g.mx;
    const int r = row / g.per;
    p = (row - r * g.per + 1) * (g.mx + 2) + col + 1;
    return r;
  }
  const int r = c / g.per;
  p = c - r * g.per + 1;
  return r;
}

// Element of slab array `a` at grid cell c, in this rank's or another rank's
// shared memory.
template <typename T>
__device__ __forceinline__ T* at(T* a, int c, const Geo& g, const Cl& cl) {
  int p;
  const int r = owner_of(c, g, p);
  return (r == cl.rank) ? a + p : cl.map(a, r) + p;
}

// The neighbours' copies of a slab array (their halo rows receive this rank's
// boundary values).
template <typename T>
struct Halo {
  T* up;
  T* dn;
};

template <typename T>
__device__ __forceinline__ Halo<T> halo_of(T* a, const Geo& g, const Cl& cl) {
  Halo<T> hl;
  hl.up = g.up ? cl.map(a, cl.rank - 1) : nullptr;
  hl.dn = g.dn ? cl.map(a, cl.rank + 1) : nullptr;
  return hl;
}

// Store v at own cell q (padded position p) and, on a boundary row, into the
// neighbours' halo.
template <typename T>
__device__ __forceinline__ void put(T* a, const Halo<T>& hl, const Geo& g, int q, int p, T v) {
  a[p] = v;
  if (g.up && q < g.edge) hl.up[p + g.up_off] = v;
  if (g.dn && q >= g.n - g.edge) hl.dn[p - g.dn_off] = v;
}

// Zero the padded positions of `a` that no rank writes in a work item: the
// column pads and the halo rows at the grid boundary (the Dirichlet ring).
template <typename V>
__device__ __forceinline__ void zero_ring(V* a, const Geo& g) {
  if (g.n == 0) return;
  if (g.dim == 2) {
    for (int jj = threadIdx.x; jj < g.rows + 2; jj += blockDim.x) {
      a[jj * g.W] = V(0);
      a[jj * g.W + g.W - 1] = V(0);
    }
    if (!g.up)
      for (int i = threadIdx.x; i < g.W; i += blockDim.x) a[i] = V(0);
    if (!g.dn)
      for (int i = threadIdx.x; i < g.W; i += blockDim.x) a[(g.rows + 1) * g.W + i] = V(0);
  } else if (threadIdx.x == 0) {
    if (!g.up) a[0] = V(0);
    if (!g.dn) a[g.n + 1] = V(0);
  }
}

// Weighted sum of the four (2D) or two (1D) stencil neighbours of padded
// position p.
template <typename V, typename F>
__device__ __forceinline__ V stencil(const Geo& g, int p, V cx, V cy, F a) {
  const V sx = a(p - 1) + a(p + 1);
  if (g.dim == 2) return cx * sx + cy * (a(p - g.W) + a(p + g.W));
  return cx * sx;
}

// One pass over the rank's n cells, CPT cells per thread per round: every
// cell's loads and arithmetic (ld) come before any of the round's stores
// (st), so the CPT cells form independent dependency chains.
template <int CPT, typename V, typename LD, typename ST>
__device__ __forceinline__ void pass(int n, LD ld, ST st) {
  for (int base = threadIdx.x; base < n; base += CPT * blockDim.x) {
    V v[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int q = base + k * blockDim.x;
      if (q < n) v[k] = ld(q);
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int q = base + k * blockDim.x;
      if (q < n) st(q, v[k]);
    }
  }
}

__device__ __forceinline__ double phi_d(double w, double k0, double k1) {
  return k0 * (w + 0.5 * k1 * w * w);
}

__device__ __forceinline__ double abs_or_inf(double v) {
  const double a = fabs(v);
  return (a <= 1.79e308) ? a : CUDART_INF;  // NaN and Inf count as +Inf
}

__device__ __forceinline__ float abs_or_inf_f(float v) {
  const float a = fabsf(v);
  return (a <= 3.4e38f) ? a : CUDART_INF_F;
}

// float64 <-> float32 by IEEE-754 bit manipulation on the integer ALUs (the
// float64 pipe issues 2 lanes per clock per SM on this part).  d2f truncates
// toward zero (relative error < 2^-23); zero/subnormal doubles become +-0 and
// out-of-range or NaN doubles become +-Inf.  f2d is exact for normal floats;
// subnormal floats become +-0.
__device__ __forceinline__ float d2f(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // rebias 1023 -> 127
  const unsigned man = ((hi & 0xfffffu) << 3) | (lo >> 29);
  unsigned bits = sign | ((unsigned)e << 23) | man;
  bits = (e <= 0) ? sign : bits;
  bits = (e >= 255) ? (sign | 0x7f800000u) : bits;
  return __uint_as_float(bits);
}

__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned man = b & 0x7fffffu;
  unsigned hi = sign | ((e + 896u) << 20) | (man >> 3);
  unsigned lo = man << 29;
  hi = (e == 0u) ? sign : hi;
  lo = (e == 0u) ? 0u : lo;
  hi = (e == 255u) ? (sign | 0x7ff00000u | (man >> 3)) : hi;
  return __hiloint2double((int)hi, (int)lo);
}

// Sum of the stencil neighbours' values, each weighted by its axis
// coefficient; cells outside the interior grid are zero (Dirichlet ring).
template <typename V, typename G>
__device__ __forceinline__ V nbr_sum(int c, int ix, int iy, int mx, int my, V cx, V cy, G g) {
  V sx = V(0), sy = V(0);
  if (ix > 0) sx += g(c - 1);
  if (ix < mx - 1) sx += g(c + 1);
  if (iy > 0) sy += g(c - mx);
  if (iy < my - 1) sy += g(c + mx);
  return cx * sx + cy * sy;
}

struct BlockRed {
  double mx[32];
  double sq[32];
  float4 mg[32];
};

__device__ __forceinline__ void block_reduce_store(double vmax, double vsq, BlockRed* red,
                                                   double* out_max, double* out_sq) {
  for (int o = 16; o > 0; o >>= 1) {
    vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    vsq += __shfl_xor_sync(0xffffffffu, vsq, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red->mx[wid] = vmax;
    red->sq[wid] = vsq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0, s = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) {
      m = fmax(m, red->mx[w]);
      s += red->sq[w];
    }
    *out_max = m;
    *out_sq = s;
  }
}

// Split residual: float32 partial norms (max, sum of squares) and the four
// magnitude maxima of its rounding bound, block-reduced; thread 0 receives the
// norms in float64 and the maxima in mags[4].
__device__ __forceinline__ void block_reduce_store_f(float vmax, float vsq, float4 mg,
                                                     BlockRed* red, double* out_max,
                                                     double* out_sq, float* mags) {
  for (int o = 16; o > 0; o >>= 1) {
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    vsq += __shfl_xor_sync(0xffffffffu, vsq, o);
    mg.x = fmaxf(mg.x, __shfl_xor_sync(0xffffffffu, mg.x, o));
    mg.y = fmaxf(mg.y, __shfl_xor_sync(0xffffffffu, mg.y, o));
    mg.z = fmaxf(mg.z, __shfl_xor_sync(0xffffffffu, mg.z, o));
    mg.w = fmaxf(mg.w, __shfl_xor_sync(0xffffffffu, mg.w, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red->mx[wid] = f2d(vmax);
    red->sq[wid] = f2d(vsq);
    red->mg[wid] = mg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0, s = 0.0;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) {
      m = fmax(m, red->mx[w]);
      s += red->sq[w];
      g.x = fmaxf(g.x, red->mg[w].x);
      g.y = fmaxf(g.y, red->mg[w].y);
      g.z = fmaxf(g.z, red->mg[w].z);
      g.w = fmaxf(g.w, red->mg[w].w);
    }
    *out_max = m;
    *out_sq = s;
    mags[0] = g.x;
    mags[1] = g.y;
    mags[2] = g.z;
    mags[3] = g.w;
  }
}

// Per-work-item shared scalars (the NUM_WORK_ARRAYS slab arrays follow).
template <typename T>
struct SmallShared {
  unsigned long long amask[512];  // per thread: which of its cells carry an actuator
  BlockRed red;
  double red_out[2];
  double u[MAX_NU];
  T b3[MAX_NU];
  T v3[MAX_NU];
  T b1a[MAX_NU];  // state-equation row K1 at each actuator cell (owner rank only)
  T y4a[MAX_NU];  // lambda-part of Y(0) at each actuator cell
  T v3n[MAX_NU];
  int act[MAX_NU];
  int skip;
  int full;
};

__device__ __forceinline__ double to_double(float v) { return f2d(v); }
__device__ __forceinline__ double to_double(double v) { return v; }

// float64 -> T off the float64 pipe (truncating for float)
template <typename T>
__device__ __forceinline__ T to_T(double v);
template <>
__device__ __forceinline__ float to_T<float>(double v) { return d2f(v); }
template <>
__device__ __forceinline__ double to_T<double>(double v) { return v; }

// 1 / v rounded to nearest (the same value as the IEEE division)
__device__ __forceinline__ float rcp_T(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double rcp_T(double v) { return __drcp_rn(v); }

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}

// gstage: NUM_STAGE_ARRAYS float64 arrays in shared memory in the padded
// layout (x_i and lambda_i with their halo rows; x_{i-1}, lambda_{i+1}, ref at
// the own cells), or nullptr (the stage is read from global memory in place).
template <typename T, int CPT>
__device__ void process_item(const IterArgs& A, int b, int s, int k, int rd, bool full,
                             bool resid_only, SmallShared<T>& sm, T* wk, const Cl& cl,
                             double* gstage) {
  const InstDev I = A.inst[b];
  const Geo g = geo_of(I, cl.C, cl.rank);
  const int nu = I.nu, N = I.N, ng = I.ng, n = g.n;
  const int tid = threadIdx.x, bd = blockDim.x;
  const long long so = I.s_off + (long long)s * ng;
  const double* __restrict__ X = A.xin[rd];
  const double* __restrict__ L = A.lin[rd];
  const double* __restrict__ Uin = A.uin[rd];
  const double* __restrict__ x0 = A.x0 + I.g_off;
  const double* __restrict__ ref = A.ref + I.g_off;
  const double h = I.h, cx = I.cx, cy = I.cy, k0 = I.k0, k1 = I.k1, b0 = I.b0;
  const double dcoef = 2.0 * (cx + cy);
  const bool last = (s == N - 1);
  const int SM = A.slab_max;
  const int n_lo = A.n_lo;
  const bool wide = n_lo > 2;  // sweeps 3.. read dp and the previous sweep at neighbours
  // the residual pass keeps many values live per cell: fewer cells per round
  // (float64 form: one)
  constexpr int RES_CPT = (CPT > 2) ? CPT / 2 : CPT;
  constexpr int FULL_CPT = 1;

  T* b2 = wk;               // costate row K3
  T* dp = wk + 1 * SM;      // Phi'(x)
  T* ax = wk + 2 * SM;      // A_xx
  T* rg = wk + 3 * SM;      // 1 / diag(F_x)
  T* v1 = wk + 4 * SM;      // first F_x sweep  D^{-1} c4,  c4 = F_u v3 - K1
  T* p1 = wk + 5 * SM;      // Phi' * v1 (its neighbour product)
  T* y5 = wk + 6 * SM;      // x-part of Y(v3)
  T* w1 = wk + 7 * SM;      // first F_x^T sweep
  T* y4 = wk + 8 * SM;      // lambda-part of Y(v3)
  T* e1 = wk + 9 * SM;      // ping-pong spares for n_lo > 2
  T* e2 = wk + 10 * SM;
  // residual inputs, alive in P1-P2 only: float copies of x, lambda and Phi(x)
  // (split residual), or Phi(x) in float64 (full residual, staged slab)
  float* xf = reinterpret_cast<float*>(y5);
  float* lf = reinterpret_cast<float*>(w1);
  float* pf = reinterpret_cast<float*>(y4);
  double* phid = reinterpret_cast<double*>(y5);

  // actuators: controls of this stage, and per thread a bit mask of which of
  // its cells carry one (cell q is bit q / blockDim of thread q % blockDim)
  for (int a = tid; a < nu; a += bd) {
    const int c = A.act[I.act_off + a];
    sm.act[a] = c;
    sm.u[a] = Uin[I.u_off + (long long)s * nu + a];
    sm.v3[a] = T(0);
    const int q = c - g.lo;
    if (q >= 0 && q < n && q / bd < 64) atomicOr(&sm.amask[q % bd], 1ull << (q / bd));
  }
  double* sx = gstage;
  double* sl_ = gstage + SM;
  double* sxp = gstage + 2 * SM;
  double* sln = gstage + 3 * SM;
  double* srf = gstage + 4 * SM;
  if (gstage) {
    // asynchronous copies, all in flight at once; outside the grid: zero
    for (int pp = tid; pp < g.plen; pp += bd) {
      int row, col;
      bool own;
      if (g.dim == 2) {
        const int jj = fdiv(pp, g.W, g.inv_W);
        row = g.r0 - 1 + jj;
        col = pp - jj * g.W - 1;
        own = jj >= 1 && jj <= g.rows;
      } else {
        row = 0;
        col = g.r0 - 1 + pp;
        own = pp >= 1 && pp <= n;
      }
      if (col >= 0 && col < I.mx && row >= 0 && row < I.my) {
        const int c = row * I.mx + col;
        cp_async8(sx + pp, X + so + c);
        cp_async8(sl_ + pp, L + so + c);
        if (own) {
          cp_async8(sxp + pp, (s == 0) ? x0 + c : X + so - ng + c);
          if (!last) cp_async8(sln + pp, L + so + ng + c);
          cp_async8(srf + pp, ref + c);
        }
      } else {
        sx[pp] = 0.0;
        sl_[pp] = 0.0;
      }
    }
  }
  zero_ring(p1, g);
  if (wide) {
    zero_ring(dp, g);
    zero_ring(e1, g);
    zero_ring(e2, g);
  }
  if (gstage) asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  // own-cell float64 inputs at cell q (padded position p)
  auto OX = [&](int q, int p) { return gstage ? sx[p] : X[so + g.lo + q]; };
  auto OL = [&](int q, int p) { return gstage ? sl_[p] : L[so + g.lo + q]; };
  auto OXP = [&](int q, int p) {
    return gstage ? sxp[p] : ((s == 0) ? x0[g.lo + q] : X[so - ng + g.lo + q]);
  };
  auto OLN = [&](int q, int p) { return gstage ? sln[p] : L[so + ng + g.lo + q]; };
  auto ORF = [&](int q, int p) { return gstage ? srf[p] : ref[g.lo + q]; };
  // float64 x or lambda at padded position pp read in place (zero outside the grid)
  auto gpad = [&](const double* base, int pp) {
    int row, col;
    if (g.dim == 2) {
      const int jj = fdiv(pp, g.W, g.inv_W);
      row = g.r0 - 1 + jj;
      col = pp - jj * g.W - 1;
    } else {
      row = 0;
      col = g.r0 - 1 + pp;
    }
    return (col >= 0 && col < I.mx && row >= 0 && row < I.my) ? base[so + row * I.mx + col] : 0.0;
  };

  // ---- P1: residual inputs on the padded slab, halo rows included ----
  const float k0f = (float)k0, k1h = (float)(0.5 * k1);
  struct F3 { float x, l, p; };
  // magnitudes for the split residual's rounding bound: max |x|, |lambda| over
  // the padded slab, max |float64 difference|, |ref| over the own cells
  float4 mg = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!full) {
    pass<CPT, F3>(g.plen,
        [&](int pp) {
          F3 o;
          o.x = d2f(gstage ? sx[pp] : gpad(X, pp));
          o.l = d2f(gstage ? sl_[pp] : gpad(L, pp));
          o.p = k0f * (o.x + k1h * o.x * o.x);
          mg.x = fmaxf(mg.x, fabsf(o.x));
          mg.y = fmaxf(mg.y, fabsf(o.l));
          return o;
        },
        [&](int pp, F3 o) {
          xf[pp] = o.x;
          lf[pp] = o.l;
          pf[pp] = o.p;
        });
  } else if (gstage) {
    pass<CPT, double>(g.plen, [&](int pp) { return phi_d(sx[pp], k0, k1); },
                      [&](int pp, double v) { phid[pp] = v; });
  }
  __syncthreads();

  // ---- P2: K_i (eq. 9), coefficient fields, norms ----
  double vmax = 0.0, vsq = 0.0;
  float fmax_ = 0.0f, fsq = 0.0f;
  const T th = (T)h, tdc = (T)dcoef;
  const float cxf = (float)cx, cyf = (float)cy, dcf = (float)dcoef, hf = (float)h;
  const float k0f_ = (float)k0, k1f_ = (float)k1, qf_ = (float)I.q, b0f = (float)b0;
  const float k01f = (float)(k0 * k1), hqff = last ? (float)(h * I.qf) : 0.0f;
  const double hqf = h * I.qf;
  const unsigned long long amask = sm.amask[tid];
  sm.amask[tid] = 0ull;  // ready for the next work item
  struct P2Out {
    int p;
    bool act;
    T K1, K3, dp, ax;
  };
  const Halo<T> hdp = halo_of(dp, g, cl);
  const Halo<T> hp1 = halo_of(p1, g, cl);
  auto p2_store = [&](int q, P2Out o) {
    if (resid_only) return;
    const int p = o.p;
    const T r = rcp_T(-T(1) - th * tdc * o.dp);
    b2[p] = o.K3;
    ax[p] = o.ax;
    rg[p] = r;
    const T v = -o.K1 * r;  // first sweep of F_x v5 = -K1 (v3 = 0)
    v1[p] = v;
    if (wide) put(dp, hdp, g, q, p, o.dp);
    else dp[p] = o.dp;
    put(p1, hp1, g, q, p, o.dp * v);
    if (o.act) {
      const int c = g.lo + q;
      for (int a = 0; a < nu; ++a)
        if (sm.act[a] == c) sm.b1a[a] = o.K1;
    }
  };
  if (full) {
    pass<FULL_CPT, P2Out>(n,
        [&](int q) {
          P2Out o;
          const int p = g.pidx(q);
          const int c = g.lo + q;
          const int slot = q / bd;  // this cell's bit in the thread's mask
          bool isact = (slot < 64) ? ((amask >> slot) & 1ull) != 0ull : false;
          if (slot >= 64)
            for (int a = 0; a < nu; ++a) isact |= (sm.act[a] == c);
          o.p = p;
          o.act = isact;
          const double x = OX(q, p);
          const double lam = OL(q, p);
          const double xp = OXP(q, p);
          const double rc_ = ORF(q, p);
          const double ln = last ? hqf * (x - rc_) : OLN(q, p);
          double srcd = 0.0;
          if (isact) {
            for (int a = 0; a < nu; ++a)
              if (sm.act[a] == c) srcd += sm.u[a];
            srcd *= b0;
          }
          double lphi, mu;
          if (gstage) {
            lphi = stencil<double>(g, p, cx, cy, [&](int m) { return phid[m]; }) - dcoef * phid[p];
            mu = stencil<double>(g, p, cx, cy, [&](int m) { return sl_[m]; }) - dcoef * lam;
          } else {
            const int iy = (g.dim == 2) ? g.r0 + fdiv(q, g.cols, g.inv_cols) : 0;
            const int ix = c - iy * I.mx;
            const double* Xs = X + so;
            const double* Ls = L + so;
            lphi = nbr_sum<double>(c, ix, iy, I.mx, I.my, cx, cy,
                                   [&](int m) { return phi_d(Xs[m], k0, k1); }) -
                   dcoef * phi_d(x, k0, k1);
            mu = nbr_sum<double>(c, ix, iy, I.mx, I.my, cx, cy, [&](int m) { return Ls[m]; }) -
                 dcoef * lam;
          }
          const double dphi = k0 * (1.0 + k1 * x);
          const double K1 = xp - x + h * (lphi + srcd);
          const double K3 = ln - lam + h * (I.q * (x - rc_) + dphi * mu);
          vmax = fmax(vmax, fmax(abs_or_inf(K1), abs_or_inf(K3)));
          vsq += K1 * K1 + K3 * K3;
          o.K1 = to_T<T>(K1);
          o.K3 = to_T<T>(K3);
          o.dp = to_T<T>(dphi);
          o.ax = to_T<T>(h * (I.q + k0 * k1 * mu) + (last ? hqf : 0.0));
          return o;
        },
        p2_store);
  } else {
    pass<RES_CPT, P2Out>(n,
        [&](int q) {
          P2Out o;
          const int p = g.pidx(q);
          const int c = g.lo + q;
          const int slot = q / bd;  // this cell's bit in the thread's mask
          bool isact = (slot < 64) ? ((amask >> slot) & 1ull) != 0ull : false;
          if (slot >= 64)
            for (int a = 0; a < nu; ++a) isact |= (sm.act[a] == c);
          o.p = p;
          o.act = isact;
          const double x = OX(q, p);
          const double lam = OL(q, p);
          const double xp = OXP(q, p);
          const double rc_ = ORF(q, p);
          const float lphi = stencil<float>(g, p, cxf, cyf, [&](int m) { return pf[m]; }) - dcf * pf[p];
          const float mu = stencil<float>(g, p, cxf, cyf, [&](int m) { return lf[m]; }) - dcf * lf[p];
          const float xv = xf[p];
          const float rv = d2f(rc_);
          float srcf = 0.0f;
          if (isact)
            for (int a = 0; a < nu; ++a)
              if (sm.act[a] == c) srcf += d2f(sm.u[a]);
          const float dphi = k0f_ * (1.0f + k1f_ * xv);
          const float t1 = hf * (lphi + b0f * srcf);
          const float t3 = hf * (qf_ * (xv - rv) + dphi * mu);
          // the O(1) differences in float64; at the last stage lambda_{N+1} is
          // h qf (x_N - ref), an O(h) term
          const double d3 = last ? -lam : OLN(q, p) - lam;
          const float dx = d2f(xp - x), dl = d2f(d3);
          mg.z = fmaxf(mg.z, fmaxf(fabsf(dx), fabsf(dl)));
          mg.w = fmaxf(mg.w, fabsf(rv));
          const float K1 = dx + t1;
          const float K3 = dl + t3 + (last ? hqff * (xv - rv) : 0.0f);
          fmax_ = fmaxf(fmax_, fmaxf(abs_or_inf_f(K1), abs_or_inf_f(K3)));
          fsq += K1 * K1 + K3 * K3;
          o.K1 = (T)K1;
          o.K3 = (T)K3;
          o.dp = (T)dphi;
          o.ax = (T)(hf * (qf_ + k01f * mu) + hqff);
          return o;
        },
        p2_store);
  }
  for (int a = tid; a < nu; a += bd) {
    const double K2 = h * (I.r * sm.u[a] + b0 * L[so + sm.act[a]]);
    if (cl.rank == 0) {
      if (full) {
        vmax = fmax(vmax, abs_or_inf(K2));
        vsq += K2 * K2;
      } else {
        const float K2f = d2f(K2);
        fmax_ = fmaxf(fmax_, abs_or_inf_f(K2f));
        fsq += K2f * K2f;
        mg.z = fmaxf(mg.z, fabsf(K2f));
      }
    }
    sm.b3[a] = (T)K2;
  }
  float mags[4];
  if (full) block_reduce_store(vmax, vsq, &sm.red, &sm.red_out[0], &sm.red_out[1]);
  else block_reduce_store_f(fmax_, fsq, mg, &sm.red, &sm.red_out[0], &sm.red_out[1], mags);
  if (tid == 0) {
    const int slot = (k % RES_SLOTS) * A.n_inst + b;
    if (!full) {
      // Rounding bound of the split residual on this slab (unit roundoff
      // u = 2^-24).  x and lambda are truncated to float32 (2u), Phi, Phi' and
      // the five-point sums are evaluated in float32 (a few u each): with
      // X, Lm the maxima of |x|, |lambda| over the padded slab, every O(h) term
      // is off by at most 16 u h S, S = 4 (cx + cy) (Phi_max + Phi'_max Lm) +
      // b0 sum|u| + (q + qf [last stage]) (X + max|ref|); the float64
      // differences and the stage-gradient rows are truncated once (2u) and
      // summed (u).  Every cell's |K_split - K| is below the bound.
      const double u32 = 5.9604644775390625e-08;
      const double Xm = f2d(mags[0]), Lm = f2d(mags[1]), Dm = f2d(mags[2]), Rm = f2d(mags[3]);
      double usum = 0.0;
      for (int a = 0; a < nu; ++a) usum += fabs(sm.u[a]);
      const double pmax = fabs(k0) * (Xm + 0.5 * fabs(k1) * Xm * Xm);
      const double dpmax = fabs(k0) * (1.0 + fabs(k1) * Xm);
      const double S = 4.0 * (cx + cy) * (pmax + dpmax * Lm) + fabs(b0) * usum +
                       (I.q + (last ? I.qf : 0.0)) * (Xm + Rm);
      const double e = u32 * (3.0 * Dm + 16.0 * h * S);
      atomicMax(&A.res_err[slot], (unsigned long long)__double_as_longlong(e));
    }
    atomicMax(&A.res_inf[slot], (unsigned long long)__double_as_longlong(sm.red_out[0]));
    atomicAdd(&A.res_sq[slot], sm.red_out[1]);
    if (k == 0 && A.res_first)
      atomicMax(&A.res_first[b], (unsigned long long)__double_as_longlong(sm.red_out[0]));
  }
  cl.sync();
  if (resid_only) return;

  // ---- P3: lower layer in T ----
  // the residual inputs are dead: restore the zero ring of the arrays they used
  zero_ring(y5, g);
  zero_ring(w1, g);
  zero_ring(y4, g);
  const T tcx = (T)cx, tcy = (T)cy, tb0 = (T)b0;
  const T auu = (T)(h * I.r + I.gamma);
  T* y5c = y5;
  T* y4c = y4;
  const Halo<T> hw1 = halo_of(w1, g, cl);
  struct PV {
    int p;
    T v;
  };
  struct PV2 {
    int p;
    T v, w;
  };
  const int n_full = A.local_u ? 1 : A.n_u_it + 1;  // full-field Y applications
  for (int it = 0; it < n_full; ++it) {
    if (it > 0) {
      // c4 = F_u v3 - K1 changes only on actuator cells: refresh v1, p1 there
      for (int a = tid; a < nu; a += bd) {
        const int c = sm.act[a];
        const int q = c - g.lo;
        bool first = (q >= 0 && q < n);
        for (int a2 = 0; a2 < a && first; ++a2)
          if (sm.act[a2] == c) first = false;
        if (first) {
          T inj = T(0);
          for (int a2 = 0; a2 < nu; ++a2)
            if (sm.act[a2] == c) inj += sm.v3[a2];
          const int p = g.pidx(q);
          const T v = (th * tb0 * inj - sm.b1a[a]) * rg[p];
          v1[p] = v;
          put(p1, hp1, g, q, p, dp[p] * v);
        }
      }
      cl.sync();
    }
    // F_x v5 = c4 by n_lo pointwise Jacobi sweeps from zero: sweep 1 is v1;
    // sweep s+1 = v1 - D^{-1} (offdiag F_x) sweep s, reading neighbours.  The
    // last sweep also forms sweep 1 of F_x^T v4 = -K3 - A_xx v5 (own cells).
    T* cur = v1;
    if (n_lo == 1) {
      pass<CPT, PV>(n,
          [&](int q) {
            const int p = g.pidx(q);
            return PV{p, (-b2[p] - ax[p] * v1[p]) * rg[p]};
          },
          [&](int q, PV o) { put(w1, hw1, g, q, o.p, o.v); });
    } else {
      cur = y5;
      const Halo<T> hc = halo_of(cur, g, cl);
      const bool lastsw = (n_lo == 2);
      pass<CPT, PV2>(n,
          [&](int q) {
            const int p = g.pidx(q);
            const T off = th * stencil<T>(g, p, tcx, tcy, [&](int m) { return p1[m]; });
            const T v = v1[p] - rg[p] * off;
            return PV2{p, v, (-b2[p] - ax[p] * v) * rg[p]};
          },
          [&](int q, PV2 o) {
            if (wide) put(cur, hc, g, q, o.p, o.v);
            else cur[o.p] = o.v;
            if (lastsw) put(w1, hw1, g, q, o.p, o.w);
          });
      T* nxt = e1;
      for (int sw = 2; sw < n_lo; ++sw) {
        cl.sync();
        const Halo<T> hn = halo_of(nxt, g, cl);
        const bool fin = (sw == n_lo - 1);
        pass<CPT, PV2>(n,
            [&](int q) {
              const int p = g.pidx(q);
              const T off = th * stencil<T>(g, p, tcx, tcy, [&](int m) { return dp[m] * cur[m]; });
              const T v = v1[p] - rg[p] * off;
              return PV2{p, v, (-b2[p] - ax[p] * v) * rg[p]};
            },
            [&](int q, PV2 o) {
              put(nxt, hn, g, q, o.p, o.v);
              if (fin) put(w1, hw1, g, q, o.p, o.w);
            });
        T* t = cur; cur = nxt; nxt = t;
      }
    }
    y5c = cur;
    cur = w1;
    if (n_lo >= 2) {
      cl.sync();
      cur = y4;
      const Halo<T> hc = halo_of(cur, g, cl);
      pass<CPT, PV>(n,
          [&](int q) {
            const int p = g.pidx(q);
            const T off = th * dp[p] * stencil<T>(g, p, tcx, tcy, [&](int m) { return w1[m]; });
            return PV{p, w1[p] - rg[p] * off};
          },
          [&](int q, PV o) {
            if (wide) put(cur, hc, g, q, o.p, o.v);
            else cur[o.p] = o.v;
          });
      T* nxt = (y5c == e1) ? e2 : e1;  // the spare that does not hold v5
      for (int sw = 2; sw < n_lo; ++sw) {
        cl.sync();
        const Halo<T> hn = halo_of(nxt, g, cl);
        pass<CPT, PV>(n,
            [&](int q) {
              const int p = g.pidx(q);
              const T off = th * dp[p] * stencil<T>(g, p, tcx, tcy, [&](int m) { return cur[m]; });
              return PV{p, w1[p] - rg[p] * off};
            },
            [&](int q, PV o) { put(nxt, hn, g, q, o.p, o.v); });
        T* t = cur; cur = nxt; nxt = t;
      }
    }
    y4c = cur;
    if (A.local_u || it < A.n_u_it) {
      cl.sync();  // Y(.) at the actuator cells is read across ranks below
      if (!A.local_u) {
        // A_uu v3 = K2 + F_u^T y_lambda (A_ux = 0); every rank keeps all of v3
        for (int a = tid; a < nu; a += bd)
          sm.v3[a] = (sm.b3[a] + th * tb0 * *at(y4c, sm.act[a], g, cl)) / auu;
        __syncthreads();
      }
    }
  }
  if (A.local_u) {
    // Y(v3) = Y(0) + sum_b v3_b Z(e_b), Z(e_b) = P^{-1}(F_u e_b, 0): the fixed
    // sweeps are linear and Z(e_b) vanishes outside a box of half-width
    // R = 2 (n_lo - 1) around actuator b (each sweep reaches one cell further).
    // The u-iteration then needs Y(0) at the actuator cells and the boxes.
    for (int a = tid; a < nu; a += bd) sm.y4a[a] = *at(y4c, sm.act[a], g, cl);
    const int R = A.box_r;
    const int mx = I.mx, my = I.my;
    const int Sx = 2 * R + 1, Sy = (I.dim == 2) ? 2 * R + 1 : 1, Ry = (I.dim == 2) ? R : 0;
    const int S2 = Sx * Sy;
    T* boxes = wk + (size_t)NUM_WORK_ARRAYS * SM;
    const int lane = tid & 31, nw = bd >> 5;
    for (int bb = tid >> 5; bb < nu; bb += nw) {
      T* z5 = boxes + (size_t)bb * 4 * S2;
      T* z4 = z5 + S2;
      T* t0 = z5 + 2 * S2;
      T* t1 = z5 + 3 * S2;
      const int ca = sm.act[bb], ixb = ca % mx, iyb = ca / mx;
      auto cell = [&](int j, int i, int& c) {
        const int gy = iyb + j - Ry, gx = ixb + i - R;
        c = gy * mx + gx;
        return gx >= 0 && gx < mx && gy >= 0 && gy < my;
      };
      // off-diagonal stencil of a box field v at box cell (j, i), weight on the neighbour
      auto boxnbr = [&](const T* v, int j, int i, bool with_dp) {
        T sx = T(0), sy = T(0);
        int c;
        if (i > 0 && cell(j, i - 1, c)) sx += (with_dp ? *at(dp, c, g, cl) : T(1)) * v[j * Sx + i - 1];
        if (i < Sx - 1 && cell(j, i + 1, c)) sx += (with_dp ? *at(dp, c, g, cl) : T(1)) * v[j * Sx + i + 1];
        if (j > 0 && cell(j - 1, i, c)) sy += (with_dp ? *at(dp, c, g, cl) : T(1)) * v[(j - 1) * Sx + i];
        if (j < Sy - 1 && cell(j + 1, i, c)) sy += (with_dp ? *at(dp, c, g, cl) : T(1)) * v[(j + 1) * Sx + i];
        return tcx * sx + tcy * sy;
      };
      const T v1c = th * tb0 * *at(rg, ca, g, cl);  // first F_x sweep: D^{-1} h b0 e_b
      for (int q = lane; q < S2; q += 32) t0[q] = (q == Ry * Sx + R) ? v1c : T(0);
      __syncwarp();
      T* cur = t0;
      T* nxt = t1;
      for (int sw = 1; sw < n_lo; ++sw) {
        for (int q = lane; q < S2; q += 32) {
          const int j = q / Sx, i = q % Sx;
          int c;
          T v = T(0);
          if (cell(j, i, c))
            v = ((q == Ry * Sx + R) ? v1c : T(0)) - *at(rg, c, g, cl) * th * boxnbr(cur, j, i, true);
          nxt[q] = v;
        }
        __syncwarp();
        T* t = cur; cur = nxt; nxt = t;
      }
      for (int q = lane; q < S2; q += 32) z5[q] = cur[q];
      __syncwarp();
      // F_x^T sweeps with right-hand side -A_xx z5: w^1 stays in t0; the
      // n_lo - 1 later sweeps alternate between t1 and z4, the last one in z4
      for (int q = lane; q < S2; q += 32) {
        const int j = q / Sx, i = q % Sx;
        int c;
        t0[q] = cell(j, i, c) ? -*at(ax, c, g, cl) * z5[q] * *at(rg, c, g, cl) : T(0);
      }
      __syncwarp();
      if (n_lo == 1) {
        for (int q = lane; q < S2; q += 32) z4[q] = t0[q];
      } else {
        const T* src = t0;
        for (int sw = 1; sw < n_lo; ++sw) {
          T* dst = (((n_lo - 1 - sw) & 1) == 0) ? z4 : t1;
          for (int q = lane; q < S2; q += 32) {
            const int j = q / Sx, i = q % Sx;
            int c;
            T v = T(0);
            if (cell(j, i, c))
              v = t0[q] - *at(rg, c, g, cl) * th * *at(dp, c, g, cl) * boxnbr(src, j, i, false);
            dst[q] = v;
          }
          __syncwarp();
          src = dst;
        }
      }
      __syncwarp();
    }
    cl.sync();  // boxes ready; every rank has read Y(0) at the actuator cells
    // u fixed-point iteration on n_u numbers: y_lambda(act_a) = Y(0) + sum_b G_ab v3_b
    for (int it = 0; it < A.n_u_it; ++it) {
      for (int a = tid; a < nu; a += bd) {
        T y = sm.y4a[a];
        const int ca = sm.act[a], ixa = ca % mx, iya = ca / mx;
        for (int bb = 0; bb < nu; ++bb) {
          const int cb = sm.act[bb];
          const int di = ixa - cb % mx + R, dj = iya - cb / mx + Ry;
          if (di >= 0 && di < Sx && dj >= 0 && dj < Sy)
            y += sm.v3[bb] * boxes[(size_t)bb * 4 * S2 + S2 + dj * Sx + di];
        }
        sm.v3n[a] = (sm.b3[a] + th * tb0 * y) / auu;
      }
      __syncthreads();
      for (int a = tid; a < nu; a += bd) sm.v3[a] = sm.v3n[a];
      __syncthreads();
    }
    // Y(v3) = Y(0) + sum_b v3_b Z(e_b) on this rank's cells
    for (int e = tid; e < nu * S2; e += bd) {
      const int bb = e / S2, q = e % S2;
      const int cb = sm.act[bb];
      const int gy = cb / mx + q / Sx - Ry, gx = cb % mx + q % Sx - R;
      if (gx < 0 || gx >= mx || gy < 0 || gy >= my) continue;
      const int c = gy * mx + gx;
      const int qc = c - g.lo;
      if (qc < 0 || qc >= n) continue;
      const int p = g.pidx(qc);
      const T* z5 = boxes + (size_t)bb * 4 * S2;
      atomicAdd(&y5c[p], sm.v3[bb] * z5[q]);
      atomicAdd(&y4c[p], sm.v3[bb] * z5[S2 + q]);
    }
    __syncthreads();
  }
  // back-solve (eq. 23b): (v1, v2) = P^{-1}(K1 - F_u v3, K3) = -Y(v3)

  // ---- P4: S_i <- S_i - alpha Delta s_i (float64) ----
  const double alpha = A.alpha;
  double* Xo = A.xout[rd ^ 1] + so + g.lo;
  double* Lo = A.lout[rd ^ 1] + so + g.lo;
  double* Uo = A.uout[rd ^ 1];
  struct D2 {
    double x, l;
  };
  pass<CPT, D2>(n,
      [&](int q) {
        const int p = g.pidx(q);
        return D2{fma(alpha, to_double(y5c[p]), OX(q, p)), fma(alpha, to_double(y4c[p]), OL(q, p))};
      },
      [&](int q, D2 o) {
        Xo[q] = o.x;
        Lo[q] = o.l;
      });
  if (cl.rank == 0)
    for (int a = tid; a < nu; a += bd)
      Uo[I.u_off + (long long)s * nu + a] = sm.u[a] - alpha * (double)sm.v3[a];
  cl.sync();
}

// CPT: cells per thread per pass round (2 or 4); with 4 the register budget
// of a thread grows and the CTA is limited to 384 threads.
template <typename T, int MODE, int CPT>
__global__ void __launch_bounds__(CPT >= 4 ? 384 : 512) k_iterate(IterArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallShared<T>& sm = *reinterpret_cast<SmallShared<T>*>(smem_raw);
  T* wk;
  double* gstage = nullptr;
  if (A.scratch == nullptr) {
    const size_t off = (sizeof(SmallShared<T>) + 15) & ~size_t(15);
    gstage = A.stage ? reinterpret_cast<double*>(smem_raw + off) : nullptr;
    wk = reinterpret_cast<T*>(
        smem_raw + off + (A.stage ? (size_t)NUM_STAGE_ARRAYS * A.slab_max * sizeof(double) : 0));
  } else {
    wk = reinterpret_cast<T*>(A.scratch + (long long)blockIdx.x * A.scratch_stride);
  }
  Cl cl;
  cl.C = A.csize;
  cl.rank = (A.csize > 1) ? (int)cg::this_cluster().block_rank() : 0;
  sm.amask[threadIdx.x] = 0ull;
  if (MODE == MODE_ONESHOT) __syncthreads();  // solve mode: the prologue's barrier
  const int k = (MODE == MODE_SOLVE) ? *(volatile int*)A.iter_k : 0;
  const int n_clusters = gridDim.x / A.csize;

  for (int w = blockIdx.x / A.csize; w < A.n_work; w += n_clusters) {
    const int2 item = A.work[w];
    const int b = item.x, s = item.y;
    bool resid_only = false;
    bool full = true;
    if (MODE == MODE_ONESHOT) {
      resid_only = (A.resid_only != 0);
      full = resid_only || (A.full_all != 0);
    } else {
      if (threadIdx.x == 0) {
        int skip = 0, fl = 1;
        if (k > A.max_iter || A.status[b] != ST_RUNNING) {
          skip = 1;
        } else {
          const int ffrom = A.full_from[b];
          const int f0 = A.full0[b];
          int st = ST_RUNNING;
          bool switch_now = false;
          double r = 0.0;
          int pslot = 0;
          if (k > 0) {
            pslot = ((k - 1) % RES_SLOTS) * A.n_inst + b;
            r = __longlong_as_double((long long)A.res_inf[pslot]);
            const double r0 = __longlong_as_double((long long)A.res_first[b]);
            const bool prev_full = (k - 1 >= ffrom) || (k == 1 && f0);
            if (!(r <= 1.79e308) || r > A.div_limit * fmax(r0, 1e-300)) st = ST_DIVERGED;
            else if (prev_full && r <= A.tol) st = ST_CONVERGED;
            else if (!prev_full) {
              // leave the split residual once it can no longer show that the
              // float64 residual is above the threshold: r minus its rounding
              // bound at or below max(tol, split_min)
              const double e = __longlong_as_double((long long)A.res_err[pslot]);
              if (r - e <= fmax(A.tol, A.split_min)) switch_now = true;
            }
          }
          if (st != ST_RUNNING) {
            skip = 1;
            if (s == 0 && cl.rank == 0) {
              A.status[b] = st;
              A.iters[b] = k - 1;
              A.final_buf[b] = (k - 1) & 1;
              A.fin_inf[b] = r;
              A.fin_2[b] = sqrt(A.res_sq[pslot]);
              atomicSub(A.n_active, 1);
            }
          } else {
            fl = (A.full_all || k >= ffrom || switch_now || k == A.max_iter || (k == 0 && f0))
                     ? 1 : 0;
            if (s == 0 && cl.rank == 0) {
              if (fl && ffrom > k) A.full_from[b] = k;
              const int nslot = ((k + 1) % RES_SLOTS) * A.n_inst + b;
              A.res_inf[nslot] = 0ull;
              A.res_err[nslot] = 0ull;
              A.res_sq[nslot] = 0.0;
            }
          }
        }
        sm.skip = skip;
        sm.full = fl;
      }
      __syncthreads();
      const bool sk = sm.skip != 0;
      full = sm.full != 0;
      __syncthreads();
      if (sk) continue;  // uniform across the cluster: every rank read the same slots
      resid_only = (k == A.max_iter);
    }
    process_item<T, CPT>(A, b, s, k, (MODE == MODE_SOLVE) ? (k & 1) : 0, full, resid_only, sm, wk,
                    cl, gstage);
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

// Reset the per-instance control and write S^0 into buffer 0: the cold start
// (mode 0), nothing (mode 1: buffer 0 already holds S^0) or the current state
// shifted by one stage with the last stage repeated (mode 2; receding
// horizon, the paper's closed loop).  first_full: iteration 0 evaluates the
// float64 residual (warm starts that may already be converged).
__global__ void k_init_control(IterArgs A, int mode, int first_full, const double* xc,
                               const double* uc, const double* lc) {
  const int b = blockIdx.y;
  if (b >= A.n_inst) return;
  const InstDev I = A.inst[b];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int q = 0; q < RES_SLOTS; ++q) {
      A.res_inf[q * A.n_inst + b] = 0ull;
      A.res_err[q * A.n_inst + b] = 0ull;
      A.res_sq[q * A.n_inst + b] = 0.0;
    }
    A.res_first[b] = 0ull;
    A.status[b] = ST_RUNNING;
    A.iters[b] = 0;
    A.final_buf[b] = 0;
    A.fin_inf[b] = 0.0;
    A.fin_2[b] = 0.0;
    A.full_from[b] = A.full_all ? 0 : 0x7fffffff;
    A.full0[b] = first_full;
    if (b == 0) {
      *A.n_active = A.n_inst;
      *A.iter_k = 0;
      *A.block_done = 0;
    }
  }
  if (mode == 1) return;
  const long long n = (long long)I.N * I.ng;
  double* X = A.xout[0];
  double* L = A.lout[0];
  double* U = A.uout[0];
  const long long nu_all = (long long)I.N * I.nu;
  if (mode == 0) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
      X[I.s_off + e] = A.x0[I.g_off + (e % I.ng)];
      L[I.s_off + e] = 0.0;
    }
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nu_all;
         e += (long long)gridDim.x * blockDim.x)
      U[I.u_off + e] = 0.0;
    return;
  }
  // shift: stage i takes stage i+1 of the current state; the last is repeated
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / I.ng;
    const long long src = (i + 1 < I.N) ? e + I.ng : e;
    X[I.s_off + e] = xc[I.s_off + src];
    L[I.s_off + e] = lc[I.s_off + src];
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nu_all;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / I.nu;
    U[I.u_off + e] = uc[I.u_off + ((i + 1 < I.N) ? e + I.nu : e)];
  }
}

// One explicit-Euler sub-step of the plant for every instance:
//   w_out = w_in + (dt / n_sub) (Lap Phi(w_in) + b0 B u_1),
// u_1 the first-stage controls of the current solution (u_cur).  Optionally
// records u_1 into u_rec (packed [sum n_u]).
__global__ void k_plant_substep(const InstDev* inst, int n_inst, const int* act,
                                const double* w_in, double* w_out, const double* u_cur,
                                double* u_rec, double dt_all, int n_sub) {
  const int b = blockIdx.y;
  if (b >= n_inst) return;
  const InstDev I = inst[b];
  // each instance's sampling period is its own stage length unless dt_all > 0
  const double dt = ((dt_all > 0.0) ? dt_all : I.h) / n_sub;
  const double* wi = w_in + I.g_off;
  const double cx = I.cx, cy = I.cy, k0 = I.k0, k1 = I.k1;
  const double dc = 2.0 * (cx + cy);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < I.ng; c += gridDim.x * blockDim.x) {
    const int ix = c % I.mx, iy = c / I.mx;
    double src = 0.0;
    for (int a = 0; a < I.nu; ++a)
      if (act[I.act_off + a] == c) src += u_cur[I.u_off + a];
    const double lphi = nbr_sum<double>(c, ix, iy, I.mx, I.my, cx, cy,
                                        [&](int m) { return phi_d(wi[m], k0, k1); }) -
                        dc * phi_d(wi[c], k0, k1);
    w_out[I.g_off + c] = wi[c] + dt * (lphi + I.b0 * src);
  }
  if (u_rec && blockIdx.x == 0)
    for (int a = threadIdx.x; a < I.nu; a += blockDim.x)
      u_rec[I.act_off + a] = u_cur[I.u_off + a];
}

// After the iteration chunks: settle instances still running at max_iter,
// gather every instance's returned iterate into the "current" buffers and
// u_out.  xs/us/ls[0..1] are the ping-pong buffers.
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
    // iteration max_iter always evaluates the float64 residual
    const int slot = (F.max_iter % RES_SLOTS) * F.n_inst + b;
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
