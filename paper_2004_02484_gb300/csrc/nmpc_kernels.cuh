// Device code of the double-layer Jacobi NMPC solver (sm_103a).
//
// One thread-block cluster of C CTAs processes one (instance, stage) work
// item of one upper-layer iteration (eq. 15); every stage of every instance
// is updated at once from iterate k, so one launch is one iteration.  The
// stage grid is split into C slabs (rows in 2D, segments in 1D) held as
// padded records in shared memory; a CTA also stores its boundary values into
// the neighbouring CTAs' halo records through the cluster's distributed shared
// memory, so every stencil read is local.  Inside a work item:
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
#include <type_traits>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stddef.h>
#include <stdint.h>

namespace nmpc_dev {

namespace cg = cooperative_groups;

constexpr int RES_SLOTS = 16;    // rolling residual history per instance
// iterations over which a split residual r with r - e <= threshold (e its
// rounding bound) that has not decreased hands over to the float64 residual
// although r itself stays above the threshold (its rounding floor)
constexpr int SPLIT_PATIENCE = 12;
static_assert(SPLIT_PATIENCE + 2 < RES_SLOTS, "history slots read by decide()");
// res_err of an iteration that evaluated the float64 residual (above the bits
// of every non-negative double or NaN, so atomicMax keeps it)
constexpr unsigned long long RES_FULL_MARK = 0xfff0000000000000ull;
constexpr int MAX_NU = 64;

struct InstDev {
  int dim, mx, my, ng;
  int N, nu, act_off, pad;
  long long s_off;  // offset of stage 1 in packed x / lam
  long long u_off;  // offset in packed u
  long long g_off;  // offset in packed x0 / ref
  double h, q, r, qf, gamma, k0, k1, b0, cx, cy;
  // derived (derive()): float64 2 (cx + cy), h qf, h r + gamma; float32 copies
  double dcoef, hqf, auu;
  float fh, fcx, fcy, fdc, fk0, fk1, fk1h, fk01, fq, fb0, fhqf, fauu;
};

// Fill the derived fields of an instance from its parameters.
__host__ __device__ inline void derive(InstDev& I) {
  I.dcoef = 2.0 * (I.cx + I.cy);
  I.hqf = I.h * I.qf;
  I.auu = I.h * I.r + I.gamma;
  I.fh = (float)I.h;
  I.fcx = (float)I.cx;
  I.fcy = (float)I.cy;
  I.fdc = (float)I.dcoef;
  I.fk0 = (float)I.k0;
  I.fk1 = (float)I.k1;
  I.fk1h = (float)(0.5 * I.k1);
  I.fk01 = (float)(I.k0 * I.k1);
  I.fq = (float)I.q;
  I.fb0 = (float)I.b0;
  I.fhqf = (float)I.hqf;
  I.fauu = (float)I.auu;
}

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
  unsigned long long* res_inf;   // [RES_SLOTS][n_inst], bits of non-negative doubles
  unsigned long long* res_err;   // [RES_SLOTS][n_inst] bound on a split residual's rounding error
  double* res_sq;                // [RES_SLOTS][n_inst]
  unsigned long long* res_first; // [n_inst] ||K(S^0)||_inf
  int* status;
  int* iters;
  int* final_buf;
  double* fin_inf;
  double* fin_2;
  int* f64_count;  // [n_inst] iterations that evaluated the float64 residual
  int* full0;      // [n_inst] 1: iteration 0 does (warm starts)
  int* n_active;
  // persistent launch: [0] barrier arrivals, [1] barrier generation, [2] stop
  // (no instance running), [3] a wait ran out of time
  unsigned* gsync;
  double tol, div_limit, alpha;
  double split_min;  // below max(tol, split_min) iterations use the float64 residual
  int max_iter, n_lo, n_u_it;
  // upper-layer variant: 0 Jacobi (eq. 15, every stage from iterate k);
  // 1 red-black Gauss-Seidel (the stage-block form of eq. 18 in the order
  // even stages, then odd stages): an iteration is two launches, half 0
  // updating the even 0-based stages from iterate k, half 1 the odd ones
  // with x_{i-1}, lambda_{i+1} already updated (launch index j = 2 i + half)
  int rb;
  // red-black: the cluster, strip and patch lists hold the items of even
  // stages first (this many), then those of odd stages; a half-sweep
  // launch covers its own range only
  int n_work_even, n_strips_even, n_patches_even;
  long long grid_wait;  // spin budget of one grid-barrier wait (SM clock cycles)
  int resid_only;  // one-shot: residual norms only (float64)
  int full_all;    // every residual in float64 (FP64 precision)
  int csize;       // CTAs per work item (cluster size)
  int stage;       // float64 slab inputs staged in shared memory (1) or read in place
  int local_u;     // u-iteration through the actuators' local responses (1) or full sweeps
  int box_r;       // half-width of a local-response box, 2 (n_lo - 1)
  int slab_max;    // records per slab (padded positions, halo rows and pads included)
  // lower-layer work arrays: shared memory (scratch == nullptr) or a global
  // slab of scratch_stride bytes per CTA
  char* scratch;
  long long scratch_stride;
  // strip path (k_strip): (instance, stage, first own column, first own row)
  // per strip
  const int4* strips;
  int n_strips;
  int strip_x, strip_y;  // own columns and rows per strip
  const float* ref_f;    // ref truncated to float32 (d2f) for k_strip2's split residual
  // the tail plan (k_strip2, solves): strips of tail_y own rows, taken by a
  // launch when the running-instance count that k_patch recorded before it
  // (*strip_run) is at most tail_below (n_tail = 0: no tail plan)
  const int4* tail;
  int n_tail, n_tail_even, tail_y, tail_below;
  int* strip_run;
  // k_patch: (instance, stage, actuator) per warp; v3 per control (float64)
  const int4* patches;
  int n_patches;
  double* v3g;
  // line path (k_line): (instance, stage, cells per lane, 0) per 1D stage;
  // solve mode walks the items of running instances (k_compact_lines)
  const int4* lines;
  int n_lines;
  int4* lines_act;
  int* n_lines_act;
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

// ---------------------------------------------------------------------------
// Work-item slab in shared memory (or a global scratch slab).
//
// The stage grid is split across the C cluster ranks in whole rows (2D) or
// segments (1D), `per` rows or cells per rank (the last non-empty rank may
// hold fewer, later ranks none).  2D: a rank's slab is a padded layout of
// (rows + 2) x W positions, W = mx + 2, interior cell (row j, column i) at
// p = (j + 1) W + i + 1; padded rows 0 and rows + 1 hold the neighbouring
// ranks' boundary rows (the halo) or zeros at the grid's Dirichlet ring,
// columns 0 and W - 1 are zero.  1D: one padded row, cell q at p = q + 1,
// positions 0 and n + 1 the halo or zero.  The five-point stencil reads
// p +- 1 and p +- Wv with Wv = W in 2D and Wv = 0 in 1D (the cell itself,
// under the zero vertical weight).  Each position holds one record of
// NUM_FIELDS values of T (work record) and, when the float64 inputs are
// staged, one record of NUM_SFIELDS doubles: a field access is one
// shared-memory access at a fixed offset from the record.  A rank that writes
// a boundary value also stores it into the neighbour's halo record.
enum WField { F_B2 = 0, F_DP, F_AX, F_RG, F_V1, F_P1, F_Y5, F_W1, F_Y4, F_E1, F_E2, NUM_FIELDS };
// NUM_FIELDS is odd: consecutive records start in distinct banks.
// Split residual: float copies of x, lambda and Phi(x) in the F_Y5, F_W1 and
// F_Y4 fields (dead before those are written).
enum SField { S_X = 0, S_L, S_XP, S_LN, S_RF, S_PH };
constexpr int NUM_SFIELDS = 7;  // 14 words per record: 16 consecutive records hit distinct bank pairs

struct Geo {
  int n;       // cells of this rank
  int cols;    // cells per interior row: 2D mx, 1D n
  int rows;    // interior rows: 2D slab rows, 1D 1
  int W;       // padded row length
  int Wv;      // position distance of the vertical stencil neighbours: 2D W, 1D 0
  int p0;      // position of the first cell: 2D W + 1, 1D 1
  int plen;    // padded positions: 2D (rows + 2) W, 1D n + 2
  int lo;      // first grid cell of the slab
  int r0;      // first grid row (2D) / cell (1D) of the slab
  int per;     // rows (2D) / cells (1D) per rank
  int edge;    // cells of the first (last) row: 2D mx, 1D 1
  int up_off;  // position shift into rank - 1's layout (its bottom / right halo)
  int dn_off;  // position shift back into rank + 1's layout (its top / left halo)
  bool d2;     // 2D grid
  bool up, dn; // rank - 1 / rank + 1 hold cells and exchange halos with this rank
};

__device__ __forceinline__ Geo geo_of(const InstDev& I, int C, int rank) {
  Geo g;
  g.d2 = (I.dim == 2);
  const int nun = g.d2 ? I.my : I.mx;
  g.per = (nun + C - 1) / C;
  const int a = min(rank * g.per, nun), b = min(a + g.per, nun);
  g.r0 = a;
  g.n = g.d2 ? (b - a) * I.mx : b - a;
  g.cols = g.d2 ? I.mx : b - a;
  g.rows = g.d2 ? b - a : 1;
  g.W = g.d2 ? I.mx + 2 : g.per + 2;
  g.Wv = g.d2 ? g.W : 0;
  g.p0 = g.d2 ? g.W + 1 : 1;
  g.plen = g.d2 ? (g.rows + 2) * g.W : g.n + 2;
  g.lo = g.d2 ? a * I.mx : a;
  g.edge = g.d2 ? I.mx : 1;
  g.up_off = g.d2 ? g.per * g.W : g.per;
  g.dn_off = g.d2 ? (b - a) * g.W : (b - a);
  g.up = (rank > 0) && (b > a);
  g.dn = (b < nun) && (b > a);
  return g;
}

// The NC cells a thread carries through a pass: positions, and bit masks of
// the slots that hold a cell and of those whose value also goes to
// rank - 1's / rank + 1's halo.  Slot k holds cell q = first + k blockDim.  A
// slot past the slab gets position p0, whose stencil neighbours lie inside
// every rank's records: its loads are harmless, its stores are skipped.
template <int NC>
struct Cells {
  int p[NC];
  unsigned valid, pu, pd;
};

template <int NC>
__device__ __forceinline__ Cells<NC> cells_of(const Geo& g, int first) {
  Cells<NC> cs;
  cs.valid = 0u;
  cs.pu = 0u;
  cs.pd = 0u;
  const int bd = blockDim.x;
  const int cols = max(g.cols, 1);
  int j = first / cols, i = first - j * cols;
  const int dj = bd / cols, di = bd - dj * cols;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const int q = first + k * bd;
    const bool v = q < g.n;
    cs.p[k] = v ? g.p0 + j * g.W + i : g.p0;
    cs.valid |= (v ? 1u : 0u) << k;
    cs.pu |= ((v && g.up && q < g.edge) ? 1u : 0u) << k;
    cs.pd |= ((v && g.dn && q >= g.n - g.edge) ? 1u : 0u) << k;
    i += di;
    j += dj;
    if (i >= cols) {
      i -= cols;
      ++j;
    }
  }
  return cs;
}

// Slot of a pass: mask bit (round * NC + k), slot k, cell q, position p, and
// whether it holds a cell.
struct Slot {
  int kk, k, q, p;
  bool v;
};

// One pass over the rank's cells.  Rounds of NC cells per thread (one round
// for shared-memory slabs, whose cells the host sizes to fit; several for
// global slabs); within a round, groups of G slots: every slot's loads and
// arithmetic (ld) come before the group's stores (st), so a group forms G
// independent dependency chains.
template <int NC, int G, bool MULTI, typename V, typename LD, typename ST>
__device__ __forceinline__ void pass(const Geo& g, const Cells<NC>& c0, LD ld, ST st) {
  static_assert(NC % G == 0, "group size must divide the cells per thread");
  const int rounds = MULTI ? (g.n + NC * (int)blockDim.x - 1) / (NC * (int)blockDim.x) : 1;
  for (int r = 0; r < rounds; ++r) {
    Cells<NC> cs = c0;
    if (MULTI && r > 0) cs = cells_of<NC>(g, threadIdx.x + r * NC * blockDim.x);
#pragma unroll
    for (int k0 = 0; k0 < NC; k0 += G) {
      V v[G];
#pragma unroll
      for (int k = 0; k < G; ++k) {
        const Slot sl{r * NC + k0 + k, k0 + k, (int)threadIdx.x + (r * NC + k0 + k) * (int)blockDim.x,
                      cs.p[k0 + k], ((cs.valid >> (k0 + k)) & 1u) != 0u};
        v[k] = ld(sl, cs);
      }
#pragma unroll
      for (int k = 0; k < G; ++k) {
        const Slot sl{r * NC + k0 + k, k0 + k, (int)threadIdx.x + (r * NC + k0 + k) * (int)blockDim.x,
                      cs.p[k0 + k], ((cs.valid >> (k0 + k)) & 1u) != 0u};
        st(sl, cs, v[k]);
      }
    }
  }
}

// Shared-memory address of a generic pointer into this CTA's shared memory,
// and the same location in cluster rank r's shared memory.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned map_rank(unsigned a, int r) {
  unsigned out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(a), "r"(r));
  return out;
}
// Store v to a cluster shared-memory address when flag != 0 (predicated, no branch).
__device__ __forceinline__ void push_if(unsigned addr, float v, unsigned flag) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q st.shared::cluster.f32 [%0], %1;\n}"
               :: "r"(addr), "f"(v), "r"(flag) : "memory");
}
__device__ __forceinline__ void push_if(unsigned addr, double v, unsigned flag) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q st.shared::cluster.f64 [%0], %1;\n}"
               :: "r"(addr), "d"(v), "r"(flag) : "memory");
}

// Programmatic dependent launch: let the next launch in the stream start its
// CTAs now, and wait until the previous launch has finished and its writes
// are visible (both no-ops for launches without the attribute).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Rank owning grid cell c and its padded position there.
__device__ __forceinline__ int owner_of(int c, const Geo& g, int mx, int& p) {
  if (g.d2) {
    const int row = c / mx, col = c - row * mx;
    const int r = row / g.per;
    p = (row - r * g.per + 1) * g.W + col + 1;
    return r;
  }
  const int r = c / g.per;
  p = c - r * g.per + 1;
  return r;
}

__device__ __forceinline__ double phi_d(double w, double k0, double k1) {
  return k0 * (w + 0.5 * k1 * w * w);
}

__device__ __forceinline__ double abs_or_inf(double v) {
  const double a = fabs(v);
  return (a <= 1.79e308) ? a : CUDART_INF;  // NaN and Inf count as +Inf
}

// max(a, b) that returns NaN when either is NaN (one instruction)
__device__ __forceinline__ float fmax_nan(float a, float b) {
  float d;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ double dmax_nan(double a, double b) {
  return (a != a) ? a : ((b != b || b > a) ? b : a);
}

// float64 <-> float32 by IEEE-754 bit manipulation on the integer ALUs (the
// float64 pipe issues 2 lanes per clock per SM on this part).  d2f truncates
// toward zero (relative error < 2^-23) for magnitudes in [2^-126, 2^128);
// the magnitude's high word is clamped to that range first (two min/max
// instructions instead of two compare/select pairs), so +-0 stays +-0,
// smaller magnitudes become floats below 2^-146 (of the right sign), and
// 2^128 and beyond, Inf and NaN become Inf or NaN (never a finite value).
// f2d is exact for normal floats; subnormal floats become +-0.
__device__ __forceinline__ float d2f(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned a = min(hi & 0x7fffffffu, 0x47f00000u);
  // exponent rebiased (1023 -> 127) and the top 23 mantissa bits, in one funnel shift
  const unsigned bits = __funnelshift_l(lo, max(a, 0x38000000u) - 0x38000000u, 3);
  return __uint_as_float(bits | (hi & 0x80000000u));
}

__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned a = b & 0x7fffffffu;
  unsigned hi = (a >> 3) + 0x38000000u;  // exponent rebiased (127 -> 1023)
  unsigned lo = a << 29;
  hi = (a < 0x00800000u) ? 0u : hi;  // zero or subnormal
  lo = (a < 0x00800000u) ? 0u : lo;
  hi = (a >= 0x7f800000u) ? (0x7ff00000u | (a >> 3)) : hi;  // Inf, NaN
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)lo);
}

// dst = d2f(src): a float32 copy of a float64 field with the kernels' own
// truncation (a copy read in place of truncating the field again every
// iteration).
__global__ void k_f32_copy(const double* src, float* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = d2f(src[i]);
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
    vmax = fmax_nan(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
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
      m = dmax_nan(m, red->mx[w]);
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

// Per-work-item shared scalars (the slab records follow).
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
  double lact[MAX_NU];  // lambda at the actuator cells
  int bar_code;         // persistent launch: the grid barrier's stop / error bits
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

// The float64 or the float32 copy of a constant, for arithmetic in T.
template <typename T>
__device__ __forceinline__ T pick(double d, float f);
template <>
__device__ __forceinline__ float pick<float>(double, float f) { return f; }
template <>
__device__ __forceinline__ double pick<double>(double d, float) { return d; }

// 1 / v rounded to nearest (the same value as the IEEE division)
__device__ __forceinline__ float rcp_T(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double rcp_T(double v) { return __drcp_rn(v); }

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}

// cp_async8 that writes zeros instead when `valid` is false (source size 0:
// nothing is read; src must still be a valid address)
__device__ __forceinline__ void cp_async8_zfill(void* dst_smem, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
               "r"(valid ? 8 : 0));
}

// Iteration index (relative to *iter_k) and half-sweep of launch j.
__device__ __forceinline__ int launch_iter(const IterArgs& A, int j) { return A.rb ? (j >> 1) : j; }
__device__ __forceinline__ int launch_half(const IterArgs& A, int j) { return A.rb ? (j & 1) : 0; }
// Whether stage s is updated by half-sweep `half` (every stage under Jacobi).
__device__ __forceinline__ bool stage_in_half(const IterArgs& A, int s, int half) {
  return !A.rb || ((s & 1) == half);
}

// Iteration k's decision for instance b, from its residual history
// (iteration k - 1), with no side effects: skip (finished before, or k past
// max_iter: `before`; or finished now: st != ST_RUNNING) and whether the
// residual is evaluated in float64.  Control words are read around L1 (other
// CTAs write them within a persistent launch).
struct Decision {
  int skip, full, before, st, pslot;
  double r;
};

__device__ __forceinline__ Decision decide(const IterArgs& A, int b, int k) {
  Decision d{0, 1, 0, ST_RUNNING, (k > 0) ? ((k - 1) % RES_SLOTS) * A.n_inst + b : 0, 0.0};
  // every control word the decision reads, loaded at once
  const int status_b = __ldcg(A.status + b);
  const int f0 = __ldcg(A.full0 + b);
  const unsigned long long r_bits = __ldcg(A.res_inf + d.pslot);
  const unsigned long long r0_bits = __ldcg(A.res_first + b);
  const unsigned long long e_bits = __ldcg(A.res_err + d.pslot);
  if (k > A.max_iter || status_b != ST_RUNNING) {
    d.skip = 1;
    d.before = 1;
    return d;
  }
  bool switch_now = false;
  if (k > 0) {
    d.r = __longlong_as_double((long long)r_bits);
    const double r0 = __longlong_as_double((long long)r0_bits);
    const bool prev_full = e_bits == RES_FULL_MARK;
    if (!(d.r <= 1.79e308) || d.r > A.div_limit * fmax(r0, 1e-300)) {
      d.st = ST_DIVERGED;
    } else if (prev_full && d.r <= A.tol) {
      d.st = ST_CONVERGED;
    } else {
      // evaluate the float64 residual of S^k once r (split or float64) is at
      // or below T = max(tol, split_min): it is then expected at or below T
      // (or the split residual could not resolve it).  A float64 residual
      // above T hands back to the split residual where the split residual
      // itself had reached T (the iterates' residual rose again) or the
      // float64 one was iteration 0's; a float64 phase that began on the
      // split residual's rounding floor or has lasted longer stays.  The
      // floor: a split residual with r - e <= T (it can no longer show that
      // the float64 residual is above T) and no lower than SPLIT_PATIENCE
      // iterations before.
      const double T = fmax(A.tol, A.split_min);
      if (d.r <= T) {
        switch_now = true;
      } else if (prev_full) {
        if (k >= 2) {
          const int sl = ((k - 2) % RES_SLOTS) * A.n_inst + b;
          const unsigned long long e2 = __ldcg(A.res_err + sl);
          const double r2 = __longlong_as_double((long long)__ldcg(A.res_inf + sl));
          switch_now = e2 == RES_FULL_MARK || !(r2 <= T);
        }
      } else {
        const double e = __longlong_as_double((long long)e_bits);
        if (d.r - e <= T && k - 1 - SPLIT_PATIENCE >= 0) {
          const int sl = ((k - 1 - SPLIT_PATIENCE) % RES_SLOTS) * A.n_inst + b;
          switch_now = d.r >= __longlong_as_double((long long)__ldcg(A.res_inf + sl));
        }
      }
    }
  }
  if (d.st != ST_RUNNING) {
    d.skip = 1;
  } else {
    d.full = (A.full_all || switch_now || k == A.max_iter || (k == 0 && f0)) ? 1 : 0;
  }
  return d;
}

// decide() for work item (b, s), taken by one thread; the CTA of stage 0,
// cluster rank 0 keeps the books: it records a finished instance (status,
// returned iterate k - 1), counts the float64-residual iterations, and clears
// the residual slot of iteration k + 1.
__device__ __noinline__ void control_decision(const IterArgs& A, int b, int s, int k, const Cl& cl,
                                              int& skip_out, int& full_out) {
  const Decision d = decide(A, b, k);
  if (!d.before && s == 0 && cl.rank == 0) {
    if (d.st != ST_RUNNING) {
      A.status[b] = d.st;
      A.iters[b] = k - 1;
      A.final_buf[b] = (k - 1) & 1;
      A.fin_inf[b] = d.r;
      A.fin_2[b] = sqrt(__ldcg(A.res_sq + d.pslot));
      atomicSub(A.n_active, 1);
    } else {
      if (d.full) A.f64_count[b] += 1;
      const int nslot = ((k + 1) % RES_SLOTS) * A.n_inst + b;
      A.res_inf[nslot] = 0ull;
      A.res_err[nslot] = 0ull;
      A.res_sq[nslot] = 0.0;
    }
  }
  skip_out = d.skip;
  full_out = d.full;
}

// Rounding bound of the split residual over a set of cells (unit roundoff
// u = 2^-24).  x and lambda are truncated to float32 (2u), Phi, Phi' and the
// five-point sums are evaluated in float32 (a few u each): with X, Lm the
// maxima of |x|, |lambda| over the cells and their stencil neighbours, every
// O(h) term is off by at most 16 u h S, S = 4 (cx + cy) (Phi_max + Phi'_max
// Lm) + b0 sum|u| + (q + qf [last stage]) (X + max|ref|); the float64
// differences and the stage-gradient rows are truncated once (2u) and summed
// (u).  With diff32 the differences are instead taken in float32 from the
// truncated values (2u each, then rounded: u), which adds 4u max(X, Lm) with
// X, Lm covering the neighbouring stages' values as well.  Every cell's
// |K_split - K| is below the bound.  It is evaluated in float32 (its own
// rounding, a few u relative, is far inside the factor 16) and rounded up by
// 1%.  mags: X, Lm, max |difference or K2|, max |ref|; usum: sum over the
// stage's controls of |u| (float32).
// With Gm >= 0 the Laplacian of Phi is instead summed in difference form,
// sum_n c_n k0 (x_n - x_c)(1 + k1/2 (x_n + x_c)), from the truncated values:
// each term is off by k0 (1 + |k1| X)(4u X + 7u Gm), Gm the largest
// neighbour difference, so that part of S is dcoef k0 (1 + |k1| X)(4 X + 7
// Gm) / 8 (no cancellation of the O(dcoef Phi) terms).
__device__ __forceinline__ double split_bound(const InstDev& I, bool last, const float* mags,
                                              float usum, bool diff32 = false, float Gm = -1.0f) {
  const float u32 = 5.9604645e-08f;
  const float Xm = mags[0], Lm = mags[1], Dm = mags[2], Rm = mags[3];
  const float ak0 = fabsf(I.fk0), ak1 = fabsf(I.fk1);
  const float pmax = ak0 * (Xm + 0.5f * ak1 * Xm * Xm);
  const float dpmax = ak0 * (1.0f + ak1 * Xm);
  const float phi_part = (Gm >= 0.0f) ? I.fdc * dpmax * (4.0f * Xm + 7.0f * Gm) * 0.125f
                                      : 2.0f * I.fdc * pmax;
  const float S = phi_part + 2.0f * I.fdc * dpmax * Lm + fabsf(I.fb0) * usum +
                  (I.fq + (last ? I.fhqf / I.fh : 0.0f)) * (Xm + Rm);
  const float Dterm = 3.0f * Dm + (diff32 ? 4.0f * fmaxf(Xm, Lm) : 0.0f);
  return f2d(1.01f * u32 * (Dterm + 16.0f * I.fh * S));
}

// Residual norms of a work item (max, sum of squares) and, for the split
// residual, its rounding bound (else RES_FULL_MARK), into iteration k's slot of
// instance b.
__device__ __forceinline__ void publish_residual(const IterArgs& A, int slot, int b, int k,
                                                 double rmax, double rsq, double e, bool full) {
  atomicMax(&A.res_err[slot], full ? RES_FULL_MARK : (unsigned long long)__double_as_longlong(e));
  atomicMax(&A.res_inf[slot], (unsigned long long)__double_as_longlong(rmax));
  atomicAdd(&A.res_sq[slot], rsq);
  if (k == 0 && A.res_first)
    atomicMax(&A.res_first[b], (unsigned long long)__double_as_longlong(rmax));
}

// One (instance, stage) work item of an upper-layer iteration on this rank's
// slab.  B: base of the slab region (shared memory when SMEM), work records at
// byte offset wk_off, staged float64 records at st_off (when `staged`).
// resident: the staged records, the zeroed ring, the actuator cells and the
// controls u still hold this item's state from the previous iteration of a
// persistent launch (only x_{i-1} and lambda_{i+1} are loaded).  keep: the
// update also goes into the staged records (own cells and the neighbours'
// halo copies) and into every rank's u, for the next resident iteration.
template <typename T, int NC, bool SMEM>
__device__ void process_item(const IterArgs& A, int b, int s, int k, int rd, bool full,
                             bool resid_only, SmallShared<T>& sm, char* B, int wk_off, int st_off,
                             bool staged, const Cl& cl, bool resident = false, bool keep = false,
                             bool rbn = false) {
  constexpr int TS = (int)sizeof(T);
  constexpr int RB = NUM_FIELDS * TS;  // bytes per work record
  constexpr int SB = NUM_SFIELDS * 8;  // bytes per staged record
  constexpr bool MULTI = !SMEM;        // global slabs: several rounds of cells per thread
  constexpr int G2 = (NC >= 2) ? 2 : 1;  // residual pass: two cells per group (register budget)
  const InstDev I = A.inst[b];
  const Geo g = geo_of(I, cl.C, cl.rank);
  const int nu = I.nu, N = I.N, ng = I.ng;
  const int tid = threadIdx.x, bd = blockDim.x;
  const long long so = I.s_off + (long long)s * ng;
  const double* __restrict__ X = A.xin[rd];
  const double* __restrict__ L = A.lin[rd];
  const double* __restrict__ Uin = A.uin[rd];
  const double* __restrict__ x0 = A.x0 + I.g_off;
  const double* __restrict__ ref = A.ref + I.g_off;
  const double h = I.h, cx = I.cx, cy = I.cy, k0 = I.k0, k1 = I.k1, b0 = I.b0;
  const double dcoef = I.dcoef;
  const bool last = (s == N - 1);
  const int n_lo = A.n_lo;
  const bool wide = n_lo > 2;  // sweeps 3.. read dp and the previous sweep at neighbours
  const int WRB = g.Wv * RB, WSB = g.Wv * SB;
  const Cells<NC> c0 = cells_of<NC>(g, tid);

  // field f of the work record at byte offset pb (relative to B); float view
  // for the split residual's copies; staged field f of record sb
  auto WV = [&](int pb, int f) -> T& { return *reinterpret_cast<T*>(B + pb + f * TS); };
  auto WF = [&](int pb, int f) -> float& { return *reinterpret_cast<float*>(B + pb + f * TS); };
  auto SV = [&](int sb, int f) -> double& { return *reinterpret_cast<double*>(B + sb + f * 8); };
  auto wpos = [&](int p) { return wk_off + p * RB; };
  auto spos = [&](int p) { return st_off + p * SB; };
  // this CTA's work records in the neighbours' shared memory (halo stores)
  // (mapa is given this CTA's record base, a valid local address; the
  // position shifts are applied to the mapped address, and every store lands
  // inside the neighbour's records)
  unsigned up_base = 0u, dn_base = 0u, sup_base = 0u, sdn_base = 0u;
  if constexpr (SMEM) {
    const unsigned mine = smem_u32(B) + (unsigned)wk_off;
    if (g.up) up_base = map_rank(mine, cl.rank - 1) + (unsigned)(g.up_off * RB);
    if (g.dn) dn_base = map_rank(mine, cl.rank + 1) - (unsigned)(g.dn_off * RB);
    if (keep) {
      const unsigned smine = smem_u32(B) + (unsigned)st_off;
      if (g.up) sup_base = map_rank(smine, cl.rank - 1) + (unsigned)(g.up_off * SB);
      if (g.dn) sdn_base = map_rank(smine, cl.rank + 1) - (unsigned)(g.dn_off * SB);
    }
  }
  // store v into field f of own position p and of the neighbours' halo copies
  // (slots past the slab store nothing)
  auto put = [&](const Cells<NC>& cs, const Slot& sl, int f, T v) {
    if (sl.v) WV(wpos(sl.p), f) = v;
    if constexpr (SMEM) {
      const unsigned rel = (unsigned)(sl.p * RB + f * TS);
      push_if(up_base + rel, v, (cs.pu >> sl.k) & 1u);
      push_if(dn_base + rel, v, (cs.pd >> sl.k) & 1u);
    }
  };
  // generic pointer to field f at grid cell c (this rank's or another rank's record)
  auto at = [&](int c, int f) -> T* {
    int p;
    const int r = owner_of(c, g, I.mx, p);
    T* a = reinterpret_cast<T*>(B + wpos(p) + f * TS);
    return (r == cl.rank) ? a : cl.map(a, r);
  };

  // actuators: controls of this stage, and per thread a bit mask of which of
  // its cells carry one (cell q is bit q / blockDim of thread q % blockDim)
  for (int a = tid; a < nu; a += bd) {
    if (!resident) {
      sm.act[a] = A.act[I.act_off + a];
      sm.u[a] = Uin[I.u_off + (long long)s * nu + a];
    }
    const int c = sm.act[a];
    sm.lact[a] = __ldcg(L + so + c);  // lambda at the actuator cell, for the stage-gradient row K2
    sm.v3[a] = T(0);
    const int q = c - g.lo;
    if (q >= 0 && q < g.n && q / bd < 64) atomicOr(&sm.amask[q % bd], 1ull << (q / bd));
  }
  // padded position pp -> grid cell (or -1 outside the grid), own flag
  const float invW = 1.0f / (float)g.W;
  auto grid_cell = [&](int pp, bool& own) {
    if (g.d2) {
      const int jj = fdiv(pp, g.W, invW), ii = pp - jj * g.W;
      own = jj >= 1 && jj <= g.rows && ii >= 1 && ii <= g.cols;
      const int gr = g.r0 - 1 + jj, gc = ii - 1;
      return (gr >= 0 && gr < I.my && gc >= 0 && gc < I.mx) ? gr * I.mx + gc : -1;
    }
    own = pp >= 1 && pp <= g.n;
    const int gc = g.r0 - 1 + pp;
    return (gc >= 0 && gc < I.mx) ? gc : -1;
  };
  if (resident) {
    // x_{i-1} (x0 is resident) and lambda_{i+1} of the own cells, around L1
    // (other CTAs wrote them in this launch)
    double xp_[NC], ln_[NC];
#pragma unroll
    for (int kq = 0; kq < NC; ++kq) {
      const bool v = (c0.valid >> kq) & 1u;
      const int c = g.lo + tid + kq * bd;
      xp_[kq] = (v && s > 0) ? __ldcg(X + so - ng + c) : 0.0;
      ln_[kq] = (v && !last) ? __ldcg(L + so + ng + c) : 0.0;
    }
#pragma unroll
    for (int kq = 0; kq < NC; ++kq) {
      if ((c0.valid >> kq) & 1u) {
        if (s > 0) SV(spos(c0.p[kq]), S_XP) = xp_[kq];
        SV(spos(c0.p[kq]), S_LN) = ln_[kq];
      }
    }
  } else if (staged) {
    // float64 inputs by asynchronous copies, all in flight at once; zero
    // outside the grid
    for (int pp = tid; pp < g.plen; pp += bd) {
      bool own;
      const int c = grid_cell(pp, own);
      const int sb = spos(pp);
      if (c >= 0) {
        cp_async8(&SV(sb, S_X), X + so + c);
        cp_async8(&SV(sb, S_L), L + so + c);
        if (own) {
          cp_async8(&SV(sb, S_XP), (s == 0) ? x0 + c : X + so - ng + c);
          if (!last) cp_async8(&SV(sb, S_LN), L + so + ng + c);
          cp_async8(&SV(sb, S_RF), ref + c);
        }
      } else {
        SV(sb, S_X) = 0.0;
        SV(sb, S_L) = 0.0;
      }
    }
  }
  // zero the work records that no rank writes in this item: the column pads
  // and the halo rows at the grid boundary (2D), the halo cells at the grid
  // boundary (1D)
  if (g.n > 0 && !resident) {
    auto zrec = [&](int p) {
#pragma unroll
      for (int f = 0; f < NUM_FIELDS; ++f) WV(wpos(p), f) = T(0);
    };
    if (g.d2) {
      for (int jj = tid; jj < g.rows + 2; jj += bd) {
        zrec(jj * g.W);
        zrec(jj * g.W + g.W - 1);
      }
      if (!g.up)
        for (int i = tid; i < g.W; i += bd) zrec(i);
      if (!g.dn)
        for (int i = tid; i < g.W; i += bd) zrec((g.rows + 1) * g.W + i);
    } else if (tid == 0) {
      if (!g.up) zrec(0);
      if (!g.dn) zrec(g.n + 1);
    }
  }
  if (staged && !resident) asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  // own-cell float64 inputs of slot sl (staged record, or global memory for
  // slots that hold a cell; zero otherwise)
  auto OX = [&](const Slot& sl) {
    return staged ? SV(spos(sl.p), S_X) : (sl.v ? X[so + g.lo + sl.q] : 0.0);
  };
  auto OL = [&](const Slot& sl) {
    return staged ? SV(spos(sl.p), S_L) : (sl.v ? L[so + g.lo + sl.q] : 0.0);
  };
  auto OXP = [&](const Slot& sl) {
    return staged ? SV(spos(sl.p), S_XP)
                  : (sl.v ? ((s == 0) ? x0[g.lo + sl.q] : X[so - ng + g.lo + sl.q]) : 0.0);
  };
  auto OLN = [&](const Slot& sl) {
    return staged ? SV(spos(sl.p), S_LN) : (sl.v ? L[so + ng + g.lo + sl.q] : 0.0);
  };
  auto ORF = [&](const Slot& sl) { return staged ? SV(spos(sl.p), S_RF) : (sl.v ? ref[g.lo + sl.q] : 0.0); };
  // red-black half 1 (rbn): x_{i-1} and lambda_{i+1} as updated by half 0 of
  // this iteration (the buffer being written); K_i with them is the
  // right-hand side of the Gauss-Seidel stage solve, K_i with the values of
  // iterate k (above) gives the norms of K(S^k)
  const double* __restrict__ XNw = A.xout[rd ^ 1];
  const double* __restrict__ LNw = A.lout[rd ^ 1];
  auto OXPN = [&](const Slot& sl) {
    return sl.v ? ((s == 0) ? x0[g.lo + sl.q] : XNw[so - ng + g.lo + sl.q]) : 0.0;
  };
  auto OLNN = [&](const Slot& sl) { return sl.v ? LNw[so + ng + g.lo + sl.q] : 0.0; };

  // ---- P1: residual inputs on the padded slab, halo rows included ----
  const float k0f = I.fk0, k1h = I.fk1h;
  // magnitudes for the split residual's rounding bound: max |x|, |lambda| over
  // the padded slab, max |float64 difference|, |ref| over the own cells
  float4 mg = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!full) {
    for (int p0 = tid; p0 < g.plen; p0 += 4 * bd) {
      float xv[4], lv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int pp = p0 + u * bd;
        double xd = 0.0, ld = 0.0;
        if (pp < g.plen) {
          if (staged) {
            xd = SV(spos(pp), S_X);
            ld = SV(spos(pp), S_L);
          } else {
            bool own;
            const int c = grid_cell(pp, own);
            if (c >= 0) {
              xd = X[so + c];
              ld = L[so + c];
            }
          }
        }
        xv[u] = d2f(xd);
        lv[u] = d2f(ld);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int pp = p0 + u * bd;
        if (pp < g.plen) {
          const int pb = wpos(pp);
          WF(pb, F_Y5) = xv[u];
          WF(pb, F_W1) = lv[u];
          WF(pb, F_Y4) = k0f * (xv[u] + k1h * xv[u] * xv[u]);
          mg.x = fmaxf(mg.x, fabsf(xv[u]));
          mg.y = fmaxf(mg.y, fabsf(lv[u]));
        }
      }
    }
  } else if (staged) {
    for (int pp = tid; pp < g.plen; pp += bd) SV(spos(pp), S_PH) = phi_d(SV(spos(pp), S_X), k0, k1);
  }
  __syncthreads();

  // ---- P2: K_i (eq. 9), coefficient fields, norms ----
  double vmax = 0.0, vsq = 0.0;
  float fmax_ = 0.0f, fsq = 0.0f;
  const T th = pick<T>(h, I.fh), tdc = pick<T>(dcoef, I.fdc);
  const unsigned long long amask = sm.amask[tid];
  sm.amask[tid] = 0ull;  // ready for the next work item
  struct P2Out {
    T K1, K3, dp, ax;
    bool act;
  };
  auto is_act = [&](const Slot& sl) {
    if (!MULTI || sl.kk < 64) return ((amask >> sl.kk) & 1ull) != 0ull;
    bool a_ = false;
    for (int a = 0; a < nu; ++a) a_ |= (sm.act[a] == g.lo + sl.q);
    return a_;
  };
  auto p2_store = [&](const Slot& sl, const Cells<NC>& cs, P2Out o) {
    if (resid_only) return;
    const int pb = wpos(sl.p);
    const T r = rcp_T(-T(1) - th * tdc * o.dp);
    const T v = -o.K1 * r;  // first sweep of F_x v5 = -K1 (v3 = 0)
    if (sl.v) {
      WV(pb, F_B2) = o.K3;
      WV(pb, F_AX) = o.ax;
      WV(pb, F_RG) = r;
      WV(pb, F_V1) = v;
    }
    if (wide) put(cs, sl, F_DP, o.dp);
    else if (sl.v) WV(pb, F_DP) = o.dp;
    put(cs, sl, F_P1, o.dp * v);
    if (o.act) {
      const int c = g.lo + sl.q;
      for (int a = 0; a < nu; ++a)
        if (sm.act[a] == c) sm.b1a[a] = o.K1;
    }
  };
  if (full) {
    pass<NC, 1, MULTI, P2Out>(g, c0,
        [&](const Slot& sl, const Cells<NC>&) {
          P2Out o{T(0), T(0), T(0), T(0), false};
          if (!sl.v) return o;
          const bool valid = true;
          const int c = g.lo + sl.q;
          o.act = is_act(sl);
          const double x = OX(sl), lam = OL(sl), xp = OXP(sl), rc_ = ORF(sl);
          const double ln = last ? I.hqf * (x - rc_) : OLN(sl);
          double srcd = 0.0;
          if (o.act) {
            for (int a = 0; a < nu; ++a)
              if (sm.act[a] == c) srcd += sm.u[a];
            srcd *= b0;
          }
          double lphi, mu;
          if (staged) {
            const int sb = spos(sl.p);
            lphi = cx * (SV(sb - SB, S_PH) + SV(sb + SB, S_PH)) +
                   cy * (SV(sb - WSB, S_PH) + SV(sb + WSB, S_PH)) - dcoef * SV(sb, S_PH);
            mu = cx * (SV(sb - SB, S_L) + SV(sb + SB, S_L)) +
                 cy * (SV(sb - WSB, S_L) + SV(sb + WSB, S_L)) - dcoef * lam;
          } else {
            const int iy = g.d2 ? c / I.mx : 0, ix = c - iy * I.mx;
            const double* Xs = X + so;
            const double* Ls = L + so;
            lphi = nbr_sum<double>(c, ix, iy, I.mx, I.my, cx, cy,
                                   [&](int m) { return phi_d(Xs[m], k0, k1); }) -
                   dcoef * phi_d(x, k0, k1);
            mu = nbr_sum<double>(c, ix, iy, I.mx, I.my, cx, cy, [&](int m) { return Ls[m]; }) -
                 dcoef * lam;
          }
          const double dphi = k0 * (1.0 + k1 * x);
          // explicit fused multiply-adds: the same rounding in every
          // instantiation (with and without the red-black branch)
          const double s1 = lphi + srcd;
          const double s3 = I.q * (x - rc_) + dphi * mu;
          const double K1 = __fma_rn(h, s1, xp - x);
          const double K3 = __fma_rn(h, s3, ln - lam);
          if (valid) {
            vmax = fmax(vmax, fmax(abs_or_inf(K1), abs_or_inf(K3)));
            vsq += K1 * K1 + K3 * K3;
          }
          double K1r = K1, K3r = K3;
          if (rbn) {
            K1r = __fma_rn(h, s1, OXPN(sl) - x);
            if (!last) K3r = __fma_rn(h, s3, OLNN(sl) - lam);
          }
          o.K1 = to_T<T>(K1r);
          o.K3 = to_T<T>(K3r);
          o.dp = to_T<T>(dphi);
          o.ax = to_T<T>(h * (I.q + k0 * k1 * mu) + (last ? I.hqf : 0.0));
          return o;
        },
        p2_store);
  } else {
    const float cxf = I.fcx, cyf = I.fcy, dcf = I.fdc, hf = I.fh;
    const float k0f_ = I.fk0, k1f_ = I.fk1, qf_ = I.fq, b0f = I.fb0;
    const float k01f = I.fk01, hqff = last ? I.fhqf : 0.0f;
    pass<NC, G2, MULTI, P2Out>(g, c0,
        [&](const Slot& sl, const Cells<NC>&) {
          P2Out o;
          const bool valid = sl.v;
          const int pb = wpos(sl.p);
          o.act = valid && is_act(sl);
          const float lphi = cxf * (WF(pb - RB, F_Y4) + WF(pb + RB, F_Y4)) +
                             cyf * (WF(pb - WRB, F_Y4) + WF(pb + WRB, F_Y4)) - dcf * WF(pb, F_Y4);
          const float mu = cxf * (WF(pb - RB, F_W1) + WF(pb + RB, F_W1)) +
                           cyf * (WF(pb - WRB, F_W1) + WF(pb + WRB, F_W1)) - dcf * WF(pb, F_W1);
          const float xv = WF(pb, F_Y5);
          const double x = OX(sl), lam = OL(sl), xp = OXP(sl), rc_ = ORF(sl);
          const float rv = d2f(rc_);
          float srcf = 0.0f;
          if (o.act) {
            const int c = g.lo + sl.q;
            for (int a = 0; a < nu; ++a)
              if (sm.act[a] == c) srcf += d2f(sm.u[a]);
          }
          const float dphi = k0f_ * (1.0f + k1f_ * xv);
          const float s1 = lphi + b0f * srcf;
          const float s3 = qf_ * (xv - rv) + dphi * mu;
          // the O(1) differences in float64; at the last stage lambda_{N+1} is
          // h qf (x_N - ref), an O(h) term (explicit fused multiply-adds, as
          // in the float64 form)
          const double d3 = last ? -lam : OLN(sl) - lam;
          const float dx = d2f(xp - x), dl = d2f(d3);
          const float K1 = __fmaf_rn(hf, s1, dx);
          const float K3 = __fmaf_rn(hf, s3, dl) + (last ? hqff * (xv - rv) : 0.0f);
          // slots past the slab contribute nothing (selects, no branch)
          const float K1v = valid ? K1 : 0.0f, K3v = valid ? K3 : 0.0f;
          mg.z = fmaxf(mg.z, valid ? fmaxf(fabsf(dx), fabsf(dl)) : 0.0f);
          mg.w = fmaxf(mg.w, valid ? fabsf(rv) : 0.0f);
          fmax_ = fmax_nan(fmax_, fmax_nan(fabsf(K1v), fabsf(K3v)));
          fsq += K1v * K1v + K3v * K3v;
          float K1r = K1, K3r = K3;
          if (rbn) {
            K1r = __fmaf_rn(hf, s1, d2f(OXPN(sl) - x));
            if (!last) K3r = __fmaf_rn(hf, s3, d2f(OLNN(sl) - lam));
          }
          o.K1 = (T)K1r;
          o.K3 = (T)K3r;
          o.dp = (T)dphi;
          o.ax = (T)(hf * (qf_ + k01f * mu) + hqff);
          return o;
        },
        p2_store);
  }
  for (int a = tid; a < nu; a += bd) {
    const double K2 = h * (I.r * sm.u[a] + b0 * sm.lact[a]);
    if (cl.rank == 0) {
      if (full) {
        vmax = fmax(vmax, abs_or_inf(K2));
        vsq += K2 * K2;
      } else {
        const float K2f = d2f(K2);
        fmax_ = fmax_nan(fmax_, fabsf(K2f));
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
    double e = 0.0;
    if (!full) {
      float usum = 0.0f;
      for (int a = 0; a < nu; ++a) usum += fabsf(d2f(sm.u[a]));
      e = split_bound(I, last, mags, usum);
    }
    // each CTA's own atomics, issued before the barrier (they do not block)
    publish_residual(A, slot, b, k, sm.red_out[0], sm.red_out[1], e, full);
  }
  cl.sync();
  if (resid_only) return;

  // ---- P3: lower layer in T ----
  const T tcx = pick<T>(cx, I.fcx), tcy = pick<T>(cy, I.fcy), tb0 = pick<T>(b0, I.fb0);
  const T auu = pick<T>(I.auu, I.fauu);
  int y5f = F_Y5, y4f = F_Y4;  // fields holding Y(v3) = (v5, v4)
  const int n_full = A.local_u ? 1 : A.n_u_it + 1;  // full-field Y applications
  struct V2 {
    T v, w;
  };
  for (int it = 0; it < n_full; ++it) {
    if (it > 0) {
      // c4 = F_u v3 - K1 changes only on actuator cells: refresh v1, p1 there
      for (int a = tid; a < nu; a += bd) {
        const int c = sm.act[a];
        const int q = c - g.lo;
        bool first = (q >= 0 && q < g.n);
        for (int a2 = 0; a2 < a && first; ++a2)
          if (sm.act[a2] == c) first = false;
        if (first) {
          T inj = T(0);
          for (int a2 = 0; a2 < nu; ++a2)
            if (sm.act[a2] == c) inj += sm.v3[a2];
          int p;
          owner_of(c, g, I.mx, p);
          const int pb = wpos(p);
          const T v = (th * tb0 * inj - sm.b1a[a]) * WV(pb, F_RG);
          WV(pb, F_V1) = v;
          // halo copies of p1 for a boundary-row actuator cell
          Cells<NC> one{};
          one.pu = (g.up && q < g.edge) ? 1u : 0u;
          one.pd = (g.dn && q >= g.n - g.edge) ? 1u : 0u;
          put(one, Slot{0, 0, q, p, true}, F_P1, WV(pb, F_DP) * v);
        }
      }
      cl.sync();
    }
    // F_x v5 = c4 by n_lo pointwise Jacobi sweeps from zero: sweep 1 is v1;
    // sweep s+1 = v1 - D^{-1} (offdiag F_x) sweep s, reading neighbours.  The
    // last sweep also forms sweep 1 of F_x^T v4 = -K3 - A_xx v5 (own cells).
    int cur = F_V1;
    if (n_lo == 1) {
      pass<NC, NC, MULTI, T>(g, c0,
          [&](const Slot& sl, const Cells<NC>&) {
            const int pb = wpos(sl.p);
            return (-WV(pb, F_B2) - WV(pb, F_AX) * WV(pb, F_V1)) * WV(pb, F_RG);
          },
          [&](const Slot& sl, const Cells<NC>& cs, T w) { put(cs, sl, F_W1, w); });
    } else {
      cur = F_Y5;
      const bool lastsw = (n_lo == 2);
      pass<NC, NC, MULTI, V2>(g, c0,
          [&](const Slot& sl, const Cells<NC>&) {
            const int pb = wpos(sl.p);
            const T off = th * (tcx * (WV(pb - RB, F_P1) + WV(pb + RB, F_P1)) +
                                tcy * (WV(pb - WRB, F_P1) + WV(pb + WRB, F_P1)));
            const T v = WV(pb, F_V1) - WV(pb, F_RG) * off;
            return V2{v, (-WV(pb, F_B2) - WV(pb, F_AX) * v) * WV(pb, F_RG)};
          },
          [&](const Slot& sl, const Cells<NC>& cs, V2 o) {
            if (wide) put(cs, sl, F_Y5, o.v);
            else if (sl.v) WV(wpos(sl.p), F_Y5) = o.v;
            if (lastsw) put(cs, sl, F_W1, o.w);
          });
      int nxt = F_E1;
      for (int sw = 2; sw < n_lo; ++sw) {
        cl.sync();
        const bool fin = (sw == n_lo - 1);
        const int cf = cur, nf = nxt;
        pass<NC, NC, MULTI, V2>(g, c0,
            [&](const Slot& sl, const Cells<NC>&) {
              const int pb = wpos(sl.p);
              const T off = th * (tcx * (WV(pb - RB, F_DP) * WV(pb - RB, cf) +
                                         WV(pb + RB, F_DP) * WV(pb + RB, cf)) +
                                  tcy * (WV(pb - WRB, F_DP) * WV(pb - WRB, cf) +
                                         WV(pb + WRB, F_DP) * WV(pb + WRB, cf)));
              const T v = WV(pb, F_V1) - WV(pb, F_RG) * off;
              return V2{v, (-WV(pb, F_B2) - WV(pb, F_AX) * v) * WV(pb, F_RG)};
            },
            [&](const Slot& sl, const Cells<NC>& cs, V2 o) {
              put(cs, sl, nf, o.v);
              if (fin) put(cs, sl, F_W1, o.w);
            });
        const int t = cur; cur = nxt; nxt = t;
      }
    }
    y5f = cur;
    cur = F_W1;
    if (n_lo >= 2) {
      cl.sync();
      cur = F_Y4;
      pass<NC, NC, MULTI, T>(g, c0,
          [&](const Slot& sl, const Cells<NC>&) {
            const int pb = wpos(sl.p);
            const T off = th * WV(pb, F_DP) *
                          (tcx * (WV(pb - RB, F_W1) + WV(pb + RB, F_W1)) +
                           tcy * (WV(pb - WRB, F_W1) + WV(pb + WRB, F_W1)));
            return WV(pb, F_W1) - WV(pb, F_RG) * off;
          },
          [&](const Slot& sl, const Cells<NC>& cs, T v) {
            if (wide) put(cs, sl, F_Y4, v);
            else if (sl.v) WV(wpos(sl.p), F_Y4) = v;
          });
      int nxt = (y5f == F_E1) ? F_E2 : F_E1;  // the spare that does not hold v5
      for (int sw = 2; sw < n_lo; ++sw) {
        cl.sync();
        const int cf = cur, nf = nxt;
        pass<NC, NC, MULTI, T>(g, c0,
            [&](const Slot& sl, const Cells<NC>&) {
              const int pb = wpos(sl.p);
              const T off = th * WV(pb, F_DP) *
                            (tcx * (WV(pb - RB, cf) + WV(pb + RB, cf)) +
                             tcy * (WV(pb - WRB, cf) + WV(pb + WRB, cf)));
              return WV(pb, F_W1) - WV(pb, F_RG) * off;
            },
            [&](const Slot& sl, const Cells<NC>& cs, T v) { put(cs, sl, nf, v); });
        const int t = cur; cur = nxt; nxt = t;
      }
    }
    y4f = cur;
    if (A.local_u || it < A.n_u_it) {
      cl.sync();  // Y(.) at the actuator cells is read across ranks below
      if (!A.local_u) {
        // A_uu v3 = K2 + F_u^T y_lambda (A_ux = 0); every rank keeps all of v3
        for (int a = tid; a < nu; a += bd)
          sm.v3[a] = (sm.b3[a] + th * tb0 * *at(sm.act[a], y4f)) / auu;
        __syncthreads();
      }
    }
  }
  if (A.local_u) {
    // Y(v3) = Y(0) + sum_b v3_b Z(e_b), Z(e_b) = P^{-1}(F_u e_b, 0): the fixed
    // sweeps are linear and Z(e_b) vanishes outside a box of half-width
    // R = 2 (n_lo - 1) around actuator b (each sweep reaches one cell further).
    // The u-iteration then needs Y(0) at the actuator cells and the boxes.
    for (int a = tid; a < nu; a += bd) sm.y4a[a] = *at(sm.act[a], y4f);
    const int R = A.box_r;
    const int mx = I.mx, my = I.my;
    const int Sx = 2 * R + 1, Sy = g.d2 ? 2 * R + 1 : 1, Ry = g.d2 ? R : 0;
    const int S2 = Sx * Sy;
    T* boxes = reinterpret_cast<T*>(B + wpos(A.slab_max));  // after the work records
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
        if (i > 0 && cell(j, i - 1, c)) sx += (with_dp ? *at(c, F_DP) : T(1)) * v[j * Sx + i - 1];
        if (i < Sx - 1 && cell(j, i + 1, c)) sx += (with_dp ? *at(c, F_DP) : T(1)) * v[j * Sx + i + 1];
        if (j > 0 && cell(j - 1, i, c)) sy += (with_dp ? *at(c, F_DP) : T(1)) * v[(j - 1) * Sx + i];
        if (j < Sy - 1 && cell(j + 1, i, c)) sy += (with_dp ? *at(c, F_DP) : T(1)) * v[(j + 1) * Sx + i];
        return tcx * sx + tcy * sy;
      };
      const T v1c = th * tb0 * *at(ca, F_RG);  // first F_x sweep: D^{-1} h b0 e_b
      for (int q = lane; q < S2; q += 32) t0[q] = (q == Ry * Sx + R) ? v1c : T(0);
      __syncwarp();
      T* cb = t0;
      T* nb = t1;
      for (int sw = 1; sw < n_lo; ++sw) {
        for (int q = lane; q < S2; q += 32) {
          const int j = q / Sx, i = q % Sx;
          int c;
          T v = T(0);
          if (cell(j, i, c))
            v = ((q == Ry * Sx + R) ? v1c : T(0)) - *at(c, F_RG) * th * boxnbr(cb, j, i, true);
          nb[q] = v;
        }
        __syncwarp();
        T* t = cb; cb = nb; nb = t;
      }
      for (int q = lane; q < S2; q += 32) z5[q] = cb[q];
      __syncwarp();
      // F_x^T sweeps with right-hand side -A_xx z5: w^1 stays in t0; the
      // n_lo - 1 later sweeps alternate between t1 and z4, the last one in z4
      for (int q = lane; q < S2; q += 32) {
        const int j = q / Sx, i = q % Sx;
        int c;
        t0[q] = cell(j, i, c) ? -*at(c, F_AX) * z5[q] * *at(c, F_RG) : T(0);
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
              v = t0[q] - *at(c, F_RG) * th * *at(c, F_DP) * boxnbr(src, j, i, false);
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
          const int cb2 = sm.act[bb];
          const int di = ixa - cb2 % mx + R, dj = iya - cb2 / mx + Ry;
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
      const int cb2 = sm.act[bb];
      const int gy = cb2 / mx + q / Sx - Ry, gx = cb2 % mx + q % Sx - R;
      if (gx < 0 || gx >= mx || gy < 0 || gy >= my) continue;
      const int c = gy * mx + gx;
      const int qc = c - g.lo;
      if (qc < 0 || qc >= g.n) continue;
      int p;
      owner_of(c, g, mx, p);
      const T* z5 = boxes + (size_t)bb * 4 * S2;
      atomicAdd(&WV(wpos(p), y5f), sm.v3[bb] * z5[q]);
      atomicAdd(&WV(wpos(p), y4f), sm.v3[bb] * z5[S2 + q]);
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
  const int f5 = y5f, f4 = y4f;
  pass<NC, NC, MULTI, D2>(g, c0,
      [&](const Slot& sl, const Cells<NC>&) {
        const int pb = wpos(sl.p);
        return D2{fma(alpha, to_double(WV(pb, f5)), OX(sl)), fma(alpha, to_double(WV(pb, f4)), OL(sl))};
      },
      [&](const Slot& sl, const Cells<NC>& cs, D2 o) {
        if (sl.v) {
          Xo[sl.q] = o.x;
          Lo[sl.q] = o.l;
        }
        if constexpr (SMEM) {
          if (keep) {
            // the next iteration's staged x, lambda: own record and the
            // neighbours' halo copies
            const int sb = spos(sl.p);
            if (sl.v) {
              SV(sb, S_X) = o.x;
              SV(sb, S_L) = o.l;
            }
            const unsigned rel = (unsigned)(sl.p * SB);
            push_if(sup_base + rel + S_X * 8, o.x, (cs.pu >> sl.k) & 1u);
            push_if(sup_base + rel + S_L * 8, o.l, (cs.pu >> sl.k) & 1u);
            push_if(sdn_base + rel + S_X * 8, o.x, (cs.pd >> sl.k) & 1u);
            push_if(sdn_base + rel + S_L * 8, o.l, (cs.pd >> sl.k) & 1u);
          }
        }
      });
  for (int a = tid; a < nu; a += bd) {
    const double un = sm.u[a] - alpha * (double)sm.v3[a];
    if (cl.rank == 0) Uo[I.u_off + (long long)s * nu + a] = un;
    if (keep) sm.u[a] = un;  // every rank computes the same value
  }
  cl.sync();
}

// One upper-layer iteration (MODE_SOLVE: iteration *iter_k + j of a running
// solve with its convergence bookkeeping, j the launch's index in its chunk
// (k_advance moves *iter_k on after each chunk); MODE_ONESHOT: one residual or
// iteration from the given buffers).  NC: cells per thread per pass round.  SMEM: the
// slab records live in shared memory (a compile-time fact, so every record
// access is a shared-memory access; one round of cells per thread) or in a
// global scratch slab per CTA (several rounds).
template <typename T, int NC, bool SMEM>
__global__ void __launch_bounds__(512) k_iterate(IterArgs A, int MODE, int j) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallShared<T>& sm = *reinterpret_cast<SmallShared<T>*>(smem_raw);
  char* B;
  int wk_off = 0, st_off = 0;
  bool staged = false;
  if constexpr (SMEM) {
    B = reinterpret_cast<char*>(smem_raw);
    st_off = (int)((sizeof(SmallShared<T>) + 15) & ~size_t(15));
    staged = (A.stage != 0);
    wk_off = st_off + (staged ? A.slab_max * NUM_SFIELDS * 8 : 0);
  } else {
    B = A.scratch + (long long)blockIdx.x * A.scratch_stride;
  }
  Cl cl;
  cl.C = A.csize;
  cl.rank = (A.csize > 1) ? (int)cg::this_cluster().block_rank() : 0;
  sm.amask[threadIdx.x] = 0ull;
  if (MODE == MODE_ONESHOT) __syncthreads();  // solve mode: the prologue's barrier
  // the next iteration's CTAs may start as soon as every CTA of this one has
  // (they hold their state loads behind pdl_wait until this launch is done)
  pdl_trigger();
  // *iter_k only changes between chunks of launches (k_advance), never while
  // an iteration launch of the chunk is in flight
  const int k = (MODE == MODE_SOLVE) ? *(volatile int*)A.iter_k + launch_iter(A, j) : 0;
  const int half = launch_half(A, j);
  const int n_clusters = gridDim.x / A.csize;
  pdl_wait();  // the previous iteration's state, residuals and control words

  const int w_begin = (A.rb && half) ? A.n_work_even : 0;
  const int w_end = A.rb ? (half ? A.n_work : A.n_work_even) : A.n_work;
  for (int w = w_begin + blockIdx.x / A.csize; w < w_end; w += n_clusters) {
    const int2 item = A.work[w];
    const int b = item.x, s = item.y;
    if (!stage_in_half(A, s, half)) continue;  // uniform across the cluster
    bool resid_only = false;
    bool full = true;
    if (MODE == MODE_ONESHOT) {
      resid_only = (A.resid_only != 0);
      full = resid_only || (A.full_all != 0);
    } else {
      if (threadIdx.x == 0) control_decision(A, b, s, k, cl, sm.skip, sm.full);
      __syncthreads();
      const bool sk = sm.skip != 0;
      full = sm.full != 0;
      __syncthreads();
      if (sk) continue;  // uniform across the cluster: every rank read the same slots
      resid_only = (k == A.max_iter);
    }
    process_item<T, NC, SMEM>(A, b, s, k, (MODE == MODE_SOLVE) ? (k & 1) : 0, full, resid_only, sm,
                              B, wk_off, st_off, staged, cl, false, false, A.rb && half == 1);
  }

}

// Default spin budget of one grid-barrier wait (SM clock cycles, about two
// seconds); IterArgs.grid_wait holds the handle's budget.
constexpr long long GRID_WAIT_CYCLES = 4000000000LL;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a persistent launch with n_clusters clusters: the
// cluster's CTAs meet (after publishing their global writes), rank 0 arrives
// on the counter, the last arrival decides whether to stop (no instance
// running) and opens the next generation; the others wait for it, for at most
// A.grid_wait cycles, and on timeout raise the error word.  Returns
// stop | error << 1 to every thread of the cluster.
template <typename T>
__device__ int grid_barrier(const IterArgs& A, int n_clusters, unsigned& gen, const Cl& cl,
                            SmallShared<T>& sm) {
  __syncthreads();
  if (threadIdx.x == 0) __threadfence();
  cl.sync();
  if (cl.rank == 0 && threadIdx.x == 0) {
    unsigned* gs = A.gsync;
    const unsigned target = gen + 1u;
    if (atomicAdd(&gs[0], 1u) == (unsigned)n_clusters - 1u) {
      gs[0] = 0u;
      if (atomicOr(A.n_active, 0) == 0) gs[2] = 1u;
      __threadfence();
      atomicExch(&gs[1], target);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_u32(&gs[1]) != target) {
        if (ld_acquire_u32(&gs[3]) != 0u) break;
        if (clock64() - t0 > A.grid_wait) {
          atomicExch(&gs[3], 1u);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    const int code = (int)(ld_acquire_u32(&gs[2]) | (ld_acquire_u32(&gs[3]) << 1));
    gen = target;
    if (cl.C == 1) sm.bar_code = code;
    else
      for (int r = 0; r < cl.C; ++r) *cl.map(&sm.bar_code, r) = code;
  }
  cl.sync();
  return sm.bar_code;
}

// Persistent solve: cluster w owns work item w for the whole launch (the
// host launches one cluster per item and only when all are resident at once)
// and runs iterations k = *iter_k .. max_iter, with a grid barrier between
// iterations, until no instance is running.  The item's staged inputs stay
// in shared memory between iterations (only x_{i-1} and lambda_{i+1} are
// reloaded), so the launch needs staged slabs.  A barrier wait that runs out
// ends the launch with gsync[3] set; the host then restarts the solve with
// one launch per iteration.
template <typename T, int NC>
__global__ void __launch_bounds__(512) k_solve(IterArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallShared<T>& sm = *reinterpret_cast<SmallShared<T>*>(smem_raw);
  char* B = reinterpret_cast<char*>(smem_raw);
  const int st_off = (int)((sizeof(SmallShared<T>) + 15) & ~size_t(15));
  const int wk_off = st_off + A.slab_max * NUM_SFIELDS * 8;
  Cl cl;
  cl.C = A.csize;
  cl.rank = (A.csize > 1) ? (int)cg::this_cluster().block_rank() : 0;
  sm.amask[threadIdx.x] = 0ull;
  const int n_clusters = gridDim.x / A.csize;
  const int2 item = A.work[blockIdx.x / A.csize];
  const int b = item.x, s = item.y;
  unsigned gen = 0u;
  if (cl.rank == 0 && threadIdx.x == 0) gen = ld_acquire_u32(&A.gsync[1]);
  bool resident = false;
  for (int k = *(volatile int*)A.iter_k; k <= A.max_iter; ++k) {
    if (threadIdx.x == 0) control_decision(A, b, s, k, cl, sm.skip, sm.full);
    __syncthreads();
    const bool sk = sm.skip != 0;
    const bool full = sm.full != 0;
    __syncthreads();
    if (!sk) {
      process_item<T, NC, true>(A, b, s, k, k & 1, full, k == A.max_iter, sm, B, wk_off, st_off,
                                true, cl, resident, true);
      resident = true;
    }
    if (grid_barrier(A, n_clusters, gen, cl, sm) != 0) break;
  }
}

// Condition of the solve loop's graph WHILE node: run another chunk of
// iteration launches while some instance is running and the next iteration
// is at most max_iter (the counter grows by the chunk length per pass, so the
// loop always ends).
__global__ void k_loop_cond(cudaGraphConditionalHandle c, const int* n_active, const int* iter_k,
                            int max_iter) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int act = *(volatile const int*)n_active;
    const int k = *(volatile const int*)iter_k;
    cudaGraphSetConditional(c, (act > 0 && k <= max_iter) ? 1u : 0u);
  }
}

// After a chunk of n iteration launches: the next chunk starts at iteration
// *iter_k + n.
__global__ void k_advance(int* iter_k, int n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *iter_k += n;
}

// Reset the per-instance control and write S^0 into buffer 0: the cold start
// (mode 0), nothing (mode 1: buffer 0 already holds S^0) or the current state
// shifted by one stage with the last stage repeated (mode 2; receding
// horizon, the paper's closed loop).  first_full: iteration 0 evaluates the
// float64 residual (warm starts that may already be converged).
// step: null, or the closed loop's device step counter (after the first step
// the start is always the shift, mode 2).
__global__ void k_init_control(IterArgs A, int mode, int first_full, const double* xc,
                               const double* uc, const double* lc, const int* step = nullptr) {
  const int b = blockIdx.y;
  if (b >= A.n_inst) return;
  if (step && *step != 0) mode = 2;
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
    A.f64_count[b] = 0;
    A.full0[b] = first_full;
    if (b == 0) {
      *A.n_active = A.n_inst;
      *A.iter_k = 0;
      A.gsync[0] = 0u;  // the barrier generation (gsync[1]) carries on
      A.gsync[2] = 0u;
      A.gsync[3] = 0u;
      A.gsync[4] = 0u;  // the persistent line launch's item counters
      A.gsync[5] = 0u;
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
// rec_step: null, or a device step counter t; u_rec then points at row t of
// a [steps][sum n_u] history (rec_stride = sum n_u).
__global__ void k_plant_substep(const InstDev* inst, int n_inst, const int* act,
                                const double* w_in, double* w_out, const double* u_cur,
                                double* u_rec, double dt_all, int n_sub,
                                const int* rec_step = nullptr, long long rec_stride = 0) {
  const int b = blockIdx.y;
  if (b >= n_inst) return;
  if (u_rec && rec_step) u_rec += (long long)*rec_step * rec_stride;
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

// A start iterate written to (xo, uo, lo): with x0 == nullptr the
// receding-horizon shift of (xc, uc, lc) (stage i takes stage i + 1, the last
// stage is repeated); otherwise the cold start x_i = x0, u = 0, lambda = 0.
__global__ void k_shift_state(const InstDev* inst, int n_inst, const double* xc, const double* uc,
                              const double* lc, double* xo, double* uo, double* lo,
                              const double* x0 = nullptr) {
  const int b = blockIdx.y;
  if (b >= n_inst) return;
  const InstDev I = inst[b];
  const long long n = (long long)I.N * I.ng;
  if (x0) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
      xo[I.s_off + e] = x0[I.g_off + (e % I.ng)];
      lo[I.s_off + e] = 0.0;
    }
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)I.N * I.nu;
         e += (long long)gridDim.x * blockDim.x)
      uo[I.u_off + e] = 0.0;
    return;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / I.ng;
    const long long src = (i + 1 < I.N) ? e + I.ng : e;
    xo[I.s_off + e] = xc[I.s_off + src];
    lo[I.s_off + e] = lc[I.s_off + src];
  }
  const long long nu_all = (long long)I.N * I.nu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nu_all;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / I.nu;
    uo[I.u_off + e] = uc[I.u_off + ((i + 1 < I.N) ? e + I.nu : e)];
  }
}

// Arithmetic of the per-stage rollout: float64, or float32 from truncated
// values (d2f) with exact widening of the result (f2d) for start guesses.
__device__ __forceinline__ double ro_ld(double v, double) { return v; }
__device__ __forceinline__ float ro_ld(double v, float) { return d2f(v); }
__device__ __forceinline__ double ro_st(double v) { return v; }
__device__ __forceinline__ double ro_st(float v) { return f2d(v); }

// Trajectory of a control guess, one stage per launch for every instance
// (instances with N <= i skip).  State, forward: x_i = x_{i-1} + h (Lap Phi
// (x_{i-1}) + b0 B u_i), x_{-1} = x0 (the model of eq. 6 stepped explicitly),
// stage i in arithmetic T over cells c = t, t + stride, ... (t the thread's
// index in the instance's grid).  Each thread looks up once which actuators
// sit on its cells (a bit per actuator, n_u <= 64) instead of scanning them
// per cell.
template <typename T>
__global__ void k_rollout_state(const InstDev* inst, int n_inst, const int* act, const double* x0,
                                const double* u, double* x, int i) {
  const int b = blockIdx.y;
  if (b >= n_inst) return;
  const InstDev& I = inst[b];
  if (i >= I.N) return;
  const double* src = (i == 0) ? x0 + I.g_off : x + I.s_off + (long long)(i - 1) * I.ng;
  double* dst = x + I.s_off + (long long)i * I.ng;
  const double* ui = u + I.u_off + (long long)i * I.nu;
  const int* ab = act + I.act_off;
  const int stride = gridDim.x * blockDim.x, t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nu = I.nu, mx = I.mx, my = I.my, ng = I.ng;
  unsigned long long own = 0ull;
  for (int a = 0; a < nu; ++a)
    if (ab[a] % stride == t) own |= 1ull << a;
  const T z = T(0);
  const T k0 = (T)I.k0, k1h = (T)(0.5 * I.k1), cx = (T)I.cx, cy = (T)I.cy, dc = (T)I.dcoef;
  const T h = (T)I.h, b0 = (T)I.b0;
  const float inv_mx = 1.0f / (float)mx;
  auto phi = [&](int m) {
    const T w = ro_ld(src[m], z);
    return k0 * (w + k1h * w * w);
  };
  for (int c = t; c < ng; c += stride) {
    const int iy = fdiv(c, mx, inv_mx), ix = c - iy * mx;
    T srcu = z;
    for (unsigned long long m = own; m; m &= m - 1) {
      const int a = __ffsll((long long)m) - 1;
      if (ab[a] == c) srcu += ro_ld(ui[a], z);
    }
    const T lphi = nbr_sum<T>(c, ix, iy, mx, my, cx, cy, phi) - dc * phi(c);
    dst[c] = ro_st(ro_ld(src[c], z) + h * (lphi + b0 * srcu));
  }
}

// Costate, backward from lambda_{N+1} = h qf (x_N - ref): the costate rows of
// eq. 9 with the coupling term taken at the later stage,
// lambda_i = lambda_{i+1} + h (q (x_i - ref) + Phi'(x_i) Lap lambda_{i+1}),
// in arithmetic T.
template <typename T>
__global__ void k_rollout_costate(const InstDev* inst, int n_inst, const double* ref,
                                  const double* x, double* lam, int i_from_end) {
  const int b = blockIdx.y;
  if (b >= n_inst) return;
  const InstDev& I = inst[b];
  const int i = I.N - 1 - i_from_end;
  if (i < 0) return;
  const double* xi = x + I.s_off + (long long)i * I.ng;
  const double* r = ref + I.g_off;
  const double* ln = lam + I.s_off + (long long)(i + 1) * I.ng;  // used for i < N - 1
  double* li = lam + I.s_off + (long long)i * I.ng;
  const bool last = (i == I.N - 1);
  const double* xN = x + I.s_off + (long long)(I.N - 1) * I.ng;
  const T z = T(0);
  const T hqf = (T)I.hqf, k0 = (T)I.k0, k1 = (T)I.k1, cx = (T)I.cx, cy = (T)I.cy;
  const T dc = (T)I.dcoef, h = (T)I.h, q = (T)I.q;
  const int mx = I.mx, my = I.my, ng = I.ng;
  const float inv_mx = 1.0f / (float)mx;
  auto next = [&](int m) {
    return last ? hqf * (ro_ld(xN[m], z) - ro_ld(r[m], z)) : ro_ld(ln[m], z);
  };
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ng; c += gridDim.x * blockDim.x) {
    const int iy = fdiv(c, mx, inv_mx), ix = c - iy * mx;
    const T nc = next(c);
    const T lap = nbr_sum<T>(c, ix, iy, mx, my, cx, cy, next) - dc * nc;
    const T xc = ro_ld(xi[c], z);
    const T dphi = k0 * (T(1) + k1 * xc);
    li[c] = ro_st(nc + h * (q * (xc - ro_ld(r[c], z)) + dphi * lap));
  }
}

// The same two recursions in one launch, in float32 arithmetic (a start
// guess needs no more): one CTA per instance walks the stages, a block
// barrier between stages.  The recursion variable (the previous stage's x,
// or the next stage's lambda) is kept in shared memory as float32 when two
// stages fit (smem_cells >= ng; else it is read back from the float64
// output).  Stores float64.
__global__ void __launch_bounds__(1024) k_rollout_fused(const InstDev* inst, int n_inst,
                                                         const int* act, const double* x0,
                                                         const double* ref, const double* u,
                                                         double* x, double* lam,
                                                         int smem_cells) {
  extern __shared__ float rbuf[];  // [2][smem_cells]
  const int b = blockIdx.x;
  if (b >= n_inst) return;
  const InstDev& I = inst[b];
  const int ng = I.ng, mx = I.mx, my = I.my, nu = I.nu;
  const bool on_chip = ng <= smem_cells;
  const float h = I.fh, cx = I.fcx, cy = I.fcy, dc = I.fdc, k0 = I.fk0, k1 = I.fk1, k1h = I.fk1h;
  const float b0 = I.fb0, q = I.fq, hqf = I.fhqf;
  const double* r = ref + I.g_off;
  const double* x0b = x0 + I.g_off;
  auto phi = [&](float f) { return k0 * (f + k1h * f * f); };
  int cur = 0;
  // forward: x_i = x_{i-1} + h (Lap Phi(x_{i-1}) + b0 B u_i)
  for (int i = 0; i < I.N; ++i) {
    const double* srcg = (i == 0) ? x0b : x + I.s_off + (long long)(i - 1) * ng;
    const float* srcs = rbuf + (cur ^ 1) * smem_cells;
    float* dsts = rbuf + cur * smem_cells;
    auto src = [&](int m) { return (on_chip && i > 0) ? srcs[m] : d2f(srcg[m]); };
    double* dst = x + I.s_off + (long long)i * ng;
    const double* ui = u + I.u_off + (long long)i * nu;
    for (int c = threadIdx.x; c < ng; c += blockDim.x) {
      const int iy = c / mx, ix = c - iy * mx;
      float srcu = 0.0f;
      for (int a = 0; a < nu; ++a)
        if (act[I.act_off + a] == c) srcu += d2f(ui[a]);
      const float sc = src(c);
      const float lphi = cx * ((ix > 0 ? phi(src(c - 1)) : 0.0f) + (ix + 1 < mx ? phi(src(c + 1)) : 0.0f)) +
                         cy * ((iy > 0 ? phi(src(c - mx)) : 0.0f) + (iy + 1 < my ? phi(src(c + mx)) : 0.0f)) -
                         dc * phi(sc);
      const float v = sc + h * (lphi + b0 * srcu);
      if (on_chip) dsts[c] = v;
      dst[c] = f2d(v);
    }
    __syncthreads();
    cur ^= 1;
  }
  // backward: lambda_{N+1} = h qf (x_N - ref), lambda_i = lambda_{i+1} +
  // h (q (x_i - ref) + Phi'(x_i) Lap lambda_{i+1})
  const double* xN = x + I.s_off + (long long)(I.N - 1) * ng;
  for (int i = I.N - 1; i >= 0; --i) {
    const bool lst = (i == I.N - 1);
    const double* xi = x + I.s_off + (long long)i * ng;
    const double* lng = lam + I.s_off + (long long)(i + 1) * ng;  // read for i < N - 1
    const float* lns = rbuf + (cur ^ 1) * smem_cells;
    float* lds = rbuf + cur * smem_cells;
    double* li = lam + I.s_off + (long long)i * ng;
    auto next = [&](int m) {
      return lst ? hqf * (d2f(xN[m]) - d2f(r[m])) : (on_chip ? lns[m] : d2f(lng[m]));
    };
    for (int c = threadIdx.x; c < ng; c += blockDim.x) {
      const int iy = c / mx, ix = c - iy * mx;
      const float lap = cx * ((ix > 0 ? next(c - 1) : 0.0f) + (ix + 1 < mx ? next(c + 1) : 0.0f)) +
                        cy * ((iy > 0 ? next(c - mx) : 0.0f) + (iy + 1 < my ? next(c + mx) : 0.0f)) -
                        dc * next(c);
      const float xv = d2f(xi[c]);
      const float v = next(c) + h * (q * (xv - d2f(r[c])) + k0 * (1.0f + k1 * xv) * lap);
      if (on_chip) lds[c] = v;
      li[c] = f2d(v);
    }
    __syncthreads();
    cur ^= 1;
  }
}

// Closed loop on the device (one graph): the step loop's WHILE condition,
// the per-step record of each instance's status, iterations and residual,
// and a plain copy (graph loop bodies hold kernels only).
__global__ void k_cl_start(int* step, int steps, cudaGraphConditionalHandle outer) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *step = 0;
    cudaGraphSetConditional(outer, steps > 0 ? 1u : 0u);
  }
}

__global__ void k_cl_next(int* step, int steps, cudaGraphConditionalHandle outer) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int t = *step + 1;
    *step = t;
    cudaGraphSetConditional(outer, t < steps ? 1u : 0u);
  }
}

__global__ void k_cl_record(const int* step, int n_inst, const int* status, const int* iters,
                            const double* fin_inf, int* st_hist, int* it_hist, double* res_hist) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_inst) return;
  const long long o = (long long)*step * n_inst + b;
  st_hist[o] = status[b];
  it_hist[o] = iters[b];
  res_hist[o] = fin_inf[b];
}

__global__ void k_copy_f64(double* dst, const double* src, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// weights override: (q, r, qf) per instance from a device array
__global__ void k_set_weights(InstDev* inst, int n_inst, const double* w) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_inst) return;
  inst[b].q = w[3 * b + 0];
  inst[b].r = w[3 * b + 1];
  inst[b].qf = w[3 * b + 2];
  derive(inst[b]);
}

#include "nmpc_patch.cuh"
#include "nmpc_line.cuh"

}  // namespace nmpc_dev
