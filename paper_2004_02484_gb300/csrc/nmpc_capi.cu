// Host side of the C ABI declared in include/nmpc.h: descriptor validation,
// device instance table, workspace ownership, launch configuration, the
// graph-replayed iteration loop and the result gathering.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <cstdint>
#include <vector>

#include "../../include/nmpc.h"
#include "nmpc_kernels.cuh"

using nmpc_dev::InstDev;
using nmpc_dev::IterArgs;
using nmpc_dev::FinalArgs;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct nmpc_handle {
  int n_inst = 0;
  nmpc_opts opts{};
  int device = 0;
  int num_sms = 0;
  std::vector<InstDev> inst_h;
  long long n_g = 0, n_s = 0, n_u = 0;  // packed sizes: sum ng, sum N*ng, sum N*nu
  int ng_max = 0, nu_max = 0, n_work = 0, n_max_horizon = 0;
  long long nu_tot = 0;  // sum of n_u (first-stage control vector length)
  // device data
  InstDev* inst_d = nullptr;
  int2* work_d = nullptr;
  int* act_d = nullptr;
  double* x0_d = nullptr;
  double* ref_d = nullptr;
  float* ref_f_d = nullptr;  // ref truncated to float32 (two-column strip path)
  double* uo_d = nullptr;  // staging for the host-pointer solve
  double* w_d = nullptr;   // staging for host weights
  double* xb[3] = {nullptr, nullptr, nullptr};  // A, B, current
  double* ub[3] = {nullptr, nullptr, nullptr};
  double* lb[3] = {nullptr, nullptr, nullptr};
  // control
  int* ictl = nullptr;  // iter_k, closed-loop step, n_active, running line items, grid barrier
                        // and item counters [4..9], running count for the strip plan [10]
                        // words [4], the persistent line launch's item counters [2]
  unsigned long long* res_inf = nullptr;
  unsigned long long* res_err = nullptr;
  double* res_sq = nullptr;
  unsigned long long* res_first = nullptr;
  int* status = nullptr;
  int* iters = nullptr;
  int* final_buf = nullptr;
  double* fin_inf = nullptr;
  double* fin_2 = nullptr;
  int* f64_count = nullptr;
  int* full0 = nullptr;
  char* scratch = nullptr;
  long long scratch_stride = 0;
  // pinned host mirrors
  int* h_active = nullptr;
  int* h_status = nullptr;
  int* h_iters = nullptr;
  int* h_f64 = nullptr;     // float64-residual iterations per instance
  double* h_fin = nullptr;  // [2][n]
  double* h_res = nullptr;  // [2][n] for residual readback
  unsigned long long* h_resinf = nullptr;
  // launch configuration
  int threads = 0;
  int cpt = 4;
  bool persistent = false;
  int resident_clusters = 0;
  int grid = 0;
  int csize = 1;
  int slab_max = 0;
  size_t smem = 0;
  bool smem_mode = true;
  bool stage = true;
  bool local_u = false;
  int box_r = 0;
  size_t box_bytes = 0;
  bool mixed = false;
  bool rb = false;  // red-black upper layer (two half-sweep launches per iteration)
  int n_work_even = 0, n_strips_even = 0, n_patches_even = 0;  // red-black: even-stage items first
  size_t strip_smem_rb = 0;  // k_strip's shared memory in red-black half 1
  // graph of one chunk of iterations
  cudaGraphExec_t graph_exec = nullptr;
  int graph_chunk = 0;
  // the whole iteration loop as one graph: a WHILE node over chunks
  cudaGraphExec_t loop_exec = nullptr;
  int loop_chunk = 0;
  // strip path (k_patch + k_strip)
  int4* strips_d = nullptr;
  int n_strips = 0;
  int strip_x = 0, strip_y = 0, strip_threads = 0, strip_region = 0;
  int n_strip_inst = 0;
  bool strip2 = false;  // two grid columns per lane (k_strip2)
  // the tail plan of k_strip2: strips of tail_y own rows for the launches
  // that run with at most tail_below instances still running
  int4* tail_d = nullptr;
  int n_tail = 0, n_tail_even = 0, tail_y = 0, tail_below = 0;
  size_t strip_smem = 0;
  int4* patches_d = nullptr;  // k_patch work items
  int n_patches = 0;
  size_t patch_smem = 0;
  double* v3_d = nullptr;  // v3 per control, written by k_patch
  // line path (k_line): one warp per 1D stage
  int4* lines_d = nullptr;
  int4* lines_act_d = nullptr;  // items of running instances (solve mode)
  int n_lines = 0;
  int line_grid = 0;  // CTAs of a k_line launch
  bool line_persistent = false;  // one k_line_solve launch runs the whole solve
  int line_solve_grid = 0;       // its CTAs (all resident at once)
  int n_line_inst = 0;
  size_t line_smem = 0;
  long long launches = 0;
  // per-kernel CUDA-event timing (nmpc_kernel_timing): event pairs around
  // launches that are not being captured, summed per kernel kind
  bool timing = false;
  std::vector<cudaEvent_t> ev_free;
  struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<TimedLaunch> ev_pending;
  double kt_ms[4] = {0, 0, 0, 0};
  long long kt_n[4] = {0, 0, 0, 0};
  long long iter_launches = 0;  // iteration steps (each one or two kernel launches)
  bool has_state = false;
};

namespace {

// Lower limit of the residual level at which handles with strip-path
// instances switch to the float64 residual (see make_args).
constexpr double STRIP_SPLIT_FLOOR = 1e-6;

template <typename T>
size_t small_shared_bytes() {
  return (sizeof(nmpc_dev::SmallShared<T>) + 15) & ~size_t(15);
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      fprintf(stderr, "nmpc: %s failed: %s (%s:%d)\n", #call,      \
              cudaGetErrorString(e_), __FILE__, __LINE__);         \
      return NMPC_ERR_CUDA;                                        \
    }                                                              \
  } while (0)

template <typename P>
cudaError_t dev_alloc(P** p, size_t count) {
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(P));
}

// ref into the handle's buffer, and its float32 copy where the two-column
// strip path reads one.
cudaError_t load_ref(nmpc_handle* h, const double* ref, cudaMemcpyKind kind, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(h->ref_d, ref, h->n_g * sizeof(double), kind, st);
  if (e != cudaSuccess || !h->ref_f_d) return e;
  nmpc_dev::k_f32_copy<<<(unsigned)std::min<long long>(1024, (h->n_g + 255) / 256), 256, 0, st>>>(
      h->ref_d, h->ref_f_d, h->n_g);
  h->launches++;
  return cudaGetLastError();
}

void free_all(nmpc_handle* h) {
  if (!h) return;
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
  void* ptrs[] = {h->inst_d, h->work_d, h->act_d, h->x0_d, h->ref_d, h->ref_f_d, h->uo_d, h->w_d,
                  h->xb[0], h->xb[1], h->xb[2], h->ub[0], h->ub[1], h->ub[2],
                  h->lb[0], h->lb[1], h->lb[2], h->ictl, h->res_inf, h->res_err, h->res_sq,
                  h->res_first, h->status, h->iters, h->final_buf, h->fin_inf,
                  h->fin_2, h->f64_count, h->full0, h->scratch, h->strips_d, h->tail_d, h->patches_d, h->lines_d, h->lines_act_d,
                  h->v3_d};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  void* hp[] = {h->h_active, h->h_status, h->h_iters, h->h_f64, h->h_fin, h->h_res, h->h_resinf};
  for (void* p : hp)
    if (p) cudaFreeHost(p);
}

IterArgs make_args(nmpc_handle* h) {
  IterArgs A{};
  A.inst = h->inst_d;
  A.work = h->work_d;
  A.n_work = h->n_work;
  A.n_inst = h->n_inst;
  A.act = h->act_d;
  A.x0 = h->x0_d;
  A.ref = h->ref_d;
  A.ref_f = h->ref_f_d;
  for (int q = 0; q < 2; ++q) {
    A.xin[q] = h->xb[q];
    A.uin[q] = h->ub[q];
    A.lin[q] = h->lb[q];
    A.xout[q] = h->xb[q];
    A.uout[q] = h->ub[q];
    A.lout[q] = h->lb[q];
  }
  A.iter_k = h->ictl + 0;
  A.n_active = h->ictl + 2;
  A.gsync = reinterpret_cast<unsigned*>(h->ictl + 4);
  A.res_inf = h->res_inf;
  A.res_err = h->res_err;
  A.res_sq = h->res_sq;
  A.res_first = h->res_first;
  A.status = h->status;
  A.iters = h->iters;
  A.final_buf = h->final_buf;
  A.fin_inf = h->fin_inf;
  A.fin_2 = h->fin_2;
  A.tol = h->opts.tol;
  A.div_limit = h->opts.div_limit;
  A.alpha = h->opts.alpha;
  // the strip path's split residual takes the O(1) stage differences from
  // float32-truncated values: they move in steps of 2^-23 |x|, so its
  // iteration cannot settle far below ~1e-6; such handles switch to the
  // float64 residual by then at the latest
  A.split_min = (h->n_strips > 0) ? std::max(h->opts.split_min, STRIP_SPLIT_FLOOR)
                                  : h->opts.split_min;
  A.max_iter = h->opts.max_iter;
  A.n_lo = h->opts.n_lo;
  A.n_u_it = h->opts.n_u_it;
  A.rb = h->rb ? 1 : 0;
  A.n_work_even = h->n_work_even;
  A.n_strips_even = h->n_strips_even;
  A.n_patches_even = h->n_patches_even;
  A.grid_wait = h->opts.barrier_wait_cycles > 0 ? (long long)h->opts.barrier_wait_cycles
                                                : nmpc_dev::GRID_WAIT_CYCLES;
  A.resid_only = 0;
  A.f64_count = h->f64_count;
  A.full0 = h->full0;
  A.full_all = h->mixed ? 0 : 1;
  A.csize = h->csize;
  A.slab_max = h->slab_max;
  A.stage = h->stage ? 1 : 0;
  A.local_u = h->local_u ? 1 : 0;
  A.box_r = h->box_r;
  A.scratch = h->smem_mode ? nullptr : h->scratch;
  A.scratch_stride = h->scratch_stride;
  A.strips = h->strips_d;
  A.n_strips = h->n_strips;
  A.strip_x = h->strip_x;
  A.strip_y = h->strip_y;
  A.tail = h->tail_d;
  A.n_tail = h->n_tail;
  A.n_tail_even = h->n_tail_even;
  A.tail_y = h->tail_y;
  A.tail_below = h->tail_below;
  A.strip_run = h->ictl + 10;
  A.patches = h->patches_d;
  A.n_patches = h->n_patches;
  A.v3g = h->v3_d;
  A.lines = h->lines_d;
  A.n_lines = h->n_lines;
  A.lines_act = h->lines_act_d;
  A.n_lines_act = h->ictl + 3;
  return A;
}

// Launch shape of the iteration kernel: CTAs per stage (cluster size), slab
// length, threads, dynamic shared memory, grid.
struct LaunchPlan {
  int threads = 0, csize = 1, slab_max = 0, grid = 0;
  int cpt = 4;  // cells per thread (kernel variant)
  bool persistent = false;  // one launch runs the whole solve (k_solve)
  int resident_clusters = 0;  // clusters resident at once for k_solve
  size_t smem = 0;
  bool smem_mode = true;
  bool stage = true;  // float64 slab inputs staged in shared memory
  bool local_u = false;  // u-iteration through the actuators' local responses
  int box_r = 0;
  size_t box_bytes = 0;
};

// Interior cells of the largest rank slab of a stage split over C CTAs.
int slab_cells(const InstDev& I, int C) {
  const int unit = (I.dim == 2) ? I.mx : 1;
  const int nun = (I.dim == 2) ? I.my : I.mx;
  return ((nun + C - 1) / C) * unit;
}

// Records of a padded rank slab: (rows + 2) (mx + 2) in 2D, cells + 2 in 1D
// (halo rows or cells and zero pads around the slab), even.
int slab_stride(const InstDev& I, int C) {
  const int nun = (I.dim == 2) ? I.my : I.mx;
  const int per = (nun + C - 1) / C;
  const int len = (I.dim == 2) ? (per + 2) * (I.mx + 2) : per + 2;
  return (len + 1) & ~1;
}

// Largest cells per thread of the shared-memory kernels, and of a CTA.
constexpr int MAX_NC = 8;
constexpr int MAX_THREADS = 512;
// Cells per thread of the global-slab kernel per round.
constexpr int GLOBAL_NC = 4;

template <typename T>
size_t small_shared_bytes_t() {
  return (sizeof(nmpc_dev::SmallShared<T>) + 15) & ~size_t(15);
}

using IterKernel = void (*)(IterArgs, int, int);

// Kernel variants: NC cells per thread (1, 2, 4, 8) with the slab in shared
// memory, or the global-slab kernel.
template <typename T>
IterKernel iter_kernel(int nc, bool smem) {
  if (!smem) return nmpc_dev::k_iterate<T, GLOBAL_NC, false>;
  switch (nc) {
    case 1: return nmpc_dev::k_iterate<T, 1, true>;
    case 2: return nmpc_dev::k_iterate<T, 2, true>;
    case 4: return nmpc_dev::k_iterate<T, 4, true>;
    default: return nmpc_dev::k_iterate<T, 8, true>;
  }
}

IterKernel iter_kernel_of(bool mixed, int nc, bool smem) {
  return mixed ? iter_kernel<float>(nc, smem) : iter_kernel<double>(nc, smem);
}

using SolveKernel = void (*)(IterArgs);

template <typename T>
SolveKernel solve_kernel(int nc) {
  switch (nc) {
    case 1: return nmpc_dev::k_solve<T, 1>;
    case 2: return nmpc_dev::k_solve<T, 2>;
    case 4: return nmpc_dev::k_solve<T, 4>;
    default: return nmpc_dev::k_solve<T, 8>;
  }
}

SolveKernel solve_kernel_of(bool mixed, int nc) {
  return mixed ? solve_kernel<float>(nc) : solve_kernel<double>(nc);
}

// Threads per CTA and cells per thread for a shared-memory slab of `slab`
// interior cells: opts.cells (default 4) cells per thread, at least 128
// threads, at most 512; the kernel variant's cells per thread is the power of
// two that covers the slab.  Returns false if no variant covers it.
bool thread_shape(int slab, const nmpc_opts& o, int* threads, int* nc) {
  const int target = o.cells ? o.cells : 4;
  int t = o.threads;
  if (!t) {
    t = ((slab + target - 1) / target + 31) / 32 * 32;
    t = std::min(MAX_THREADS, std::max(128, t));
    while ((long long)MAX_NC * t < slab && t < MAX_THREADS) t += 32;
  }
  int c = 1;
  while ((long long)c * t < slab && c < MAX_NC) c *= 2;
  *threads = t;
  *nc = c;
  return (long long)c * t >= slab;
}

// Clusters of C CTAs (`threads` threads, `smem` bytes) the device keeps
// resident at once for the iteration kernel (or, with `solve`, the
// persistent kernel).
int clusters_resident(int C, int threads, int nc, size_t smem, bool mixed, bool solve = false) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * 256));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  const void* fn = solve ? (const void*)solve_kernel_of(mixed, nc)
                         : (const void*)iter_kernel_of(mixed, nc, true);
  cudaError_t e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Cluster size: the smallest that fits a stage slab (with the float64 inputs
// staged in shared memory if possible) in shared memory and in the threads
// of a CTA (at most MAX_NC cells each), then grown up to 8 while every
// cluster of the batch stays resident in one wave; cluster sizes above 8 are
// 16 only.  A stage that does not fit even at 16 runs one CTA per stage on a
// global slab.
LaunchPlan plan_launch(const InstDev* insts, int n_inst, int n_work, const nmpc_opts& o,
                       bool mixed, int num_sms, int max_optin) {
  LaunchPlan P;
  const size_t elem = mixed ? sizeof(float) : sizeof(double);
  const size_t small = mixed ? small_shared_bytes_t<float>() : small_shared_bytes_t<double>();
  // local-response boxes: 4 arrays of (2R+1)^dim cells per actuator, R = 2 (n_lo - 1)
  int nu_max = 0, dim_max = 1;
  for (int b = 0; b < n_inst; ++b) {
    nu_max = std::max(nu_max, insts[b].nu);
    dim_max = std::max(dim_max, insts[b].dim);
  }
  P.box_r = 2 * (o.n_lo - 1);
  const size_t side = (size_t)(2 * P.box_r + 1);
  const size_t box_bytes = (size_t)nu_max * 4 * (dim_max == 2 ? side * side : side) * elem;
  P.local_u = o.u_local && (o.n_lo <= 4) && box_bytes <= 32768;
  P.box_bytes = P.local_u ? ((box_bytes + 15) & ~size_t(15)) : 0;
  auto slab = [&](int C) {  // interior cells
    int m = 0;
    for (int b = 0; b < n_inst; ++b) m = std::max(m, slab_cells(insts[b], C));
    return m;
  };
  auto stride = [&](int C) {  // records per slab
    int m = 0;
    for (int b = 0; b < n_inst; ++b) m = std::max(m, slab_stride(insts[b], C));
    return m;
  };
  bool stage = true;
  auto bytes = [&](int C) {
    return small + P.box_bytes +
           (size_t)stride(C) * (nmpc_dev::NUM_FIELDS * elem +
                                (stage ? nmpc_dev::NUM_SFIELDS * sizeof(double) : 0));
  };
  auto next_c = [](int C) { return C < 8 ? C + 1 : 16; };
  auto fits = [&](int C) {
    int t, c;
    return bytes(C) <= (size_t)max_optin && thread_shape(slab(C), o, &t, &c);
  };
  int C = 1;
  if (o.cluster > 0) {
    C = o.cluster;
    if (!fits(C)) stage = false;
  } else {
    // the smallest cluster that fits with staging, else without staging
    while (C < 16 && !fits(C)) C = next_c(C);
    if (!fits(C)) {
      stage = false;
      C = 1;
      while (C < 16 && !fits(C)) C = next_c(C);
    }
    if (fits(C)) {
      // grow while every cluster of the batch is still resident in one wave
      // (clusters are packed per GPC, so this is a cluster-occupancy query,
      // not a CTA count) and slabs keep at least 512 cells
      while (C < 8) {
        const int C2 = C + 1;
        if (!fits(C2) || slab(C2) < 512) break;
        int t2, c2;
        thread_shape(slab(C2), o, &t2, &c2);
        if (clusters_resident(C2, t2, c2, bytes(C2), mixed) < n_work) break;
        C = C2;
      }
    }
  }
  P.smem_mode = fits(C);
  if (!P.smem_mode) {
    C = 1;
    stage = false;
  }
  P.stage = stage;
  P.csize = C;
  P.slab_max = stride(C);
  if (P.smem_mode) {
    thread_shape(slab(C), o, &P.threads, &P.cpt);
  } else {
    P.threads = o.threads ? o.threads : MAX_THREADS;
    P.cpt = GLOBAL_NC;
  }
  P.smem = P.smem_mode ? bytes(C) : small;
  P.grid = n_work * C;
  // one cluster per work item for the whole solve, if all fit at once
  P.resident_clusters =
      P.smem_mode ? clusters_resident(C, P.threads, P.cpt, P.smem, mixed, true) : 0;
  P.persistent = o.persistent && o.variant == 0 && P.smem_mode && P.stage &&
                 P.resident_clusters >= n_work;
  return P;
}

template <typename T>
cudaError_t launch_k(const LaunchPlan& P, const IterArgs& A, cudaStream_t st, int mode, int j) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)P.grid);
  cfg.blockDim = dim3((unsigned)P.threads);
  cfg.dynamicSmemBytes = P.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)P.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // consecutive iteration launches overlap their start with the previous
  // launch's end (programmatic dependent launch; the kernel waits for the
  // previous iteration before it reads any state)
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (mode == nmpc_dev::MODE_SOLVE) ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, iter_kernel<T>(P.cpt, P.smem_mode), A, mode, j);
}

// The persistent solve launch: one cluster per work item, launched as a
// cooperative launch where the runtime accepts one with clusters (co-resident
// by construction), else as a plain cluster launch (the host has checked that
// all clusters fit at once; the kernel's waits are bounded either way).
template <typename T>
cudaError_t launch_solve(const LaunchPlan& P, const IterArgs& A, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)P.grid);
  cfg.blockDim = dim3((unsigned)P.threads);
  cfg.dynamicSmemBytes = P.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)P.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaError_t e = cudaLaunchKernelEx(&cfg, solve_kernel<T>(P.cpt), A);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, solve_kernel<T>(P.cpt), A);
  }
  return e;
}

LaunchPlan plan_of(const nmpc_handle* h) {
  LaunchPlan P;
  P.threads = h->threads;
  P.cpt = h->cpt;
  P.persistent = h->persistent;
  P.csize = h->csize;
  P.stage = h->stage;
  P.local_u = h->local_u;
  P.box_r = h->box_r;
  P.box_bytes = h->box_bytes;
  P.slab_max = h->slab_max;
  P.grid = h->grid;
  P.smem = h->smem;
  P.smem_mode = h->smem_mode;
  return P;
}

// Strip kernel variants, one per n_lo = 1 .. 4.
using TileKernel = void (*)(IterArgs, int, int);

template <typename T>
TileKernel strip_kernel(int n_lo, bool rbn = false, bool two = false) {
  if (two) {  // float32 lower layer, n_lo <= 2 (checked at setup)
    if (n_lo <= 1) return rbn ? nmpc_dev::k_strip2<1, true> : nmpc_dev::k_strip2<1, false>;
    return rbn ? nmpc_dev::k_strip2<2, true> : nmpc_dev::k_strip2<2, false>;
  }
  if (rbn) {
    switch (n_lo) {
      case 1: return nmpc_dev::k_strip<T, 1, true>;
      case 2: return nmpc_dev::k_strip<T, 2, true>;
      case 3: return nmpc_dev::k_strip<T, 3, true>;
      default: return nmpc_dev::k_strip<T, 4, true>;
    }
  }
  switch (n_lo) {
    case 1: return nmpc_dev::k_strip<T, 1, false>;
    case 2: return nmpc_dev::k_strip<T, 2, false>;
    case 3: return nmpc_dev::k_strip<T, 3, false>;
    default: return nmpc_dev::k_strip<T, 4, false>;
  }
}

// Whether launch j of an iteration is red-black half 1.
inline bool rb_half1(const IterArgs& A, int j) { return A.rb && (j & 1); }

// Items of a list of n (n_even of them at even stages, first) that launch j
// covers: all of them, or one half-sweep's share.
inline int half_count(const IterArgs& A, int j, int n, int n_even) {
  if (!A.rb) return n;
  return (j & 1) ? n - n_even : n_even;
}

template <typename T>
TileKernel patch_kernel(int n_lo) {
  switch (n_lo) {
    case 1: return nmpc_dev::k_patch<T, 1>;
    case 2: return nmpc_dev::k_patch<T, 2>;
    case 3: return nmpc_dev::k_patch<T, 3>;
    default: return nmpc_dev::k_patch<T, 4>;
  }
}

constexpr int PATCH_WARPS = 4;  // warps per k_patch block


template <typename T>
cudaError_t launch_patch(const nmpc_handle* h, const IterArgs& A, cudaStream_t st, int mode, int j) {
  int count = half_count(A, j, h->n_patches, h->n_patches_even);
  // with a tail plan every solve-mode strip launch follows a k_patch launch,
  // which records the running-instance count for it
  if (h->n_tail > 0 && mode == nmpc_dev::MODE_SOLVE) count = std::max(count, 1);
  if (count == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((count + PATCH_WARPS - 1) / PATCH_WARPS));
  cfg.blockDim = dim3(32 * PATCH_WARPS);
  cfg.dynamicSmemBytes = h->patch_smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (mode == nmpc_dev::MODE_SOLVE) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, patch_kernel<T>(h->opts.n_lo), A, mode, j);
}

template <typename T>
cudaError_t launch_strip(const nmpc_handle* h, const IterArgs& A, cudaStream_t st, int mode, int j) {
  int count = half_count(A, j, h->n_strips, h->n_strips_even);
  // solve launches cover either plan (warps past the chosen plan's items return)
  if (h->n_tail > 0 && mode == nmpc_dev::MODE_SOLVE)
    count = std::max(count, half_count(A, j, h->n_tail, h->n_tail_even));
  if (count == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  const int warps = h->strip2 ? nmpc_dev::STRIP2_WARPS : nmpc_dev::STRIP_WARPS;
  cfg.gridDim = dim3((unsigned)((count + warps - 1) / warps));
  cfg.blockDim = dim3((unsigned)h->strip_threads);
  cfg.dynamicSmemBytes = rb_half1(A, j) ? h->strip_smem_rb : h->strip_smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (mode == nmpc_dev::MODE_SOLVE) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, strip_kernel<T>(h->opts.n_lo, rb_half1(A, j), h->strip2), A,
                            mode, j);
}

cudaError_t launch_line(const nmpc_handle* h, const IterArgs& A, cudaStream_t st, int mode, int j) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)h->line_grid);
  cfg.blockDim = dim3(32 * nmpc_dev::LINE_WARPS);
  cfg.dynamicSmemBytes = h->line_smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (mode == nmpc_dev::MODE_SOLVE) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, rb_half1(A, j) ? nmpc_dev::k_line<true> : nmpc_dev::k_line<false>,
                            A, mode, j);
}

// Kernel kinds of nmpc_kernel_times.
enum { KT_CLUSTER = 0, KT_PATCH = 1, KT_STRIP = 2, KT_LINE = 3 };

// Sum the elapsed times of the recorded launches into the per-kind totals and
// recycle their events (waits for the last one).
cudaError_t harvest_timing(nmpc_handle* h) {
  if (h->ev_pending.empty()) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(h->ev_pending.back().b);
  for (auto& t : h->ev_pending) {
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
    h->kt_ms[t.kind] += ms;
    h->kt_n[t.kind] += 1;
    h->ev_free.push_back(t.a);
    h->ev_free.push_back(t.b);
  }
  h->ev_pending.clear();
  return e;
}

cudaError_t take_event(nmpc_handle* h, cudaEvent_t* ev) {
  if (h->ev_free.empty()) return cudaEventCreate(ev);
  *ev = h->ev_free.back();
  h->ev_free.pop_back();
  return cudaSuccess;
}

// launch() bracketed by a CUDA event pair on st when the handle times kernels
// and st is not capturing a graph (events in a capture would become graph
// dependencies, not timestamps).
template <typename F>
cudaError_t timed(nmpc_handle* h, int kind, cudaStream_t st, F launch) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!h->timing || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone)
    return launch();
  if (h->ev_pending.size() >= 4096) {
    cudaError_t e = harvest_timing(h);
    if (e != cudaSuccess) return e;
  }
  cudaEvent_t a, b;
  cudaError_t e = take_event(h, &a);
  if (e == cudaSuccess) e = take_event(h, &b);
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e != cudaSuccess) return e;
  e = launch();
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(b, st);
  if (e == cudaSuccess) h->ev_pending.push_back({kind, a, b});
  return e;
}

// One iteration (or one-shot pass): the cluster kernel over the cluster
// path's work items, the strip kernels over the strips and the line kernel
// over the 1D stages, whichever exist.
template <int MODE>
cudaError_t launch_iterate(nmpc_handle* h, const IterArgs& A, cudaStream_t st, int j = 0) {
  if (!rb_half1(A, j)) h->iter_launches++;  // one iteration step per Jacobi launch or half pair
  cudaError_t e = cudaSuccess;
  const int n_cl = half_count(A, j, h->n_work, h->n_work_even);
  if (n_cl > 0) {
    h->launches++;
    LaunchPlan P = plan_of(h);
    // a red-black half launches the clusters of its own items only (a
    // global-slab launch keeps at most the CTAs it has slabs for)
    if (A.rb) P.grid = P.smem_mode ? n_cl * P.csize : std::min(P.grid, n_cl);
    e = timed(h, KT_CLUSTER, st, [&]() {
      return h->mixed ? launch_k<float>(P, A, st, MODE, j) : launch_k<double>(P, A, st, MODE, j);
    });
    if (e != cudaSuccess) return e;
  }
  if (h->n_strips > 0) {
    // the actuators' v3 first (not needed by a residual-only pass)
    if (!(MODE == nmpc_dev::MODE_ONESHOT && A.resid_only)) {
      h->launches++;
      e = timed(h, KT_PATCH, st, [&]() {
        return h->mixed ? launch_patch<float>(h, A, st, MODE, j)
                        : launch_patch<double>(h, A, st, MODE, j);
      });
      if (e != cudaSuccess) return e;
    }
    h->launches++;
    e = timed(h, KT_STRIP, st, [&]() {
      return h->mixed ? launch_strip<float>(h, A, st, MODE, j)
                      : launch_strip<double>(h, A, st, MODE, j);
    });
    if (e != cudaSuccess) return e;
  }
  if (h->n_lines > 0) {
    h->launches++;
    e = timed(h, KT_LINE, st, [&]() { return launch_line(h, A, st, MODE, j); });
  }
  return e;
}

// One chunk of solve iterations on stream st: launches j = 0 .. chunk - 1
// (iterations *iter_k + j), then the counter advance.
cudaError_t enqueue_chunk(nmpc_handle* h, const IterArgs& A, cudaStream_t st, int chunk) {
  if (h->n_lines > 0) {
    // the line items of the instances still running
    nmpc_dev::k_compact_lines<<<1, nmpc_dev::COMPACT_THREADS, 0, st>>>(A);
    h->launches++;
  }
  // red-black: launches j = 2 i (half 0) and 2 i + 1 (half 1) of iteration i
  const int per = A.rb ? 2 : 1;
  for (int i = 0; i < chunk * per; ++i) {
    cudaError_t e = launch_iterate<nmpc_dev::MODE_SOLVE>(h, A, st, i);
    if (e != cudaSuccess) return e;
  }
  nmpc_dev::k_advance<<<1, 32, 0, st>>>(A.iter_k, chunk);
  h->launches++;
  return cudaGetLastError();
}

template <typename T>
cudaError_t configure_kernels(size_t smem) {
  IterKernel fns[5] = {nmpc_dev::k_iterate<T, 1, true>, nmpc_dev::k_iterate<T, 2, true>,
                       nmpc_dev::k_iterate<T, 4, true>, nmpc_dev::k_iterate<T, 8, true>,
                       nmpc_dev::k_iterate<T, GLOBAL_NC, false>};
  for (auto fn : fns) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  SolveKernel sfns[4] = {nmpc_dev::k_solve<T, 1>, nmpc_dev::k_solve<T, 2>, nmpc_dev::k_solve<T, 4>,
                         nmpc_dev::k_solve<T, 8>};
  for (auto fn : sfns) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  for (int n_lo = 1; n_lo <= 4; ++n_lo) {
    cudaError_t e = cudaFuncSetAttribute(strip_kernel<T>(n_lo),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(strip_kernel<T>(n_lo, true),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(patch_kernel<T>(n_lo), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    if (std::is_same<T, float>::value && n_lo <= 2) {
      for (int rbn = 0; rbn < 2; ++rbn) {
        e = cudaFuncSetAttribute(strip_kernel<T>(n_lo, rbn != 0, true),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
    }
  }
  cudaError_t e = cudaFuncSetAttribute(nmpc_dev::k_line<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(nmpc_dev::k_line<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  // (k_line_solve also has static shared memory: the barrier's code word)
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, nmpc_dev::k_line_solve);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(nmpc_dev::k_line_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(smem - fa.sharedSizeBytes));
}

// Whether instance I may run on the strip path: 2D, n_lo <= 4, and for
// n_u_it > 1 actuators on distinct cells more than 2 (n_lo - 1) cells apart
// (Manhattan), so that each actuator's u-iteration sees only its own
// response.
bool strip_eligible(const InstDev& I, const int* act, const nmpc_opts& o) {
  if (I.dim != 2 || o.n_lo > 4) return false;
  if (o.n_u_it > 1) {
    const int reach = 2 * (o.n_lo - 1);
    for (int a = 0; a < I.nu; ++a)
      for (int b = a + 1; b < I.nu; ++b) {
        const int dx = std::abs(act[a] % I.mx - act[b] % I.mx);
        const int dy = std::abs(act[a] / I.mx - act[b] / I.mx);
        if (dx + dy <= reach) return false;
      }
  }
  return true;
}

// Whether instance I runs on the line path: 1D, at most 32 x LINE_MAX_CPL
// cells, float32 lower layer.
bool line_eligible(const InstDev& I, bool mixed) {
  return mixed && I.dim == 1 && I.mx >= 1 && I.mx <= 32 * nmpc_dev::LINE_MAX_CPL &&
         I.nu <= nmpc_dev::MAX_NU;
}

// Cells per lane of a line of mx cells: the smallest of 1, 2, 4, 8 that covers it.
int line_cells_per_lane(int mx) {
  int c = 1;
  while (32 * c < mx) c *= 2;
  return c;
}

// Whether a stage of instance I fits a cluster of at most 8 CTAs with its
// float64 inputs staged in shared memory (the slab path's fast shape).
bool fits_cluster_staged(const InstDev& I, const nmpc_opts& o, bool mixed, int max_optin) {
  const size_t elem = mixed ? sizeof(float) : sizeof(double);
  const size_t small = mixed ? small_shared_bytes_t<float>() : small_shared_bytes_t<double>();
  for (int C = 1; C <= 8; ++C) {
    const size_t bytes = small + (size_t)slab_stride(I, C) * (nmpc_dev::NUM_FIELDS * elem +
                                                              nmpc_dev::NUM_SFIELDS * sizeof(double));
    int t, c;
    if (bytes <= (size_t)max_optin && thread_shape(slab_cells(I, C), o, &t, &c)) return true;
  }
  return false;
}

bool opts_ok(const nmpc_opts& o) {
  return (o.tol >= 0) && o.max_iter >= 0 && o.n_lo >= 1 && o.n_u_it >= 1 && o.check_every >= 1 &&
         (o.alpha > 0 && o.alpha <= 1) && (o.div_limit > 0) &&
         (o.precision == NMPC_FP64 || o.precision == NMPC_MIXED) && o.threads >= 0 &&
         o.threads <= 512 && (o.threads % 32) == 0 && o.cluster >= 0 && o.cluster <= 16 &&
         (o.cluster <= 8 || o.cluster == 16) && (o.split_min >= 0) &&
         (o.cells >= 0 && o.cells <= 8) && (o.strips >= 0 && o.strips <= 2) && (o.lines >= 0 && o.lines <= 2) &&
         (o.strip_rows >= 0 && o.strip_rows <= 65535) &&
         (o.variant == NMPC_VARIANT_JACOBI || (o.variant == NMPC_VARIANT_REDBLACK && o.alpha == 1.0)) &&
         o.barrier_wait_cycles >= 0 && (o.strip_cols == 0 || o.strip_cols == 1) &&
         (o.tail_rows == -1 || o.tail_rows == 0 || (o.tail_rows >= 8 && o.tail_rows <= 65535)) &&
         o.tail_below >= 0;
}

int validate(const nmpc_desc* d) {
  if (!d) return NMPC_ERR_BAD_ARG;
  if (d->dim != 1 && d->dim != 2) return NMPC_ERR_BAD_ARG;
  if (d->mx < 1 || d->my < 1 || (d->dim == 1 && d->my != 1)) return NMPC_ERR_BAD_ARG;
  if (d->horizon < 1 || d->n_u < 1 || !d->act_cell) return NMPC_ERR_BAD_ARG;
  if (d->n_u > NMPC_MAX_NU) return NMPC_ERR_UNSUPPORTED;
  if ((long long)d->mx * d->my > NMPC_MAX_NG) return NMPC_ERR_UNSUPPORTED;
  const long long ng = (long long)d->mx * d->my;
  for (int a = 0; a < d->n_u; ++a)
    if (d->act_cell[a] < 0 || d->act_cell[a] >= ng) return NMPC_ERR_BAD_ARG;
  if (!(d->h > 0) || !(d->q >= 0) || !(d->r > 0) || !(d->qf >= 0) || !(d->gamma >= 0))
    return NMPC_ERR_BAD_ARG;
  if (!(d->k0 > 0) || !std::isfinite(d->k1) || !std::isfinite(d->act_gain))
    return NMPC_ERR_BAD_ARG;
  return NMPC_OK;
}

// Kernel launches of one chunk of `chunk` iterations (enqueue_chunk): the
// line-list compaction, every path's iteration kernels (twice per iteration
// for red-black), the counter advance.
long long chunk_launches(const nmpc_handle* h, int chunk) {
  const long long per_iter = (h->n_work > 0 ? 1 : 0) + (h->n_strips > 0 ? 2 : 0) +
                             (h->n_lines > 0 ? 1 : 0);
  return (h->n_lines > 0 ? 1 : 0) + (long long)chunk * per_iter * (h->rb ? 2 : 1) + 1;
}

int run_chunk(nmpc_handle* h, const IterArgs& A, cudaStream_t st, int chunk) {
  if (h->opts.use_graph) {
    if (!h->graph_exec || h->graph_chunk != chunk) {
      if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
      }
      cudaStream_t cap;
      CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      const long long l0 = h->launches, i0 = h->iter_launches;
      cudaError_t e = enqueue_chunk(h, A, cap, chunk);
      h->launches = l0;  // capture is not execution
      h->iter_launches = i0;
      if (e != cudaSuccess) {
        cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        return NMPC_ERR_CUDA;
      }
      CK(cudaStreamEndCapture(cap, &g));
      CK(cudaGraphInstantiate(&h->graph_exec, g, 0));
      cudaGraphDestroy(g);
      cudaStreamDestroy(cap);
      h->graph_chunk = chunk;
    }
    CK(cudaGraphLaunch(h->graph_exec, st));
    h->launches += chunk_launches(h, chunk);
    h->iter_launches += chunk;
  } else {
    CK(enqueue_chunk(h, A, st, chunk));
  }
  return NMPC_OK;
}

// The iteration loop of a solve as one graph: a condition kernel, then a
// WHILE node whose body is one chunk of iteration launches, the counter
// advance and the condition kernel again (no host round trip between chunks).
int build_loop_graph(nmpc_handle* h, const IterArgs& A, int chunk) {
  if (h->loop_exec && h->loop_chunk == chunk) return NMPC_OK;
  if (h->loop_exec) {
    cudaGraphExecDestroy(h->loop_exec);
    h->loop_exec = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaStream_t cap = nullptr;
  int rc = NMPC_ERR_CUDA;
  const long long l0 = h->launches, i0 = h->iter_launches;
  do {
    if (cudaGraphCreate(&g, 0) != cudaSuccess) break;
    cudaGraphConditionalHandle cond;
    if (cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault) != cudaSuccess)
      break;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) break;
    // the first decision (an already finished solve runs no chunk)
    if (cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      break;
    nmpc_dev::k_loop_cond<<<1, 32, 0, cap>>>(cond, A.n_active, A.iter_k, h->opts.max_iter);
    cudaGraph_t gc = nullptr;
    if (cudaStreamEndCapture(cap, &gc) != cudaSuccess) break;
    cudaGraphNode_t first;
    size_t nfirst = 1;
    if (cudaGraphGetNodes(g, &first, &nfirst) != cudaSuccess || nfirst != 1) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if (cudaGraphAddNode(&loop, g, &first, nullptr, 1, &cp) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      break;
    cudaError_t e = enqueue_chunk(h, A, cap, chunk);
    nmpc_dev::k_loop_cond<<<1, 32, 0, cap>>>(cond, A.n_active, A.iter_k, h->opts.max_iter);
    cudaGraph_t gb = nullptr;
    if (cudaStreamEndCapture(cap, &gb) != cudaSuccess || e != cudaSuccess) break;
    if (cudaGraphInstantiate(&h->loop_exec, g, 0) != cudaSuccess) break;
    h->loop_chunk = chunk;
    rc = NMPC_OK;
  } while (false);
  h->launches = l0;  // capture is not execution
  h->iter_launches = i0;
  if (g) cudaGraphDestroy(g);
  if (cap) cudaStreamDestroy(cap);
  if (rc != NMPC_OK) {
    cudaGetLastError();
    fprintf(stderr, "nmpc: could not build the solve-loop graph\n");
  }
  return rc;
}

FinalArgs make_final(nmpc_handle* h, double* u_out) {
  FinalArgs F{};
  F.inst = h->inst_d;
  F.n_inst = h->n_inst;
  for (int q = 0; q < 2; ++q) {
    F.xs[q] = h->xb[q];
    F.us[q] = h->ub[q];
    F.ls[q] = h->lb[q];
  }
  F.xc = h->xb[2];
  F.uc = h->ub[2];
  F.lc = h->lb[2];
  F.u_out = u_out;
  F.status = h->status;
  F.iters = h->iters;
  F.final_buf = h->final_buf;
  F.fin_inf = h->fin_inf;
  F.fin_2 = h->fin_2;
  F.res_inf = h->res_inf;
  F.res_sq = h->res_sq;
  F.tol = h->opts.tol;
  F.max_iter = h->opts.max_iter;
  return F;
}

dim3 per_instance_grid(const nmpc_handle* h) {
  return dim3(64, (unsigned)h->n_inst);
}

// The solve proper, on device buffers owned by the handle (x0_d, ref_d).
int solve_core(nmpc_handle* h, int horizon, const double* weights, int init, double* u_out,
               nmpc_stats* stats, cudaStream_t st) {
  if (horizon != 0) {
    for (const InstDev& I : h->inst_h)
      if (I.N != horizon) return NMPC_ERR_BAD_ARG;
  }
  if (init != NMPC_INIT_COLD && init != NMPC_INIT_WARM && init != NMPC_INIT_GUESS &&
      init != NMPC_INIT_SHIFT)
    return NMPC_ERR_BAD_ARG;
  if (init != NMPC_INIT_COLD && !h->has_state) return NMPC_ERR_BAD_ARG;
  if (weights) {
    nmpc_dev::k_set_weights<<<(h->n_inst + 127) / 128, 128, 0, st>>>(h->inst_d, h->n_inst,
                                                                    weights);
    h->launches++;
    CK(cudaGetLastError());
  }
  IterArgs A = make_args(h);
  // S^0 and the control words (again after a persistent launch that could not
  // finish: the state it left is discarded)
  auto start = [&]() -> int {
    if (init == NMPC_INIT_WARM || init == NMPC_INIT_GUESS) {
      CK(cudaMemcpyAsync(h->xb[0], h->xb[2], h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(h->lb[0], h->lb[2], h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(h->ub[0], h->ub[2], h->n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    const int mode = (init == NMPC_INIT_COLD) ? 0 : (init == NMPC_INIT_SHIFT ? 2 : 1);
    nmpc_dev::k_init_control<<<per_instance_grid(h), 256, 0, st>>>(
        A, mode, init == NMPC_INIT_WARM, h->xb[2], h->ub[2], h->lb[2]);
    h->launches++;
    CK(cudaGetLastError());
    return NMPC_OK;
  };
  int rc0 = start();
  if (rc0 != NMPC_OK) return rc0;

  bool done = false;
  if (h->persistent) {
    const LaunchPlan P = plan_of(h);
    CK(h->mixed ? launch_solve<float>(P, A, st) : launch_solve<double>(P, A, st));
    h->launches++;
    h->iter_launches++;
    CK(cudaMemcpyAsync(h->h_active, h->ictl, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h->h_active[7] == 0) {
      done = true;
    } else {
      // a barrier wait ran out (the clusters were not all resident): from now
      // on this handle iterates with one launch per iteration
      fprintf(stderr, "nmpc: persistent launch not co-resident; using per-iteration launches\n");
      h->persistent = false;
      rc0 = start();
      if (rc0 != NMPC_OK) return rc0;
    }
  }
  if (!done && h->line_persistent) {
    // the whole solve in one cooperative launch over the line list
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)h->line_solve_grid);
    cfg.blockDim = dim3(32 * nmpc_dev::LINE_WARPS);
    cfg.dynamicSmemBytes = h->line_smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, nmpc_dev::k_line_solve, A));
    h->launches++;
    h->iter_launches++;
    CK(cudaMemcpyAsync(h->h_active, h->ictl, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h->h_active[7] == 0) {
      done = true;
    } else {
      // a barrier wait ran out: from now on this handle iterates with one
      // launch per iteration
      fprintf(stderr, "nmpc: persistent line launch timed out; using per-iteration launches\n");
      h->line_persistent = false;
      rc0 = start();
      if (rc0 != NMPC_OK) return rc0;
    }
  }
  const int chunk = std::max(1, h->opts.check_every);
  bool loop_graph = false;
  if (!done && h->opts.use_graph) {
    // the whole loop on the device: one graph launch, no host polls
    int rc = build_loop_graph(h, A, chunk);
    if (rc != NMPC_OK) return rc;
    CK(cudaGraphLaunch(h->loop_exec, st));
    loop_graph = true;
    done = true;
  }
  long long launched = 0;
  while (!done && launched <= h->opts.max_iter) {
    int rc = run_chunk(h, A, st, chunk);
    if (rc != NMPC_OK) return rc;
    launched += chunk;
    CK(cudaMemcpyAsync(h->h_active, h->ictl + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*h->h_active == 0) break;
  }
  FinalArgs F = make_final(h, u_out);
  nmpc_dev::k_finalize_status<<<(h->n_inst + 127) / 128, 128, 0, st>>>(F);
  nmpc_dev::k_gather_final<<<per_instance_grid(h), 256, 0, st>>>(F);
  h->launches += 2;
  CK(cudaGetLastError());
  h->has_state = true;
  const int n = h->n_inst;
  CK(cudaMemcpyAsync(h->h_status, h->status, n * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->h_iters, h->iters, n * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->h_f64, h->f64_count, n * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->h_fin, h->fin_inf, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->h_fin + n, h->fin_2, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (loop_graph)
    CK(cudaMemcpyAsync(h->h_active, h->ictl, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (loop_graph) {
    // launch accounting: the loop ran iter_k / chunk chunks
    const long long runs = (h->h_active[0] + chunk - 1) / chunk;
    h->launches += 1 + runs * (chunk_launches(h, chunk) + 1);  // + the condition kernels
    h->iter_launches += runs * chunk;
  }
  int rc = NMPC_OK;
  for (int b = 0; b < n; ++b) {
    if (stats) {
      stats[b].status = h->h_status[b];
      stats[b].iters = h->h_iters[b];
      stats[b].res_inf = h->h_fin[b];
      stats[b].res_2 = h->h_fin[n + b];
      stats[b].f64_iters = h->h_f64[b];
    }
    if (rc == NMPC_OK) {
      if (h->h_status[b] == nmpc_dev::ST_DIVERGED) rc = NMPC_ERR_DIVERGED;
      else if (h->h_status[b] != nmpc_dev::ST_CONVERGED) rc = NMPC_ERR_NOT_CONVERGED;
    }
  }
  return rc;
}

}  // namespace

namespace {

// Capture what fn enqueues on `cap` into graph g after the nodes deps[0..nd);
// *last receives the capture's terminal node (the captured work is a chain).
template <typename F>
cudaError_t capture_after(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, cudaStream_t cap,
                          F fn, cudaGraphNode_t* last) {
  cudaError_t e = cudaStreamBeginCaptureToGraph(cap, g, deps, nullptr, nd,
                                                cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t ef = fn();
  cudaStreamCaptureStatus status;
  const cudaGraphNode_t* term = nullptr;
  size_t nterm = 0;
  cudaError_t ei = cudaStreamGetCaptureInfo(cap, &status, nullptr, nullptr, &term, nullptr, &nterm);
  if (ei == cudaSuccess && nterm == 1) *last = term[0];
  else if (ei == cudaSuccess) ei = cudaErrorInvalidValue;
  cudaGraph_t gg = nullptr;
  e = cudaStreamEndCapture(cap, &gg);
  if (ef != cudaSuccess) return ef;
  if (ei != cudaSuccess) return ei;
  return e;
}

// Add a WHILE node to g after `dep`; returns the node and its body graph.
cudaError_t add_while(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle c,
                      cudaGraphNode_t* node, cudaGraph_t* body) {
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = c;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaError_t e = cudaGraphAddNode(node, g, &dep, nullptr, 1, &cp);
  if (e == cudaSuccess) *body = cp.conditional.phGraph_out[0];
  return e;
}

// The closed loop as one graph: a WHILE node over the steps whose body copies
// the plant state into x0, starts the solve (cold or from the handle's state
// at step 0, shifted afterwards), runs the solve loop (a nested WHILE node
// over chunks of iteration launches), settles the instances, records the
// step's status / iterations / residual, and moves the plant.
// State (forward) and costate (backward) trajectories of controls u from x0
// into x, lam: 2 N_max launches on st.
cudaError_t enqueue_rollout(nmpc_handle* h, const double* x0, const double* ref, const double* u,
                            double* x, double* lam, cudaStream_t st) {
  int nmax = 0;
  for (const InstDev& I : h->inst_h) nmax = std::max(nmax, I.N);
  // float32 arithmetic on NMPC_MIXED handles (a start guess), else float64
  const auto ks = h->mixed ? nmpc_dev::k_rollout_state<float> : nmpc_dev::k_rollout_state<double>;
  const auto kc =
      h->mixed ? nmpc_dev::k_rollout_costate<float> : nmpc_dev::k_rollout_costate<double>;
  for (int i = 0; i < nmax; ++i) {
    ks<<<per_instance_grid(h), 256, 0, st>>>(h->inst_d, h->n_inst, h->act_d, x0, u, x, i);
    h->launches++;
  }
  for (int i = 0; i < nmax; ++i) {
    kc<<<per_instance_grid(h), 256, 0, st>>>(h->inst_d, h->n_inst, ref, x, lam, i);
    h->launches++;
  }
  return cudaGetLastError();
}

int closed_loop_graph(nmpc_handle* h, double* w, int steps, int n_sub, double* u_hist,
                      int* iters_hist, double* res_hist, cudaStream_t st,
                      nmpc_start_fn start = nullptr, void* ctx = nullptr,
                      const double* u_guess = nullptr) {
  const int n = h->n_inst;
  const int chunk = std::max(1, h->opts.check_every);
  IterArgs A = make_args(h);
  FinalArgs F = make_final(h, nullptr);
  int* step = h->ictl + 1;
  const int first_mode = h->has_state ? 2 : 0;
  int* st_hist = nullptr;
  int* it_hist = nullptr;
  double* rs_hist = nullptr;
  CK(dev_alloc(&st_hist, (size_t)steps * n));
  CK(dev_alloc(&it_hist, (size_t)steps * n));
  CK(dev_alloc(&rs_hist, (size_t)steps * n));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaStream_t cap = nullptr;
  const long long l0 = h->launches, i0 = h->iter_launches;
  int rc = NMPC_ERR_CUDA;
  do {
    if (cudaGraphCreate(&g, 0) != cudaSuccess) break;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) break;
    cudaGraphConditionalHandle outer, inner;
    if (cudaGraphConditionalHandleCreate(&outer, g, 0, cudaGraphCondAssignDefault) != cudaSuccess)
      break;
    cudaGraphNode_t n0, nloop, n1, ninner, n2;
    cudaGraph_t body_o = nullptr, body_i = nullptr;
    if (capture_after(g, nullptr, 0, cap, [&]() {
          nmpc_dev::k_cl_start<<<1, 32, 0, cap>>>(step, steps, outer);
          return cudaGetLastError();
        }, &n0) != cudaSuccess)
      break;
    if (add_while(g, n0, outer, &nloop, &body_o) != cudaSuccess) break;
    if (cudaGraphConditionalHandleCreate(&inner, body_o, 0, cudaGraphCondAssignDefault) !=
        cudaSuccess)
      break;
    // step: x0 <- w, start (cold / shifted, or the caller's guess completed
    // by its state and costate trajectories), first loop decision
    if (capture_after(body_o, nullptr, 0, cap, [&]() {
          nmpc_dev::k_copy_f64<<<256, 256, 0, cap>>>(h->x0_d, w, h->n_g);
          if (start) {
            start(ctx, (void*)cap);
            nmpc_dev::k_copy_f64<<<256, 256, 0, cap>>>(h->ub[0], u_guess, h->n_u);
            cudaError_t e = enqueue_rollout(h, h->x0_d, h->ref_d, h->ub[0], h->xb[0], h->lb[0], cap);
            if (e != cudaSuccess) return e;
            nmpc_dev::k_init_control<<<per_instance_grid(h), 256, 0, cap>>>(
                A, 1, 0, h->xb[2], h->ub[2], h->lb[2], nullptr);
          } else {
            nmpc_dev::k_init_control<<<per_instance_grid(h), 256, 0, cap>>>(
                A, first_mode, 0, h->xb[2], h->ub[2], h->lb[2], step);
          }
          nmpc_dev::k_loop_cond<<<1, 32, 0, cap>>>(inner, A.n_active, A.iter_k, h->opts.max_iter);
          return cudaGetLastError();
        }, &n1) != cudaSuccess)
      break;
    if (add_while(body_o, n1, inner, &ninner, &body_i) != cudaSuccess) break;
    if (capture_after(body_i, nullptr, 0, cap, [&]() {
          cudaError_t e = enqueue_chunk(h, A, cap, chunk);
          nmpc_dev::k_loop_cond<<<1, 32, 0, cap>>>(inner, A.n_active, A.iter_k, h->opts.max_iter);
          return e != cudaSuccess ? e : cudaGetLastError();
        }, &n2) != cudaSuccess)
      break;
    // step: settle, record, plant, next
    if (capture_after(body_o, &ninner, 1, cap, [&]() {
          nmpc_dev::k_finalize_status<<<(n + 127) / 128, 128, 0, cap>>>(F);
          nmpc_dev::k_gather_final<<<per_instance_grid(h), 256, 0, cap>>>(F);
          nmpc_dev::k_cl_record<<<(n + 127) / 128, 128, 0, cap>>>(step, n, h->status, h->iters,
                                                                  h->fin_inf, st_hist, it_hist,
                                                                  rs_hist);
          for (int k = 0; k < n_sub; ++k) {
            const bool even = (k % 2) == 0;
            nmpc_dev::k_plant_substep<<<dim3(32, n), 256, 0, cap>>>(
                h->inst_d, n, h->act_d, even ? w : h->x0_d, even ? h->x0_d : w, h->ub[2],
                (k == 0) ? u_hist : nullptr, 0.0, n_sub, step, (long long)h->nu_tot);
          }
          if (n_sub % 2 == 1) nmpc_dev::k_copy_f64<<<256, 256, 0, cap>>>(w, h->x0_d, h->n_g);
          nmpc_dev::k_cl_next<<<1, 32, 0, cap>>>(step, steps, outer);
          return cudaGetLastError();
        }, &n2) != cudaSuccess)
      break;
    if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) break;
    rc = NMPC_OK;
  } while (false);
  h->launches = l0;  // capture is not execution
  h->iter_launches = i0;
  if (rc == NMPC_OK && cudaGraphLaunch(ge, st) != cudaSuccess) rc = NMPC_ERR_CUDA;
  std::vector<int> sth((size_t)steps * n), ith((size_t)steps * n);
  std::vector<double> rsh((size_t)steps * n);
  if (rc == NMPC_OK) {
    if (cudaMemcpyAsync(sth.data(), st_hist, sth.size() * sizeof(int), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(ith.data(), it_hist, ith.size() * sizeof(int), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(rsh.data(), rs_hist, rsh.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = NMPC_ERR_CUDA;
  }
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (cap) cudaStreamDestroy(cap);
  cudaFree(st_hist);
  cudaFree(it_hist);
  cudaFree(rs_hist);
  if (rc != NMPC_OK) {
    cudaGetLastError();
    fprintf(stderr, "nmpc: closed-loop graph failed\n");
    return rc;
  }
  h->has_state = true;
  int rc_all = NMPC_OK;
  for (int t = 0; t < steps; ++t) {
    for (int b = 0; b < n; ++b) {
      const size_t o = (size_t)t * n + b;
      if (iters_hist) iters_hist[o] = ith[o];
      if (res_hist) res_hist[o] = rsh[o];
      if (rc_all == NMPC_OK) {
        if (sth[o] == nmpc_dev::ST_DIVERGED) rc_all = NMPC_ERR_DIVERGED;
        else if (sth[o] != nmpc_dev::ST_CONVERGED) rc_all = NMPC_ERR_NOT_CONVERGED;
      }
    }
    // launch accounting from the iterations each step ran
    int kmax = 0;
    for (int b = 0; b < n; ++b) kmax = std::max(kmax, ith[(size_t)t * n + b] + 2);
    const long long runs = (kmax + chunk - 1) / chunk;
    h->launches += 8 + n_sub + runs * (chunk_launches(h, chunk) + 1);
    if (start) h->launches += 1 + 2 * (long long)h->n_max_horizon;  // guess copy, rollout
    h->iter_launches += runs * chunk;
  }
  h->launches += 1;
  return rc_all;
}

}  // namespace

extern "C" {

void nmpc_default_opts(nmpc_opts* o) {
  if (!o) return;
  o->tol = 1e-6;
  o->max_iter = 2000;
  o->n_lo = 2;
  o->n_u_it = 2;
  o->precision = NMPC_FP64;
  o->check_every = 16;
  o->alpha = 1.0;
  o->div_limit = 1e8;
  o->threads = 0;
  o->use_graph = 1;
  o->cluster = 0;
  o->split_min = 1e-7;
  o->u_local = 0;
  o->cells = 0;
  o->persistent = 0;
  o->variant = NMPC_VARIANT_JACOBI;
  o->barrier_wait_cycles = 0;
  o->strips = 0;
  o->strip_rows = 0;
  o->lines = 0;
  o->strip_cols = 0;
  o->tail_rows = 0;
  o->tail_below = 0;
}

int nmpc_setup(const nmpc_desc* descs, int n_instances, const nmpc_opts* opts,
               nmpc_handle** out) {
  if (!out || !descs || n_instances < 1 || n_instances > 65535) return NMPC_ERR_BAD_ARG;
  *out = nullptr;
  nmpc_opts o;
  nmpc_default_opts(&o);
  if (opts) o = *opts;
  if (!opts_ok(o)) return NMPC_ERR_BAD_ARG;
  for (int b = 0; b < n_instances; ++b) {
    int rc = validate(&descs[b]);
    if (rc != NMPC_OK) return rc;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return NMPC_ERR_NO_DEVICE;

  nmpc_handle* h = new (std::nothrow) nmpc_handle();
  if (!h) return NMPC_ERR_CUDA;
  h->n_inst = n_instances;
  h->opts = o;
  h->mixed = (o.precision == NMPC_MIXED);
  h->rb = (o.variant == NMPC_VARIANT_REDBLACK);
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);

  std::vector<int> act_all;
  for (int b = 0; b < n_instances; ++b) {
    const nmpc_desc& d = descs[b];
    InstDev I{};
    I.dim = d.dim;
    I.mx = d.mx;
    I.my = d.my;
    I.ng = d.mx * d.my;
    I.N = d.horizon;
    I.nu = d.n_u;
    I.act_off = (int)act_all.size();
    I.s_off = h->n_s;
    I.u_off = h->n_u;
    I.g_off = h->n_g;
    I.h = d.h;
    I.q = d.q;
    I.r = d.r;
    I.qf = d.qf;
    I.gamma = d.gamma;
    I.k0 = d.k0;
    I.k1 = d.k1;
    I.b0 = d.act_gain;
    const double dx = 1.0 / (d.mx + 1), dy = 1.0 / (d.my + 1);
    I.cx = 1.0 / (dx * dx);
    I.cy = (d.dim == 2) ? 1.0 / (dy * dy) : 0.0;
    nmpc_dev::derive(I);
    for (int a = 0; a < d.n_u; ++a) act_all.push_back(d.act_cell[a]);
    h->nu_tot += d.n_u;
    h->n_s += (long long)I.N * I.ng;
    h->n_u += (long long)I.N * I.nu;
    h->n_g += I.ng;
    h->ng_max = std::max(h->ng_max, I.ng);
    h->nu_max = std::max(h->nu_max, I.nu);
    h->n_max_horizon = std::max(h->n_max_horizon, I.N);
    h->inst_h.push_back(I);
  }

  // launch configuration
  int max_optin = 0;
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  cudaError_t ce = h->mixed ? configure_kernels<float>((size_t)max_optin)
                            : configure_kernels<double>((size_t)max_optin);
  if (ce != cudaSuccess) {
    fprintf(stderr, "nmpc: kernel attribute: %s\n", cudaGetErrorString(ce));
    delete h;
    return NMPC_ERR_CUDA;
  }
  // instances on the strip path, and the strip shape (shared by all of
  // them): 32 - 2E own columns (one warp lane per region column), or with
  // two columns per lane 64 - 2P (P = 2 n_lo, k_strip2), and ty own rows, by
  // default enough strips for about four waves of warps
  std::vector<char> on_strips(n_instances, 0);
  const int E = 2 * o.n_lo - 1;
  int ty = 0, my_max = 0;
  bool two = h->mixed && o.n_lo <= 2 && o.strip_cols == 0;
  if (o.strips != 2) {
    for (int b = 0; b < n_instances; ++b) {
      const InstDev& I = h->inst_h[b];
      if (!strip_eligible(I, act_all.data() + I.act_off, o)) continue;
      if (o.strips == 0 && fits_cluster_staged(I, o, h->mixed, max_optin)) continue;
      on_strips[b] = 1;
      my_max = std::max(my_max, I.my);
      // column pairs are 16-byte aligned: even width and even array offsets
      if ((I.mx & 1) || (I.s_off & 1) || (I.g_off & 1)) two = false;
    }
  }
  const int tx = two ? 64 - 2 * nmpc_dev::strip2_pad(o.n_lo) : 32 - 2 * E;
  if (my_max > 0) {
    long long whole = 0;  // strips with whole columns
    for (int b = 0; b < n_instances; ++b)
      if (on_strips[b]) {
        const InstDev& I = h->inst_h[b];
        whole += (long long)I.N * ((I.mx + tx - 1) / tx);
      }
    if (o.strip_rows) {
      ty = std::min(o.strip_rows, my_max);
    } else {
      const long long target = 4LL * std::max(1, h->num_sms) * 32;
      const long long segs = std::max(1LL, (target + whole - 1) / whole);
      ty = (int)std::min<long long>(my_max, std::max(16LL, (my_max + segs - 1) / segs));
    }
  }
  // the tail plan (two columns per lane, solves): strips of ty_tail own rows
  // where the main plan's are at least four times taller
  int ty_tail = 0;
  if (my_max > 0 && two && o.tail_rows >= 0) {
    const int want = o.tail_rows > 0 ? o.tail_rows : 64;
    if (o.tail_rows > 0 ? want < ty : ty >= 4 * want) ty_tail = want;
  }
  std::vector<int2> work;
  std::vector<int4> strips, patches, lines, tail;
  std::vector<InstDev> cl_inst;
  for (int b = 0; b < n_instances; ++b) {
    const InstDev& I = h->inst_h[b];
    if (o.lines != 2 && line_eligible(I, h->mixed)) {
      h->n_line_inst++;
      const int cpl = line_cells_per_lane(I.mx);
      for (int s = 0; s < I.N; ++s) lines.push_back(make_int4(b, s, cpl, 0));
    } else if (on_strips[b]) {
      h->n_strip_inst++;
      for (int s = 0; s < I.N; ++s) {
        for (int y0 = 0; y0 < I.my; y0 += ty)
          for (int x0 = 0; x0 < I.mx; x0 += tx) strips.push_back(make_int4(b, s, x0, y0));
        if (ty_tail > 0)
          for (int y0 = 0; y0 < I.my; y0 += ty_tail)
            for (int x0 = 0; x0 < I.mx; x0 += tx) tail.push_back(make_int4(b, s, x0, y0));
        for (int a = 0; a < I.nu; ++a) patches.push_back(make_int4(b, s, a, 0));
      }
    } else {
      cl_inst.push_back(I);
      for (int s = 0; s < I.N; ++s) work.push_back(make_int2(b, s));
    }
  }
  // line items grouped by cells per lane (neighbouring CTAs then run the same
  // specialisation of the kernel body: instruction-cache locality)
  std::stable_sort(lines.begin(), lines.end(),
                   [](const int4& a, const int4& b) { return a.z < b.z; });
  if (h->rb) {
    // red-black: each list's even-stage items first, so that a half-sweep
    // launch covers exactly its own items
    auto even2 = [](const int2& w) { return (w.y & 1) == 0; };
    auto even4 = [](const int4& w) { return (w.y & 1) == 0; };
    h->n_work_even = (int)(std::stable_partition(work.begin(), work.end(), even2) - work.begin());
    h->n_strips_even =
        (int)(std::stable_partition(strips.begin(), strips.end(), even4) - strips.begin());
    h->n_tail_even = (int)(std::stable_partition(tail.begin(), tail.end(), even4) - tail.begin());
    h->n_patches_even =
        (int)(std::stable_partition(patches.begin(), patches.end(), even4) - patches.begin());
  }
  h->n_work = (int)work.size();
  h->n_strips = (int)strips.size();
  h->n_patches = (int)patches.size();
  h->n_lines = (int)lines.size();
  h->line_smem = nmpc_dev::LINE_WARPS * ((sizeof(nmpc_dev::LineShared) + 15) & ~size_t(15));
  if (h->n_lines > 0 && h->line_smem > (size_t)max_optin) {
    fprintf(stderr, "nmpc: line path needs %zu bytes of shared memory\n", h->line_smem);
    delete h;
    return NMPC_ERR_UNSUPPORTED;
  }
  // one warp per item of the whole list (solve-mode launches past the running
  // items' count return at once)
  h->line_grid = (h->n_lines + nmpc_dev::LINE_WARPS - 1) / nmpc_dev::LINE_WARPS;
  // persistent line solve (Jacobi, a handle whose stages are all on the line
  // path): as many CTAs as are resident at once, at most one per four items
  if (o.persistent && o.variant == NMPC_VARIANT_JACOBI && h->n_lines > 0 && h->n_work == 0 &&
      h->n_strips == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nmpc_dev::k_line_solve,
                                                      32 * nmpc_dev::LINE_WARPS,
                                                      h->line_smem) == cudaSuccess &&
        per_sm > 0) {
      h->line_solve_grid = std::min(per_sm * std::max(1, h->num_sms), h->line_grid);
      h->line_persistent = true;
    } else {
      cudaGetLastError();
    }
  }
  if (h->n_strips > 0 && two) {
    h->strip2 = true;
    h->strip_x = tx;
    h->strip_y = ty;
    if (!tail.empty()) {
      // the tail plan while the running instances' main-plan strips fill
      // fewer than six waves of resident warps (3 CTAs of 4 warps per SM)
      h->n_tail = (int)tail.size();
      h->tail_y = ty_tail;
      const long long per_launch = std::max(1, h->rb ? h->n_strips / 2 : h->n_strips);
      const long long waves6 = 6LL * std::max(1, h->num_sms) * STRIP2_MIN_BLOCKS *
                               nmpc_dev::STRIP2_WARPS;
      h->tail_below = o.tail_below > 0
                          ? o.tail_below
                          : (int)std::max(1LL, waves6 * h->n_strip_inst / per_launch);
    } else {
      h->n_tail_even = 0;
    }
    h->strip_threads = 32 * nmpc_dev::STRIP2_WARPS;
    h->strip_region = 64 * (ty + 2 * E);
    constexpr int NF1 = nmpc_dev::strip_fields(true);
    const size_t ws_bytes =
        o.n_lo <= 1 ? sizeof(nmpc_dev::StripShared2<nmpc_dev::strip_ring_rows(1)>)
                    : sizeof(nmpc_dev::StripShared2<nmpc_dev::strip_ring_rows(2)>);
    const size_t ws_rb =
        o.n_lo <= 1 ? sizeof(nmpc_dev::StripShared2<nmpc_dev::strip_ring_rows(1), NF1>)
                    : sizeof(nmpc_dev::StripShared2<nmpc_dev::strip_ring_rows(2), NF1>);
    h->strip_smem = nmpc_dev::STRIP2_WARPS * ((ws_bytes + 15) & ~size_t(15));
    h->strip_smem_rb = nmpc_dev::STRIP2_WARPS * ((ws_rb + 15) & ~size_t(15));
  } else if (h->n_strips > 0) {
    h->strip_x = tx;
    h->strip_y = ty;
    h->strip_threads = 32 * nmpc_dev::STRIP_WARPS;
    h->strip_region = 32 * (ty + 2 * E);
    const size_t ws_bytes =
        o.n_lo <= 1   ? sizeof(nmpc_dev::StripShared<nmpc_dev::strip_ring_rows(1)>)
        : o.n_lo == 2 ? sizeof(nmpc_dev::StripShared<nmpc_dev::strip_ring_rows(2)>)
        : o.n_lo == 3 ? sizeof(nmpc_dev::StripShared<nmpc_dev::strip_ring_rows(3)>)
                      : sizeof(nmpc_dev::StripShared<nmpc_dev::strip_ring_rows(4)>);
    h->strip_smem = nmpc_dev::STRIP_WARPS * ((ws_bytes + 15) & ~size_t(15));
    constexpr int NF1 = nmpc_dev::strip_fields(true);  // red-black half 1's ring
    const size_t ws_rb =
        o.n_lo <= 1   ? sizeof(nmpc_dev::StripShared<nmpc_dev::strip_ring_rows(1), NF1>)
        : o.n_lo == 2 ? sizeof(nmpc_dev::StripShared<nmpc_dev::strip_ring_rows(2), NF1>)
        : o.n_lo == 3 ? sizeof(nmpc_dev::StripShared<nmpc_dev::strip_ring_rows(3), NF1>)
                      : sizeof(nmpc_dev::StripShared<nmpc_dev::strip_ring_rows(4), NF1>);
    h->strip_smem_rb = nmpc_dev::STRIP_WARPS * ((ws_rb + 15) & ~size_t(15));
  }
  if (h->n_strips > 0) {
    // k_patch (both strip kernels): one region of radius E per warp
    const size_t P2 = (size_t)(2 * E + 1) * (2 * E + 1);
    h->patch_smem = PATCH_WARPS * (((sizeof(nmpc_dev::PatchShared) + 15) & ~size_t(15)) +
                                   8 * P2 * sizeof(double));
    if (h->strip_smem > (size_t)max_optin || h->patch_smem > (size_t)max_optin ||
        (h->rb && h->strip_smem_rb > (size_t)max_optin)) {
      fprintf(stderr, "nmpc: strip shape needs %zu bytes of shared memory\n", h->strip_smem);
      delete h;
      return NMPC_ERR_UNSUPPORTED;
    }
  }
  LaunchPlan P;
  if (h->n_work > 0)
    P = plan_launch(cl_inst.data(), (int)cl_inst.size(), h->n_work, o, h->mixed,
                    std::max(1, h->num_sms), max_optin);
  P.persistent = P.persistent && h->n_strips == 0 && h->n_lines == 0;
  if (h->n_work > 0 && !P.smem_mode) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, iter_kernel_of(h->mixed, GLOBAL_NC, false), P.threads, P.smem);
    P.grid = std::min(h->n_work, std::max(1, per_sm) * std::max(1, h->num_sms));
  }
  h->threads = P.threads;
  h->cpt = P.cpt;
  h->persistent = P.persistent;
  h->resident_clusters = P.resident_clusters;
  h->csize = P.csize;
  h->slab_max = P.slab_max;
  h->smem = P.smem;
  h->smem_mode = P.smem_mode;
  h->stage = P.stage;
  h->local_u = P.local_u;
  h->box_r = P.box_r;
  h->box_bytes = P.box_bytes;
  h->grid = P.grid;
  const size_t elem = h->mixed ? sizeof(float) : sizeof(double);
  const size_t work_bytes = (size_t)nmpc_dev::NUM_FIELDS * h->slab_max * elem + h->box_bytes;

  bool ok = true;
  auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
  A(dev_alloc(&h->inst_d, n_instances));
  A(dev_alloc(&h->work_d, h->n_work));
  A(dev_alloc(&h->strips_d, h->n_strips));
  A(dev_alloc(&h->tail_d, h->n_tail));
  A(dev_alloc(&h->patches_d, h->n_patches));
  A(dev_alloc(&h->lines_d, h->n_lines));
  A(dev_alloc(&h->lines_act_d, h->n_lines));
  A(dev_alloc(&h->v3_d, h->n_strips > 0 ? h->n_u : 0));
  A(dev_alloc(&h->act_d, act_all.size()));
  A(dev_alloc(&h->x0_d, h->n_g));
  A(dev_alloc(&h->ref_d, h->n_g));
  if (h->strip2) A(dev_alloc(&h->ref_f_d, h->n_g));
  A(dev_alloc(&h->uo_d, h->n_u));
  A(dev_alloc(&h->w_d, 3 * (size_t)n_instances));
  for (int q = 0; q < 3; ++q) {
    A(dev_alloc(&h->xb[q], h->n_s));
    A(dev_alloc(&h->lb[q], h->n_s));
    A(dev_alloc(&h->ub[q], h->n_u));
  }
  A(dev_alloc(&h->ictl, 12));
  A(dev_alloc(&h->res_inf, (size_t)nmpc_dev::RES_SLOTS * n_instances));
  A(dev_alloc(&h->res_err, (size_t)nmpc_dev::RES_SLOTS * n_instances));
  A(dev_alloc(&h->res_sq, (size_t)nmpc_dev::RES_SLOTS * n_instances));
  A(dev_alloc(&h->f64_count, n_instances));
  A(dev_alloc(&h->full0, n_instances));
  A(dev_alloc(&h->res_first, n_instances));
  A(dev_alloc(&h->status, n_instances));
  A(dev_alloc(&h->iters, n_instances));
  A(dev_alloc(&h->final_buf, n_instances));
  A(dev_alloc(&h->fin_inf, n_instances));
  A(dev_alloc(&h->fin_2, n_instances));
  if (h->n_work > 0 && !h->smem_mode) {
    h->scratch_stride = (long long)((work_bytes + 255) & ~size_t(255));
    A(cudaMalloc((void**)&h->scratch, (size_t)h->scratch_stride * h->grid));
  }
  A(cudaMallocHost((void**)&h->h_active, 8 * sizeof(int)));
  A(cudaMallocHost((void**)&h->h_status, n_instances * sizeof(int)));
  A(cudaMallocHost((void**)&h->h_iters, n_instances * sizeof(int)));
  A(cudaMallocHost((void**)&h->h_f64, n_instances * sizeof(int)));
  A(cudaMallocHost((void**)&h->h_fin, 2 * n_instances * sizeof(double)));
  A(cudaMallocHost((void**)&h->h_res, 2 * n_instances * sizeof(double)));
  A(cudaMallocHost((void**)&h->h_resinf, n_instances * sizeof(unsigned long long)));
  if (ok) {
    A(cudaMemcpy(h->inst_d, h->inst_h.data(), n_instances * sizeof(InstDev), cudaMemcpyHostToDevice));
    if (!work.empty())
      A(cudaMemcpy(h->work_d, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice));
    if (!strips.empty())
      A(cudaMemcpy(h->strips_d, strips.data(), strips.size() * sizeof(int4), cudaMemcpyHostToDevice));
    if (h->n_tail > 0)
      A(cudaMemcpy(h->tail_d, tail.data(), tail.size() * sizeof(int4), cudaMemcpyHostToDevice));
    if (!patches.empty())
      A(cudaMemcpy(h->patches_d, patches.data(), patches.size() * sizeof(int4),
                   cudaMemcpyHostToDevice));
    if (!lines.empty())
      A(cudaMemcpy(h->lines_d, lines.data(), lines.size() * sizeof(int4), cudaMemcpyHostToDevice));
    A(cudaMemcpy(h->act_d, act_all.data(), act_all.size() * sizeof(int), cudaMemcpyHostToDevice));
    A(cudaMemset(h->ictl, 0, 12 * sizeof(int)));
    A(cudaDeviceSynchronize());
  }
  if (!ok) {
    fprintf(stderr, "nmpc: setup allocation failed: %s\n", cudaGetErrorString(cudaGetLastError()));
    free_all(h);
    delete h;
    return NMPC_ERR_CUDA;
  }
  *out = h;
  return NMPC_OK;
}

int nmpc_solve(nmpc_handle* h, const double* x0, const double* ref, int horizon,
               const double* weights, int init, double* u_out, nmpc_stats* stats,
               void* stream) {
  if (!h || !x0 || !ref) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(h->x0_d, x0, h->n_g * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(load_ref(h, ref, cudaMemcpyDeviceToDevice, st));
  return solve_core(h, horizon, weights, init, u_out, stats, st);
}

int nmpc_solve_host(nmpc_handle* h, const double* x0, const double* ref, int horizon,
                    const double* weights, int init, double* u_out, nmpc_stats* stats,
                    void* stream) {
  if (!h || !x0 || !ref) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(h->x0_d, x0, h->n_g * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(load_ref(h, ref, cudaMemcpyHostToDevice, st));
  const double* wd = nullptr;
  if (weights) {
    CK(cudaMemcpyAsync(h->w_d, weights, 3 * h->n_inst * sizeof(double), cudaMemcpyHostToDevice, st));
    wd = h->w_d;
  }
  int rc = solve_core(h, horizon, wd, init, h->uo_d, stats, st);
  if (rc == NMPC_ERR_BAD_ARG || rc == NMPC_ERR_CUDA) return rc;
  if (u_out) {
    CK(cudaMemcpyAsync(u_out, h->uo_d, h->n_u * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return rc;
}

static int oneshot(nmpc_handle* h, const double* xi, const double* ui, const double* li,
                   double* xo, double* uo, double* lo, int resid_only, double* out_res,
                   cudaStream_t st) {
  if (h->strip2) {
    // k_strip2 moves x, lambda as 16-byte column pairs
    auto misaligned = [](const void* p) { return ((uintptr_t)p & 15u) != 0; };
    if (misaligned(xi) || misaligned(li) || misaligned(xo) || misaligned(lo))
      return NMPC_ERR_BAD_ARG;
  }
  IterArgs A = make_args(h);
  A.xin[0] = xi;
  A.uin[0] = ui;
  A.lin[0] = li;
  A.xout[1] = xo;
  A.uout[1] = uo;
  A.lout[1] = lo;
  A.res_first = nullptr;
  A.resid_only = resid_only;
  if (out_res) {
    CK(cudaMemsetAsync(h->res_inf, 0, h->n_inst * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(h->res_sq, 0, h->n_inst * sizeof(double), st));
  }
  // residual-only passes evaluate every stage at once
  if (resid_only) A.rb = 0;
  CK(launch_iterate<nmpc_dev::MODE_ONESHOT>(h, A, st, 0));
  if (A.rb) CK(launch_iterate<nmpc_dev::MODE_ONESHOT>(h, A, st, 1));
  if (out_res) {
    CK(cudaMemcpyAsync(h->h_resinf, h->res_inf, h->n_inst * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->h_res, h->res_sq, h->n_inst * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int b = 0; b < h->n_inst; ++b) {
      double r;
      std::memcpy(&r, &h->h_resinf[b], sizeof(double));
      out_res[2 * b] = r;
      out_res[2 * b + 1] = std::sqrt(h->h_res[b]);
    }
  }
  return NMPC_OK;
}

int nmpc_residual(nmpc_handle* h, const double* x0, const double* ref, const double* x,
                  const double* u, const double* lam, double* out, void* stream) {
  if (!h || !x0 || !ref || !x || !u || !lam || !out) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(h->x0_d, x0, h->n_g * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(load_ref(h, ref, cudaMemcpyDeviceToDevice, st));
  return oneshot(h, x, u, lam, nullptr, nullptr, nullptr, 1, out, st);
}

int nmpc_iterate(nmpc_handle* h, const double* x0, const double* ref, const double* x_in,
                 const double* u_in, const double* lam_in, double* x_out, double* u_out,
                 double* lam_out, int n_iter, double* out_res, void* stream) {
  if (!h || !x0 || !ref || !x_in || !u_in || !lam_in || !x_out || !u_out || !lam_out ||
      n_iter < 1)
    return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(h->x0_d, x0, h->n_g * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(load_ref(h, ref, cudaMemcpyDeviceToDevice, st));
  // ping-pong through the handle's A/B buffers, then copy out (so in and out
  // may alias)
  const double* xi = x_in;
  const double* ui = u_in;
  const double* li = lam_in;
  for (int it = 0; it < n_iter; ++it) {
    const bool lastit = (it == n_iter - 1);
    double* xo = h->xb[it & 1];
    double* uo = h->ub[it & 1];
    double* lo = h->lb[it & 1];
    int rc = oneshot(h, xi, ui, li, xo, uo, lo, 0, lastit ? out_res : nullptr, st);
    if (rc != NMPC_OK) return rc;
    xi = xo;
    ui = uo;
    li = lo;
  }
  CK(cudaMemcpyAsync(x_out, xi, h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(lam_out, li, h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(u_out, ui, h->n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return NMPC_OK;
}

int nmpc_plant_step(nmpc_handle* h, double* w, double dt, int n_sub, double* u_rec,
                    void* stream) {
  if (!h || !w || !(dt >= 0) || n_sub < 1 || !h->has_state) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // ping-pong through the handle's x0 staging buffer
  for (int k = 0; k < n_sub; ++k) {
    const bool even = (k % 2) == 0;
    const double* win = even ? w : h->x0_d;
    double* wout = even ? h->x0_d : w;
    nmpc_dev::k_plant_substep<<<dim3(32, h->n_inst), 256, 0, st>>>(
        h->inst_d, h->n_inst, h->act_d, win, wout, h->ub[2], (k == 0) ? u_rec : nullptr, dt,
        n_sub);
    h->launches++;
    CK(cudaGetLastError());
  }
  if (n_sub % 2 == 1)
    CK(cudaMemcpyAsync(w, h->x0_d, h->n_g * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return NMPC_OK;
}

int nmpc_closed_loop(nmpc_handle* h, double* w, const double* ref, int steps, int n_sub,
                     double* u_hist, int* iters_hist, double* res_hist, void* stream) {
  if (!h || !w || !ref || steps < 1 || n_sub < 1) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->opts.use_graph && !h->persistent) {
    CK(load_ref(h, ref, cudaMemcpyDeviceToDevice, st));
    return closed_loop_graph(h, w, steps, n_sub, u_hist, iters_hist, res_hist, st);
  }
  const int n = h->n_inst;
  std::vector<nmpc_stats> stats(n);
  int rc_all = NMPC_OK;
  for (int t = 0; t < steps; ++t) {
    // the measured plant state is the next problem's x0
    CK(cudaMemcpyAsync(h->x0_d, w, h->n_g * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(load_ref(h, ref, cudaMemcpyDeviceToDevice, st));
    int rc = solve_core(h, 0, nullptr, (t == 0 && !h->has_state) ? NMPC_INIT_COLD : NMPC_INIT_SHIFT,
                        nullptr, stats.data(), st);
    if (rc == NMPC_ERR_BAD_ARG || rc == NMPC_ERR_CUDA) return rc;
    if (rc != NMPC_OK && rc_all == NMPC_OK) rc_all = rc;
    for (int b = 0; b < n; ++b) {
      if (iters_hist) iters_hist[(size_t)t * n + b] = stats[b].iters;
      if (res_hist) res_hist[(size_t)t * n + b] = stats[b].res_inf;
    }
    // the plant moves one sampling period h under the first-stage controls
    int prc = nmpc_plant_step(h, w, 0.0, n_sub,
                              u_hist ? u_hist + (size_t)t * h->nu_tot : nullptr, stream);
    if (prc != NMPC_OK) return prc;
  }
  return rc_all;
}

int nmpc_start_state(nmpc_handle* h, int init, const double* x0, double* x, double* u,
                     double* lam, void* stream) {
  if (!h || !x || !u || !lam) return NMPC_ERR_BAD_ARG;
  if (init == NMPC_INIT_COLD) {
    if (!x0) return NMPC_ERR_BAD_ARG;
  } else if (init == NMPC_INIT_SHIFT) {
    if (!h->has_state) return NMPC_ERR_BAD_ARG;
    x0 = nullptr;
  } else {
    return NMPC_ERR_BAD_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  nmpc_dev::k_shift_state<<<per_instance_grid(h), 256, 0, st>>>(
      h->inst_d, h->n_inst, h->xb[2], h->ub[2], h->lb[2], x, u, lam, x0);
  h->launches++;
  CK(cudaGetLastError());
  return NMPC_OK;
}

int nmpc_rollout(nmpc_handle* h, const double* x0, const double* ref, const double* u, double* x,
                 double* lam, void* stream) {
  if (!h || !x0 || !ref || !u || !x || !lam) return NMPC_ERR_BAD_ARG;
  CK(enqueue_rollout(h, x0, ref, u, x, lam, (cudaStream_t)stream));
  return NMPC_OK;
}

int nmpc_rollout_fused(nmpc_handle* h, const double* x0, const double* ref, const double* u,
                       double* x, double* lam, void* stream) {
  if (!h || !x0 || !ref || !u || !x || !lam) return NMPC_ERR_BAD_ARG;
  // two stages of float32 recursion variable in shared memory when they fit
  const int cells = h->ng_max <= 12288 ? h->ng_max : 0;
  const size_t smem = 2 * (size_t)cells * sizeof(float);
  if (smem > 48 * 1024)
    CK(cudaFuncSetAttribute(nmpc_dev::k_rollout_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem));
  nmpc_dev::k_rollout_fused<<<h->n_inst, 1024, smem, (cudaStream_t)stream>>>(
      h->inst_d, h->n_inst, h->act_d, x0, ref, u, x, lam, cells);
  h->launches++;
  CK(cudaGetLastError());
  return NMPC_OK;
}

int nmpc_closed_loop_learned(nmpc_handle* h, double* w, const double* ref, int steps, int n_sub,
                             nmpc_start_fn start, void* ctx, const double* u_guess,
                             double* u_hist, int* iters_hist, double* res_hist, void* stream) {
  if (!h || !w || !ref || !start || !u_guess || steps < 1 || n_sub < 1) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(load_ref(h, ref, cudaMemcpyDeviceToDevice, st));
  if (h->opts.use_graph && !h->persistent)
    return closed_loop_graph(h, w, steps, n_sub, u_hist, iters_hist, res_hist, st, start, ctx,
                             u_guess);
  const int n = h->n_inst;
  std::vector<nmpc_stats> stats(n);
  int rc_all = NMPC_OK;
  for (int t = 0; t < steps; ++t) {
    CK(cudaMemcpyAsync(h->x0_d, w, h->n_g * sizeof(double), cudaMemcpyDeviceToDevice, st));
    start(ctx, stream);
    CK(cudaMemcpyAsync(h->ub[2], u_guess, h->n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(enqueue_rollout(h, h->x0_d, h->ref_d, h->ub[2], h->xb[2], h->lb[2], st));
    h->has_state = true;  // the guess is the handle's current state
    int rc = solve_core(h, 0, nullptr, NMPC_INIT_GUESS, nullptr, stats.data(), st);
    if (rc == NMPC_ERR_BAD_ARG || rc == NMPC_ERR_CUDA) return rc;
    if (rc != NMPC_OK && rc_all == NMPC_OK) rc_all = rc;
    for (int b = 0; b < n; ++b) {
      if (iters_hist) iters_hist[(size_t)t * n + b] = stats[b].iters;
      if (res_hist) res_hist[(size_t)t * n + b] = stats[b].res_inf;
    }
    int prc = nmpc_plant_step(h, w, 0.0, n_sub,
                              u_hist ? u_hist + (size_t)t * h->nu_tot : nullptr, stream);
    if (prc != NMPC_OK) return prc;
  }
  return rc_all;
}

int nmpc_get_state(nmpc_handle* h, double* x, double* u, double* lam, void* stream) {
  if (!h) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (x) CK(cudaMemcpyAsync(x, h->xb[2], h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (lam) CK(cudaMemcpyAsync(lam, h->lb[2], h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (u) CK(cudaMemcpyAsync(u, h->ub[2], h->n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return NMPC_OK;
}

int nmpc_set_state(nmpc_handle* h, const double* x, const double* u, const double* lam,
                   void* stream) {
  if (!h || !x || !u || !lam) return NMPC_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(h->xb[2], x, h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->lb[2], lam, h->n_s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->ub[2], u, h->n_u * sizeof(double), cudaMemcpyDeviceToDevice, st));
  h->has_state = true;
  return NMPC_OK;
}

int nmpc_sizes(const nmpc_handle* h, int64_t* out) {
  if (!h || !out) return NMPC_ERR_BAD_ARG;
  out[0] = h->n_g;
  out[1] = h->n_s;
  out[2] = h->n_u;
  return NMPC_OK;
}

int64_t nmpc_launch_count(const nmpc_handle* h) { return h ? h->launches : 0; }

int nmpc_strip_plan(const nmpc_handle* h, int64_t* out) {
  if (!h || !out) return NMPC_ERR_BAD_ARG;
  const bool on = h->n_strips > 0;
  out[0] = h->n_strips;
  out[1] = on ? h->strip_x : 0;
  out[2] = on ? h->strip_y : 0;
  out[3] = on ? h->strip_threads : 0;
  out[4] = on ? (int64_t)h->strip_smem : 0;
  out[5] = on ? h->n_patches : 0;
  out[6] = h->n_strip_inst;
  out[7] = on ? h->strip_region : 0;
  out[8] = on ? h->tail_y : 0;
  out[9] = on && h->tail_y > 0 ? h->tail_below : 0;
  return NMPC_OK;
}

int nmpc_launch_plan(const nmpc_handle* h, int64_t* out) {
  if (!h || !out) return NMPC_ERR_BAD_ARG;
  out[0] = h->threads;
  out[1] = h->csize;
  out[2] = h->cpt;
  out[3] = h->stage ? 1 : 0;
  out[4] = (h->persistent || h->line_persistent) ? 1 : 0;
  out[5] = (int64_t)h->smem;
  out[6] = h->grid;
  out[7] = h->local_u ? 1 : 0;
  out[8] = h->resident_clusters;
  out[9] = h->n_work;
  out[10] = h->iter_launches;
  return NMPC_OK;
}

int nmpc_line_plan(const nmpc_handle* h, int64_t* out) {
  if (!h || !out) return NMPC_ERR_BAD_ARG;
  const bool on = h->n_lines > 0;
  out[0] = h->n_lines;
  out[1] = h->n_line_inst;
  out[2] = on ? 32 * nmpc_dev::LINE_WARPS : 0;
  out[3] = on ? (int64_t)h->line_smem : 0;
  return NMPC_OK;
}

void nmpc_destroy(nmpc_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (auto& t : h->ev_pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto ev : h->ev_free) cudaEventDestroy(ev);
  free_all(h);
  delete h;
}

int nmpc_kernel_timing(nmpc_handle* h, int enable) {
  if (!h) return NMPC_ERR_BAD_ARG;
  CK(harvest_timing(h));
  for (int q = 0; q < 4; ++q) {
    h->kt_ms[q] = 0.0;
    h->kt_n[q] = 0;
  }
  h->timing = (enable != 0);
  return NMPC_OK;
}

int nmpc_kernel_times(nmpc_handle* h, int64_t* launches, double* ms) {
  if (!h || !launches || !ms) return NMPC_ERR_BAD_ARG;
  CK(harvest_timing(h));
  for (int q = 0; q < 4; ++q) {
    launches[q] = h->kt_n[q];
    ms[q] = h->kt_ms[q];
  }
  return NMPC_OK;
}

const char* nmpc_strerror(int code) {
  switch (code) {
    case NMPC_OK: return "ok";
    case NMPC_ERR_BAD_ARG: return "invalid argument";
    case NMPC_ERR_CUDA: return "CUDA runtime error";
    case NMPC_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case NMPC_ERR_DIVERGED: return "diverged (residual NaN/Inf or exploded)";
    case NMPC_ERR_NO_DEVICE: return "no CUDA device";
    case NMPC_ERR_UNSUPPORTED: return "size not supported";
    default: return "unknown error";
  }
}

}  // extern "C"

// ===========================================================================
// Allocation-free single-instance solve (nmpc_solve_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a
// solve: a real-time control loop that forbids allocation after start-up
// (allocation latency is unbounded), a process whose device memory is owned
// by another allocator or memory pool, or code running where cudaMalloc /
// cudaFree would synchronize the device.  This entry point needs no handle:
// its whole workspace (instance table, work list, the two ping-pong state
// copies, convergence control and, when a stage does not fit in shared
// memory, the lower-layer slab) lives in one file-scope device array of
// NMPC_NOALLOC_SCRATCH_BYTES.  Every GPU that loads this library keeps that
// array until the process exits.
//
// The host never dereferences the array's name: in host code it is only a
// stand-in symbol, so its device address is looked up with
// cudaGetSymbolAddress, once per device, with that device current, on the
// first call made on that device (that first call should therefore come
// before any stream capture).  Calls share the array and it keeps the last
// call's contents; the init kernel rewrites every part that must start from
// a known value (control counters, residual slots, the starting iterate).
// Two calls whose GPU work overlaps (different streams or threads on the same
// device) race on the array and corrupt each other's results.
// ===========================================================================
#include <mutex>

static __device__ __align__(256) unsigned char g_nmpc_noalloc_scratch[NMPC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of the static workspace on the current device; the first
// call on a device looks it up and sets the kernels' shared-memory limits.
int noalloc_workspace(void** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return NMPC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_nmpc_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "nmpc_solve_noalloc: cudaGetSymbolAddress failed: %s\n",
              cudaGetErrorString(e));
      return NMPC_ERR_CUDA;
    }
    int max_optin = 0;
    CK(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CK(configure_kernels<float>((size_t)max_optin));
    CK(configure_kernels<double>((size_t)max_optin));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return NMPC_OK;
}

size_t carve(size_t* off, size_t bytes) {
  const size_t at = *off;
  *off = (at + bytes + 255) & ~size_t(255);
  return at;
}

}  // namespace

extern "C" int nmpc_solve_noalloc(const nmpc_desc* desc, const nmpc_opts* opts,
                                  const double* x0, const double* ref, double* u_out,
                                  nmpc_stats* stats, void* stream) {
  if (!desc || !x0 || !ref || !u_out) return NMPC_ERR_BAD_ARG;
  int rc = validate(desc);
  if (rc != NMPC_OK) return rc;
  nmpc_opts o;
  nmpc_default_opts(&o);
  if (opts) o = *opts;
  if (!opts_ok(o)) return NMPC_ERR_BAD_ARG;
  // this entry point runs the cluster (or global-slab) path only: a forced
  // strip or line path cannot be honoured
  if (o.strips == 1 || o.lines == 1 || o.variant != NMPC_VARIANT_JACOBI)
    return NMPC_ERR_UNSUPPORTED;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return NMPC_ERR_NO_DEVICE;
  // per-device set-up first (the workspace address and the kernels'
  // shared-memory and cluster limits), so that the launch plan below sees
  // configured kernels on the first call in a process as on every later one
  void* base_v = nullptr;
  rc = noalloc_workspace(&base_v);
  if (rc != NMPC_OK) return rc;

  const nmpc_desc& d = *desc;
  const bool mixed = (o.precision == NMPC_MIXED);
  const int ng = d.mx * d.my, N = d.horizon, nu = d.n_u;
  const long long n_s = (long long)N * ng, n_u = (long long)N * nu;

  // launch configuration, chosen exactly as nmpc_setup chooses it
  int dev = 0, max_optin = 0, num_sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  InstDev I{};
  I.dim = d.dim;
  I.mx = d.mx;
  I.my = d.my;
  I.ng = ng;
  I.N = N;
  I.nu = nu;
  I.h = d.h;
  I.q = d.q;
  I.r = d.r;
  I.qf = d.qf;
  I.gamma = d.gamma;
  I.k0 = d.k0;
  I.k1 = d.k1;
  I.b0 = d.act_gain;
  const double dx = 1.0 / (d.mx + 1), dy = 1.0 / (d.my + 1);
  I.cx = 1.0 / (dx * dx);
  I.cy = (d.dim == 2) ? 1.0 / (dy * dy) : 0.0;
  nmpc_dev::derive(I);
  LaunchPlan P = plan_launch(&I, 1, N, o, mixed, std::max(1, num_sms), max_optin);
  const bool smem_mode = P.smem_mode;
  if (!smem_mode) P.grid = std::min(N, std::max(1, num_sms));
  const size_t elem = mixed ? sizeof(float) : sizeof(double);
  const long long slab = (long long)(((size_t)nmpc_dev::NUM_FIELDS * P.slab_max * elem +
                                      P.box_bytes + 255) & ~size_t(255));

  // workspace layout inside the static array
  size_t off = 0;
  const size_t o_inst = carve(&off, sizeof(InstDev));
  const size_t o_work = carve(&off, (size_t)N * sizeof(int2));
  const size_t o_act = carve(&off, (size_t)nu * sizeof(int));
  size_t o_x[2], o_l[2], o_u[2];
  for (int q = 0; q < 2; ++q) {
    o_x[q] = carve(&off, (size_t)n_s * sizeof(double));
    o_l[q] = carve(&off, (size_t)n_s * sizeof(double));
    o_u[q] = carve(&off, (size_t)n_u * sizeof(double));
  }
  const size_t o_ctl = carve(&off, 12 * sizeof(int));  // the handle's ictl layout
  const size_t o_rinf = carve(&off, nmpc_dev::RES_SLOTS * sizeof(unsigned long long));
  const size_t o_rerr = carve(&off, nmpc_dev::RES_SLOTS * sizeof(unsigned long long));
  const size_t o_rsq = carve(&off, nmpc_dev::RES_SLOTS * sizeof(double));
  const size_t o_f64 = carve(&off, 2 * sizeof(int));  // f64_count, full0
  const size_t o_rfirst = carve(&off, sizeof(unsigned long long));
  const size_t o_status = carve(&off, 3 * sizeof(int));  // status, iters, final_buf
  const size_t o_fin = carve(&off, 2 * sizeof(double));  // fin_inf, fin_2
  const size_t o_slab = carve(&off, smem_mode ? 0 : (size_t)slab * P.grid);
  if (off > (size_t)NMPC_NOALLOC_SCRATCH_BYTES) {
    fprintf(stderr,
            "nmpc_solve_noalloc: this instance needs %zu bytes of workspace; the static "
            "workspace holds %u bytes (use nmpc_setup/nmpc_solve for larger instances)\n",
            off, (unsigned)NMPC_NOALLOC_SCRATCH_BYTES);
    return NMPC_ERR_UNSUPPORTED;
  }
  char* base = static_cast<char*>(base_v);
  cudaStream_t st = (cudaStream_t)stream;

  // instance table, work list and actuator cells (pageable host copies are
  // staged by the runtime before cudaMemcpyAsync returns)
  CK(cudaMemcpyAsync(base + o_inst, &I, sizeof(InstDev), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + o_act, d.act_cell, nu * sizeof(int), cudaMemcpyHostToDevice, st));
  int2 chunk_buf[256];
  for (int s0 = 0; s0 < N; s0 += 256) {
    const int cnt = std::min(256, N - s0);
    for (int j = 0; j < cnt; ++j) chunk_buf[j] = make_int2(0, s0 + j);
    CK(cudaMemcpyAsync(base + o_work + (size_t)s0 * sizeof(int2), chunk_buf,
                       cnt * sizeof(int2), cudaMemcpyHostToDevice, st));
  }

  IterArgs A{};
  A.inst = reinterpret_cast<const InstDev*>(base + o_inst);
  A.work = reinterpret_cast<const int2*>(base + o_work);
  A.n_work = N;
  A.n_inst = 1;
  A.act = reinterpret_cast<const int*>(base + o_act);
  A.x0 = x0;
  A.ref = ref;
  for (int q = 0; q < 2; ++q) {
    A.xin[q] = A.xout[q] = reinterpret_cast<double*>(base + o_x[q]);
    A.lin[q] = A.lout[q] = reinterpret_cast<double*>(base + o_l[q]);
    A.uin[q] = A.uout[q] = reinterpret_cast<double*>(base + o_u[q]);
  }
  int* ctl = reinterpret_cast<int*>(base + o_ctl);
  A.iter_k = ctl + 0;
  A.n_active = ctl + 2;
  A.gsync = reinterpret_cast<unsigned*>(ctl + 4);
  A.res_inf = reinterpret_cast<unsigned long long*>(base + o_rinf);
  A.res_err = reinterpret_cast<unsigned long long*>(base + o_rerr);
  A.res_sq = reinterpret_cast<double*>(base + o_rsq);
  A.res_first = reinterpret_cast<unsigned long long*>(base + o_rfirst);
  int* stat = reinterpret_cast<int*>(base + o_status);
  A.status = stat + 0;
  A.iters = stat + 1;
  A.final_buf = stat + 2;
  double* fin = reinterpret_cast<double*>(base + o_fin);
  A.fin_inf = fin + 0;
  A.fin_2 = fin + 1;
  A.tol = o.tol;
  A.div_limit = o.div_limit;
  A.alpha = o.alpha;
  A.split_min = o.split_min;
  A.max_iter = o.max_iter;
  A.n_lo = o.n_lo;
  A.n_u_it = o.n_u_it;
  A.resid_only = 0;
  A.f64_count = reinterpret_cast<int*>(base + o_f64);
  A.full0 = A.f64_count + 1;
  A.full_all = mixed ? 0 : 1;
  A.csize = P.csize;
  A.slab_max = P.slab_max;
  A.stage = P.stage ? 1 : 0;
  A.local_u = P.local_u ? 1 : 0;
  A.box_r = P.box_r;
  A.scratch = smem_mode ? nullptr : base + o_slab;
  A.scratch_stride = slab;

  nmpc_dev::k_init_control<<<dim3(64, 1), 256, 0, st>>>(A, 0, 0, nullptr, nullptr, nullptr);
  CK(cudaGetLastError());
  long long launched = 0;
  int active = 1;
  while (launched <= o.max_iter) {
    for (int i = 0; i < o.check_every; ++i) {
      if (mixed)
        CK((launch_k<float>(P, A, st, nmpc_dev::MODE_SOLVE, i)));
      else
        CK((launch_k<double>(P, A, st, nmpc_dev::MODE_SOLVE, i)));
    }
    nmpc_dev::k_advance<<<1, 32, 0, st>>>(A.iter_k, o.check_every);
    CK(cudaGetLastError());
    launched += o.check_every;
    CK(cudaMemcpyAsync(&active, A.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (active == 0) break;
  }
  FinalArgs F{};
  F.inst = A.inst;
  F.n_inst = 1;
  for (int q = 0; q < 2; ++q) {
    F.xs[q] = A.xin[q];
    F.us[q] = A.uin[q];
    F.ls[q] = A.lin[q];
  }
  // the gathered iterate lands in buffer 0 (a copy onto itself when it is there)
  F.xc = A.xout[0];
  F.uc = A.uout[0];
  F.lc = A.lout[0];
  F.u_out = u_out;
  F.status = A.status;
  F.iters = A.iters;
  F.final_buf = A.final_buf;
  F.fin_inf = A.fin_inf;
  F.fin_2 = A.fin_2;
  F.res_inf = A.res_inf;
  F.res_sq = A.res_sq;
  F.tol = o.tol;
  F.max_iter = o.max_iter;
  nmpc_dev::k_finalize_status<<<1, 32, 0, st>>>(F);
  nmpc_dev::k_gather_final<<<dim3(64, 1), 256, 0, st>>>(F);
  CK(cudaGetLastError());
  int h_stat[3] = {0, 0, 0};
  int h_f64 = 0;
  double h_fin[2] = {0.0, 0.0};
  CK(cudaMemcpyAsync(h_stat, stat, sizeof(h_stat), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&h_f64, A.f64_count, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h_fin, fin, sizeof(h_fin), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (stats) {
    stats->status = h_stat[0];
    stats->iters = h_stat[1];
    stats->res_inf = h_fin[0];
    stats->res_2 = h_fin[1];
    stats->f64_iters = h_f64;
  }
  if (h_stat[0] == nmpc_dev::ST_DIVERGED) return NMPC_ERR_DIVERGED;
  if (h_stat[0] != nmpc_dev::ST_CONVERGED) return NMPC_ERR_NOT_CONVERGED;
  return NMPC_OK;
}
