/*
 * nmpc.h -- C ABI of the GB300 double-layer Jacobi NMPC solver.
 *
 * Method: H. Deng, T. Ohtsuka, "A Double-Layer Jacobi Method for
 * PDE-Constrained Nonlinear Model Predictive Control".
 *
 * Problem solved for each instance (Sec. 2-3 of the paper):
 *   model   w_t = div(k(w) grad w) + sum_a act_gain * u_a * [cell act_cell[a]]
 *           k(w) = k0 (1 + k1 w), interior grid of mx*my cells on [0,1]^dim
 *           with a Dirichlet-zero ring, 3-point (1D) / 5-point (2D)
 *           finite differences of the Kirchhoff form (Sec. 2, eq. 4);
 *   NLP     backward Euler x_i = x_{i-1} + h f(u_i, x_i), i = 1..N (eq. 6),
 *           cost sum_i h/2 (q|x_i - ref|^2 + r|u_i|^2) + h/2 qf|x_N - ref|^2,
 *           regularization gamma/2 |u_i - u_i^k|^2 (eq. 7, Remark 1);
 *   solve   K(S) = 0 for the KKT map of eq. 9 by the upper-layer Jacobi
 *           iteration S <- S - alpha D^{-1} K (eq. 15, all stages at once)
 *           with the lower-layer structured solve of each stage block
 *           (Sec. 4.3, eqs. 21-24; u fixed-point iteration of Sec. 5.2).
 *
 * Array layout ("packed"), for instances b = 0..n-1 in setup order, each
 * grid stored row-major (flat cell index iy*mx + ix), all float64:
 *   x0, ref   [sum_b ng_b]              ng_b = mx_b * my_b
 *   x, lam    [sum_b N_b * ng_b]        stage-major: stage i (1..N) at (i-1)*ng_b
 *   u         [sum_b N_b * n_u_b]       stage-major
 * Device pointers are plain CUDA device addresses (e.g. torch data_ptr()).
 * The caller owns every buffer it passes; the handle owns its workspace,
 * allocated in nmpc_setup and freed in nmpc_destroy.  Solves allocate
 * nothing.  All calls are asynchronous on `stream` (a cudaStream_t, NULL =
 * legacy default stream) except where stated.  Functions return NMPC_OK or a
 * negative NMPC_ERR_* code; no C++ exception crosses this interface.
 */
#ifndef NMPC_GB300_H
#define NMPC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NMPC_OK 0
#define NMPC_ERR_BAD_ARG (-1)       /* invalid argument or descriptor          */
#define NMPC_ERR_CUDA (-2)          /* a CUDA runtime call failed              */
#define NMPC_ERR_NOT_CONVERGED (-3) /* max_iter reached above tol              */
#define NMPC_ERR_DIVERGED (-4)      /* residual became NaN/Inf or exploded     */
#define NMPC_ERR_NO_DEVICE (-5)     /* no usable CUDA device                   */
#define NMPC_ERR_UNSUPPORTED (-6)   /* size beyond what the kernels support    */

#define NMPC_FP64 0  /* all arithmetic in float64                              */
#define NMPC_MIXED 1 /* lower layer (Sec. 4.3) in float32; KKT residual, norms,
                        convergence test and the update of S in float64       */

#define NMPC_VARIANT_JACOBI 0   /* upper layer: Jacobi, eq. 15 (all stages from
                                   iterate k)                                  */
#define NMPC_VARIANT_REDBLACK 1 /* upper layer: block Gauss-Seidel (the form of
                                   eq. 18, (D + L)^{-1} K) in the red-black stage
                                   order: even 0-based stages from iterate k,
                                   then odd stages with their neighbours'
                                   updated x_{i-1}, lambda_{i+1}.  The KKT
                                   matrix is block tridiagonal, so this order is
                                   consistent and the factor is the Jacobi one
                                   squared (Theorem 3); both halves are
                                   stage-parallel launches                     */

#define NMPC_INIT_COLD 0 /* S^0: x_i = x0, u_i = 0, lambda_i = 0              */
#define NMPC_INIT_WARM 1 /* S^0 = the handle's current state (last solution or
                            a state set by nmpc_set_state); in NMPC_MIXED the
                            first iteration evaluates the float64 residual, so
                            an already converged state returns at once        */
#define NMPC_INIT_GUESS 2 /* as WARM, for a state that is only a guess (e.g.
                            the learned warm start): no float64 first residual */
#define NMPC_INIT_SHIFT 3 /* receding horizon: the current state shifted by one
                            stage, (s_2, ..., s_N, s_N)                        */

/* Per-instance status in nmpc_stats.status */
#define NMPC_STATUS_CONVERGED 1
#define NMPC_STATUS_DIVERGED 2
#define NMPC_STATUS_MAX_ITER 3

/* One NMPC instance.  act_cell is a host pointer read during nmpc_setup only. */
typedef struct {
  int dim;             /* 1 or 2                                              */
  int mx, my;          /* interior cells per axis (my = 1 when dim == 1)      */
  int horizon;         /* N >= 1 stages                                       */
  int n_u;             /* actuators, 1..NMPC_MAX_NU                           */
  const int* act_cell; /* [n_u] flat cell indices, 0 <= c < mx*my             */
  double h;            /* stage length T/N                                    */
  double q, r, qf;     /* Q = q I, R = r I, terminal Qf = qf I                */
  double gamma;        /* regularization weight (> 0 in practice, Thm 2)      */
  double k0, k1;       /* k(w) = k0 (1 + k1 w)                                */
  double act_gain;     /* heating rate of an actuator cell per unit input     */
} nmpc_desc;

#define NMPC_MAX_NU 64
#define NMPC_MAX_NG (1 << 20)

/* Iteration options; nmpc_default_opts fills the paper's settings
   (two lower-layer Jacobi sweeps and two u-iterations, Table 2 / Sec. 5.2). */
typedef struct {
  double tol;      /* stop once ||K(S^k)||_inf <= tol (float64 norm)          */
  int max_iter;    /* upper-layer iterations before NMPC_STATUS_MAX_ITER      */
  int n_lo;        /* pointwise Jacobi sweeps per F_x and F_x^T solve (>= 1)  */
  int n_u_it;      /* fixed-point iterations for Delta u (>= 1)               */
  int precision;   /* NMPC_FP64 or NMPC_MIXED                                 */
  int check_every; /* iterations between host polls of the convergence count  */
  double alpha;    /* step length in (0, 1]                                   */
  double div_limit;/* residual above div_limit * ||K(S^0)||_inf => diverged   */
  int threads;     /* threads per CTA (multiple of 32, <= 512); 0 = auto      */
  int use_graph;   /* capture the iteration chunk in a CUDA graph (1) or not  */
  int cluster;     /* CTAs per stage (1..8 or 16, a thread-block cluster that
                      splits the stage grid); 0 = auto                        */
  double split_min;/* NMPC_MIXED: iterations evaluate K with float64
                      differences and float32 O(h) terms (the split residual,
                      with a computed bound e on its rounding error); the
                      float64 residual is evaluated in the iteration after
                      one whose residual r (split or float64) was at or
                      below T = max(tol, split_min), or after a split
                      residual with r - e <= T that is no lower than 12
                      iterations before (its rounding floor above T).  A
                      float64 residual above T hands back to the split
                      residual when the split residual had itself reached T
                      or it was iteration 0's; otherwise the float64
                      residual stays.  Convergence is only ever declared on
                      a float64 residual.  Handles with strip-path instances
                      use max(split_min, 1e-6): their split residual takes
                      the stage differences from float32 values        */
  int u_local;     /* 1: the u-iteration uses the actuators' local responses
                      (P^{-1} is a fixed linear map, so Y(v3) = Y(0) + sum_b
                      v3_b Z(e_b) with Z(e_b) zero outside 2(n_lo-1) cells of
                      actuator b; one full-field P^{-1} per iteration) when
                      n_lo <= 4 and the boxes fit; 0: n_u_it + 1 full-field
                      P^{-1} applications in the paper's literal order        */
  int cells;       /* target cells per thread (1..8) when threads is auto:
                      each thread carries its cells through every pass of a
                      work item as independent dependency chains; 0 = auto
                      (4)                                                     */
  int persistent;  /* 1: one launch runs the whole solve with device-wide
                      barriers between iterations (bounded waits; a wait
                      that runs out restarts the solve with one launch per
                      iteration): on the cluster path when one cluster per
                      stage fits on the device at once (staged slabs), on
                      the line path when every stage of the handle is on it
                      (the resident warps walk the line list every
                      iteration); Jacobi upper layer only.  The iterates
                      are identical to those of 0 (one launch per
                      iteration, the default) on the cluster path, equal to
                      float32 rounding on the line path                    */
  int strips;       /* 2D instances on the strip path: each warp computes a
                      strip of 32 - 2E own columns (E = 2 n_lo - 1) from a
                      region extended by E cells, walking down its rows with
                      every lower-layer pass pipelined in registers
                      (redundant border work instead of cluster exchanges);
                      actuator controls v3 from patches around the
                      actuators.  0 = auto (stages too large for a cluster of
                      <= 8 CTAs with staged inputs), 1 = every eligible 2D
                      instance, 2 = never.  Eligible: n_lo <= 4, and for
                      n_u_it > 1 no two actuators on one cell or within
                      2 (n_lo - 1) cells (Manhattan) of each other          */
  int strip_rows;   /* own rows per strip (0..65535); 0 = auto (whole columns
                      when the batch gives enough strips, else shorter
                      strips, at least 16 rows)                             */
  int lines;        /* NMPC_MIXED 1D instances of at most 256 cells on the
                      line path: one warp per stage, the stage's cells in
                      registers (8 per lane at most), every pass of the
                      iteration without a block barrier; full-field
                      u-iteration (u_local does not apply there).
                      0 = auto (every such instance), 1 = the same,
                      2 = never (cluster path)                              */
  int variant;      /* NMPC_VARIANT_JACOBI (default) or NMPC_VARIANT_REDBLACK:
                      two stage-parallel launches per iteration (half 0: even
                      stages, half 1: odd stages); convergence is still
                      declared on the float64 ||K(S^k)||_inf of whole
                      iterates.  On the strip path the NMPC_MIXED split-form
                      iterations before it (whose norms only trigger the
                      float64 residual) take at odd stages the Gauss-Seidel
                      residual, K_i with the neighbours updated by half 0;
                      nmpc_iterate keeps the norms of K(S^k).  Requires
                      alpha = 1 (BAD_ARG otherwise) and never runs the
                      persistent launch                                     */
  int64_t barrier_wait_cycles; /* persistent launch: spin budget of one grid-
                      barrier wait in SM clock cycles (0 = 4e9, about two
                      seconds).  A wait that runs out ends the launch with an
                      error word; the host then discards that launch's state
                      and solves from S^0 with one launch per iteration (the
                      handle keeps that mode).  A tiny budget exercises this
                      path                                                  */
  int strip_cols;   /* grid columns per lane on the strip path: 0 = auto (two
                      where NMPC_MIXED, n_lo <= 2 and every strip instance
                      has an even grid width and even array offsets: 64-column
                      regions with 64 - 4 n_lo own columns, packed float32
                      pairs; else one), 1 = one (32-column regions)         */
  int tail_rows;    /* two-column strip path, solves: own rows of a second,
                      finer strip plan taken by the launches of a batch's
                      tail, when at most tail_below instances still run
                      (more warps per instance: a few running instances'
                      strips no longer leave the GPU latency-bound).  0 =
                      auto (64 where the main plan's rows are >= 256, else
                      none), -1 = none, else 8..65535                      */
  int tail_below;   /* running instances at or below which a launch takes the
                      tail plan: 0 = auto (those whose main-plan strips fill
                      fewer than six waves of resident warps), else >= 1   */
} nmpc_opts;

typedef struct {
  int iters;      /* index k of the returned iterate S^k                       */
  int status;     /* NMPC_STATUS_*                                            */
  double res_inf; /* ||K(S^k)||_inf (float64)                                 */
  double res_2;   /* ||K(S^k)||_2                                             */
  int f64_iters;  /* iterations 0..k that evaluated the float64 residual (every
                     one in NMPC_FP64; in NMPC_MIXED see split_min)         */
} nmpc_stats;

typedef struct nmpc_handle nmpc_handle;

/* Fill *o with defaults: tol 1e-6, max_iter 2000, n_lo 2, n_u_it 2, FP64,
   check_every 16, alpha 1, div_limit 1e8, threads auto, graph on, cluster
   auto, split_min 1e-7, u_local 0, cells auto, persistent 0, strips auto,
   strip_rows auto, lines auto, variant Jacobi, barrier_wait_cycles 0,
   strip_cols auto, tail_rows auto, tail_below auto. */
void nmpc_default_opts(nmpc_opts* o);

/* Validate the descriptors, build the device instance table and allocate the
   workspace on the current CUDA device.  An instance is the discretized
   problem of Sec. 2 (eq. 4, a first-order model: a = 0 in eq. 1) posed as
   the N-stage NLP of eq. 6; the workspace holds the primal-dual iterates
   S = (s_1, ..., s_N), s_i = (x_i, u_i, lambda_i) of Sec. 3.2, twice (the
   iterates k and k + 1 of eq. 15) plus the handle's current state.  On success *out owns everything;
   release it with nmpc_destroy.  Errors: BAD_ARG (a descriptor field out of
   range, NULL pointers), UNSUPPORTED (n_u > NMPC_MAX_NU, ng > NMPC_MAX_NG),
   NO_DEVICE, CUDA.  Synchronous. */
int nmpc_setup(const nmpc_desc* descs, int n_instances, const nmpc_opts* opts,
               nmpc_handle** out);

/* Solve every instance from x0 (packed [sum ng], device) tracking ref
   (packed [sum ng], device): the KKT system K(S) = 0 of eq. 9 by the
   upper-layer iteration of eq. 15 (every stage's Delta s_i from iterate k,
   each by the lower-layer solve of Sec. 4.3, eqs. 21-24, with the
   u-iteration of Sec. 5.2), stopped by the rule of Table 2 with the
   threshold opts.tol: ||K(S^k)||_inf <= tol, evaluated in float64.  horizon: 0 = each instance's own N; only 0 or a
   value equal to every instance's N is accepted (BAD_ARG otherwise).
   weights: NULL, or device [n_instances][3] = (q, r, qf) overriding the
   descriptors for this and later solves.  init: NMPC_INIT_COLD / _WARM / _GUESS.
   u_out: device packed u of the returned iterates.  stats: host
   [n_instances], written before return (the call synchronizes on stream).
   Returns NMPC_OK when every instance converged, else the first of
   NOT_CONVERGED / DIVERGED met; stats are filled in either case. */
int nmpc_solve(nmpc_handle* h, const double* x0, const double* ref, int horizon,
               const double* weights, int init, double* u_out, nmpc_stats* stats,
               void* stream);

/* As nmpc_solve, but x0, ref, weights and u_out are HOST pointers; the
   host-device copies run on `stream` inside the call. */
int nmpc_solve_host(nmpc_handle* h, const double* x0, const double* ref, int horizon,
                    const double* weights, int init, double* u_out, nmpc_stats* stats,
                    void* stream);

/* Float64 KKT residual (eq. 9, u~ = u) of the state (x, u, lam) (packed,
   device) for initial states x0 and references ref (device).  out: host
   [n_instances][2] = (||K_b||_inf, ||K_b||_2).  Synchronizes on stream.
   When the handle runs its strip path with two columns per lane
   (nmpc_opts.strip_cols), x and lam must be 16-byte aligned (BAD_ARG
   otherwise); the same holds for nmpc_iterate's x and lam arrays. */
int nmpc_residual(nmpc_handle* h, const double* x0, const double* ref, const double* x,
                  const double* u, const double* lam, double* out, void* stream);

/* n_iter >= 1 plain upper-layer iterations (eq. 15) from (x_in, u_in,
   lam_in) to (x_out, u_out, lam_out), all packed device arrays, with no
   convergence test (the handle's ping-pong buffers hold the intermediate
   iterates, so in and out may alias).  out_res: NULL or host
   [n_instances][2], the norms of K at the last input iterate S^{n_iter-1}.
   Synchronizes on stream when out_res is given. */
int nmpc_iterate(nmpc_handle* h, const double* x0, const double* ref, const double* x_in,
                 const double* u_in, const double* lam_in, double* x_out, double* u_out,
                 double* lam_out, int n_iter, double* out_res, void* stream);

/* Plant simulator for the closed loop: advance the true system w (device
   [sum ng], in place) by dt (dt = 0: each instance's own stage length h)
   under the first-stage controls u_1 of the current solution, with n_sub
   explicit-Euler sub-steps of the same finite-difference model,
   w += (dt/n_sub) (Lap Phi(w) + act_gain B u_1).  Explicit Euler is
   stable for (dt/n_sub) k_max 2 (1/dx^2 + 1/dy^2) <= 1.  u_rec: NULL or device
   [sum n_u], receives u_1.  Requires a solved state. */
int nmpc_plant_step(nmpc_handle* h, double* w, double dt, int n_sub, double* u_rec,
                    void* stream);

/* Receding-horizon closed loop (the paper's Sec. 5.3 use): for each of
   `steps` sampling periods, solve with x0 = w (the first from the cold start
   unless the handle holds a state, then from the shifted previous solution,
   NMPC_INIT_SHIFT), apply u_1 to the plant for one stage length h
   (nmpc_plant_step with n_sub sub-steps).  w: device [sum ng] plant state,
   in/out; ref: device [sum ng]; u_hist: NULL or device [steps][sum n_u];
   iters_hist, res_hist: NULL or host [steps][n_instances].  Returns the first
   non-OK solve status met (the loop continues through it). */
int nmpc_closed_loop(nmpc_handle* h, double* w, const double* ref, int steps, int n_sub,
                     double* u_hist, int* iters_hist, double* res_hist, void* stream);

/* A start iterate S^0 written to packed device arrays x, lam [sum N*ng] and
   u [sum N*n_u] (caller-owned, not aliasing the handle's buffers), so that a
   caller can compare or modify candidate starts (for instance by their
   nmpc_residual) before nmpc_set_state + NMPC_INIT_GUESS:
   init = NMPC_INIT_COLD: x_i = x0 (device [sum ng]), u = 0, lambda = 0;
   init = NMPC_INIT_SHIFT: the receding-horizon shift of the handle's current
   state (Sec. 5.3's closed loop; stage i takes stage i + 1, the last stage
   is repeated; x0 is ignored).  NMPC_ERR_BAD_ARG for another init, a NULL
   array, a NULL x0 with COLD, or SHIFT without a solved state. */
int nmpc_start_state(nmpc_handle* h, int init, const double* x0, double* x, double* u,
                     double* lam, void* stream);

/* State and costate trajectories of a control trajectory u (device
   [sum N*n_u]) from x0, ref (device [sum ng]): x_i = x_{i-1} + h (Lap Phi
   (x_{i-1}) + b0 B u_i) forward (the model of eq. 6 stepped explicitly,
   stable while h k(w) 2 (1/dx^2 + 1/dy^2) <= 1), then backward from
   lambda_{N+1} = h qf (x_N - ref): lambda_i = lambda_{i+1} + h (q (x_i - ref)
   + Phi'(x_i) Lap lambda_{i+1}) (the costate rows of eq. 9 with the coupling
   taken at the later stage).  Written to device x, lam [sum N*ng]: a start
   consistent with u to O(h^2) per stage for NMPC_INIT_GUESS (no counterpart
   in the paper; it completes a control-only guess such as a learned one).
   Float64 arithmetic on NMPC_FP64 handles; float32 arithmetic from the
   float64 inputs truncated to float32 (stores float64) on NMPC_MIXED ones,
   for start guesses.  2 N launches; NMPC_ERR_BAD_ARG for a NULL array. */
int nmpc_rollout(nmpc_handle* h, const double* x0, const double* ref, const double* u, double* x,
                 double* lam, void* stream);

/* nmpc_rollout in one launch with float32 arithmetic (stores float64): one
   CTA per instance walks the stages with a block barrier between them.  For
   start guesses, where the launch count of the per-stage form dominates (a
   few hundred microseconds of launches against tens of microseconds of
   work on small grids).  Same arguments and errors as nmpc_rollout. */
int nmpc_rollout_fused(nmpc_handle* h, const double* x0, const double* ref, const double* u,
                       double* x, double* lam, void* stream);

/* Step start of nmpc_closed_loop_learned, supplied by the caller: enqueue on
   `stream` the work that writes a control trajectory guess (device float64,
   [sum N n_u], the packing of u) into the caller's u_guess buffer, reading
   the plant state in the caller's w buffer.  Kernel launches only (no
   synchronisation, allocation or host copies): with the graph loop the calls
   are captured, once, and replayed every step. */
typedef void (*nmpc_start_fn)(void* ctx, void* stream);

/* nmpc_closed_loop with a learned start (no counterpart in the paper; the
   controls come from a network, e.g. on pooled plant state and reference):
   each step copies w into x0, runs start(ctx, stream), completes the guess
   u_guess with its state and costate trajectories (nmpc_rollout) and solves
   from that start (NMPC_INIT_GUESS); then the plant moves as in
   nmpc_closed_loop.  With opts.use_graph (and no persistent launch) the whole
   loop, the start's kernels included, is one CUDA graph.  Histories and
   return codes as nmpc_closed_loop; NMPC_ERR_BAD_ARG for a NULL h, w, ref,
   start or u_guess, steps < 1 or n_sub < 1. */
int nmpc_closed_loop_learned(nmpc_handle* h, double* w, const double* ref, int steps, int n_sub,
                             nmpc_start_fn start, void* ctx, const double* u_guess,
                             double* u_hist, int* iters_hist, double* res_hist, void* stream);

/* Copy the handle's current state (after a solve: the returned iterates
   S^k = (x_i, u_i, lambda_i), i = 1..N, the primal-dual variables of
   Sec. 3.2) to packed device arrays x, u, lam; any pointer may be NULL to
   skip it. */
int nmpc_get_state(nmpc_handle* h, double* x, double* u, double* lam, void* stream);

/* Replace the handle's current state (the NMPC_INIT_WARM start). */
int nmpc_set_state(nmpc_handle* h, const double* x, const double* u, const double* lam,
                   void* stream);

/* Sizes of the packed arrays: out[0] = sum ng, out[1] = sum N*ng,
   out[2] = sum N*n_u. */
int nmpc_sizes(const nmpc_handle* h, int64_t* out);

/* Number of kernel launches issued by this handle since setup (all entry
   points), for launch accounting. */
int64_t nmpc_launch_count(const nmpc_handle* h);

/* The launch plan the handle chose (no counterpart in the paper; for tuning
   and diagnostics): out[0] threads per CTA, out[1] CTAs per stage (cluster
   size), out[2] cells per thread, out[3] 1 if the float64 inputs are staged
   in shared memory, out[4] 1 if one persistent launch runs each solve,
   out[5] dynamic shared memory bytes per CTA, out[6] CTAs per iteration
   launch, out[7] 1 if the u-iteration uses local responses, out[8] clusters
   of this shape the device keeps resident at once for the persistent
   launch, out[9] work items (instance stages) on the cluster path (the
   strip path's are in nmpc_strip_plan, the line path's in nmpc_line_plan),
   out[10] iteration steps launched
   (one per iteration, whichever kernels it takes; one per solve when
   persistent) since setup.  Returns NMPC_ERR_BAD_ARG for a null handle or array. */
int nmpc_launch_plan(const nmpc_handle* h, int64_t* out);

/* Strip path of the handle (opts.strips): out[0] strips per iteration (work
   items of k_strip, one warp each), out[1] own columns and out[2] own rows
   per strip, out[3] threads per CTA, out[4] dynamic shared memory per CTA
   (bytes), out[5] actuator patches per iteration (k_patch work items, one
   warp each), out[6] instances on the strip path, out[7] cells of a
   strip's extended region, out[8] own rows of the tail plan's strips (0:
   none), out[9] running instances at or below which solve launches take
   it.  All zero when no instance is on the strip path.  NMPC_ERR_BAD_ARG
   for NULL arguments. */
int nmpc_strip_plan(const nmpc_handle* h, int64_t* out);

/* Per-kernel device timing (no counterpart in the paper; for measurement):
   with enable != 0, every later launch of the iteration kernels that is not
   being captured into a CUDA graph is bracketed by a CUDA event pair on its
   stream (which also stops consecutive launches from overlapping their
   start and end, so each pair times its kernel alone); enable = 0 stops
   recording.  Either call clears the totals.  Solves with opts.use_graph
   run their iterations inside a graph and are not timed: use use_graph = 0
   for timed runs.  Synchronizes on the recorded events.  BAD_ARG for a NULL
   handle. */
int nmpc_kernel_timing(nmpc_handle* h, int enable);

/* Totals since the last nmpc_kernel_timing call, per kernel kind k = 0
   cluster-path iteration kernel (k_iterate), 1 actuator patches (k_patch),
   2 strips (k_strip), 3 lines (k_line): launches[k] timed launches and
   ms[k] their summed device time in milliseconds.  Waits for the recorded
   events.  BAD_ARG for NULL arguments. */
int nmpc_kernel_times(nmpc_handle* h, int64_t* launches, double* ms);

/* Line path of the handle (opts.lines): out[0] line work items per
   iteration (one warp each: an (instance, stage) of a 1D instance), out[1]
   instances on the line path, out[2] threads per CTA, out[3] dynamic shared
   memory per CTA (bytes).  All zero when no instance is on the line path.
   NMPC_ERR_BAD_ARG for NULL arguments. */
int nmpc_line_plan(const nmpc_handle* h, int64_t* out);

/* Allocation-free solve of ONE instance (no counterpart in the paper; it
   exists for callers that may not allocate device memory when they solve:
   a real-time control loop that forbids allocation after start-up, code
   whose device memory belongs to another allocator or pool, or code that
   must not trigger the device-wide synchronization of cudaMalloc/cudaFree).
   No handle is needed and nothing is allocated: the workspace is a static
   device array of NMPC_NOALLOC_SCRATCH_BYTES inside this library, which every
   GPU that loads the library holds until the process exits.  The first call
   on a device looks up that array's device address (make that first call
   before any stream capture).  desc: the instance (act_cell is read during
   the call); opts: NULL for defaults; x0, ref: device [mx*my]; u_out: device
   [horizon*n_u]; stats: host, one entry.  It always runs the cluster path
   (one thread-block cluster per stage, or one CTA per stage over a slab in
   the static array when a stage does not fit a cluster), never the strip or
   line path: opts.strips and opts.lines must be 0 or 2 (1, forcing one of
   those paths, returns UNSUPPORTED); opts.strip_rows, opts.persistent and
   opts.use_graph are ignored (the iterations are launched from the host in
   chunks of check_every).  opts.variant must be NMPC_VARIANT_JACOBI
   (UNSUPPORTED otherwise).  Returns UNSUPPORTED (and prints the
   needed size) when the instance's workspace exceeds the static array,
   otherwise as nmpc_solve.  Every call reuses the same array, and the call
   resets whatever must start from zero; calls whose GPU work overlaps (other
   streams or threads on the same device) race on it and corrupt each other's
   results.  Synchronizes on stream. */
#define NMPC_NOALLOC_SCRATCH_BYTES (32u << 20)
int nmpc_solve_noalloc(const nmpc_desc* desc, const nmpc_opts* opts, const double* x0,
                       const double* ref, double* u_out, nmpc_stats* stats, void* stream);

/* Free the workspace and the handle (NULL is a no-op).  Synchronizes. */
void nmpc_destroy(nmpc_handle* h);

/* Static string for an NMPC_* code. */
const char* nmpc_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* NMPC_GB300_H */
