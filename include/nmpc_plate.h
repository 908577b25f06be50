/*
 * nmpc_plate.h -- C ABI of the pinned-actuator solver: the double-layer
 * method on the paper's own problem class (Sec. 5.1, Tables 1-2), a heat
 * plate whose actuator points have their temperatures set directly.
 *
 * Problem per instance (Sec. 2 eq. 1 with a = 0; Sec. 3 eqs. 6-8):
 *   grid    dim = 1 or 2, m points per axis; bc 0: zero Neumann, the points
 *           include the boundary (spacing 1/(m-1)), mirrored fictitious
 *           points (eqs. 2-3); bc 1: zero Dirichlet, interior points
 *           (spacing 1/(m+1));
 *   inputs  the temperatures of the n_u points act_cell (not states): the
 *           state x holds the other n_s = m^dim - n_u points, in grid order;
 *   model   w_t = Lap Phi(w) - beta (w - t_amb) - gamma_r (w^4 - t_amb^4),
 *           Phi(w) = k0 (w + k1 w^2 / 2), with w = x at the state points
 *           and w = u at the actuator points;
 *   NLP     backward Euler x_i = x_{i-1} + h f(u_i, x_i); stage cost
 *           h (q/2 |x - x_ref|^2 + r/2 |u - u_ref|^2 + Phi_b(u)) with the
 *           log barrier Phi_b(u) = -tau sum(ln(u - u_lo) + ln(u_hi - u))
 *           (tau = 0: no bounds), terminal h qf/2 |x_N - x_ref|^2,
 *           regularization gamma/2 |u_i - u_i^k|^2 (Remark 1);
 *   solve   K(S) = 0 of eq. 9 by the upper-layer Jacobi iteration (eq. 15)
 *           or its red-black Gauss-Seidel form (eq. 18 in the even-then-odd
 *           stage order), each stage by the lower layer (Sec. 4.3, eqs.
 *           21-24; u-iteration of Sec. 5.2), step alpha_max of the
 *           fraction-to-the-boundary rule (eq. 11: G(u^{k+1}) >= 0.005 G(u^k)
 *           for both bounds of every input of every stage), until
 *           ||K(S^k)||_inf <= tol (Table 2's rule).
 * Arrays, packed per instance in setup order, float64, device pointers:
 *   x0, x_ref [sum n_s]; u_ref [sum n_u];
 *   x, lam [sum N n_s] stage-major; u [sum N n_u] stage-major.
 * Arithmetic: float64, or with NMPC_MIXED a float32 lower layer.  The
 * caller owns its buffers; the handle owns its workspace (allocated in
 * setup, freed in destroy); solves allocate nothing.  Return codes are the
 * NMPC_* codes of nmpc.h.
 */
#ifndef NMPC_GB300_PLATE_H
#define NMPC_GB300_PLATE_H

#include <stdint.h>

#include "nmpc.h"

#ifdef __cplusplus
extern "C" {
#endif

#define NMPC_PLATE_MAX_POINTS 1024 /* grid points of one instance          */

typedef struct {
  int dim;             /* 1 or 2                                              */
  int m;               /* grid points per axis                                */
  int bc;              /* 0 zero Neumann (boundary points included), 1 zero Dirichlet */
  int horizon;         /* N >= 1                                              */
  int n_u;             /* pinned actuator points, 1..NMPC_MAX_NU              */
  const int* act_cell; /* [n_u] grid point indices (host, read in setup)      */
  double h;            /* stage length                                        */
  double k0, k1;       /* Phi(w) = k0 (w + k1 w^2 / 2)                        */
  double beta, t_amb;  /* convection: -beta (w - t_amb)                       */
  double gamma_r;      /* radiation: -gamma_r (w^4 - t_amb^4)                 */
  double q, r, qf;     /* weights                                             */
  double gamma;        /* regularization (> 0)                                */
  double tau;          /* barrier weight; 0 = no input bounds                 */
  double u_lo, u_hi;   /* input bounds (used when tau > 0)                    */
} nmpc_plate_desc;

typedef struct {
  double tol;       /* stop at ||K(S^k)||_inf <= tol                         */
  int max_iter;     /* iterations before NMPC_STATUS_MAX_ITER                */
  int n_lo;         /* Jacobi sweeps per F_x, F_x^T solve (Table 2: 2)       */
  int n_u_it;       /* u fixed-point iterations (Sec. 5.2: 2)                */
  int variant;      /* NMPC_VARIANT_JACOBI or NMPC_VARIANT_REDBLACK           */
  int check_every;  /* iterations between host polls of the running count    */
  int precision;    /* NMPC_FP64 (default), or NMPC_MIXED: the lower layer's
                       sweeps and u-iteration in float32 against the float64
                       residual, coefficients and update (the root is the
                       float64 root)                                         */
} nmpc_plate_opts;

typedef struct nmpc_plate nmpc_plate;

/* Defaults: tol 1e-6, max_iter 5000, n_lo 2, n_u_it 2, Jacobi, check_every 16,
   NMPC_FP64. */
void nmpc_plate_default_opts(nmpc_plate_opts* o);

/* Validate the descriptors (BAD_ARG: dims, bounds, tau > 0 with u_lo >= u_hi,
   actuator indices out of the grid or repeated; UNSUPPORTED: more than
   NMPC_PLATE_MAX_POINTS points or NMPC_MAX_NU inputs), build the stencil
   tables and allocate the workspace on the current device.  Synchronous. */
int nmpc_plate_setup(const nmpc_plate_desc* descs, int n_instances, const nmpc_plate_opts* opts,
                     nmpc_plate** out);

/* out[0] = sum n_s, out[1] = sum N n_s, out[2] = sum N n_u, out[3] = sum n_u. */
int nmpc_plate_sizes(const nmpc_plate* h, int64_t* out);

/* Solve every instance from x0 tracking (x_ref, u_ref) (device).  init:
   NMPC_INIT_COLD (x_i = x0; u_i = (u_lo + u_hi)/2 with bounds, else 0;
   lambda = 0), NMPC_INIT_WARM (the handle's current state) or
   NMPC_INIT_SHIFT (the current state shifted by one stage, the last one
   repeated).  u_out: device [sum N n_u] or NULL; stats: host [n].
   Synchronizes.  NMPC_OK when every instance converged, else the first of
   NOT_CONVERGED / DIVERGED met. */
int nmpc_plate_solve(nmpc_plate* h, const double* x0, const double* x_ref, const double* u_ref,
                     int init, double* u_out, nmpc_stats* stats, void* stream);

/* n_iter >= 1 iterations (with alpha_max, no convergence test) from
   (x_in, u_in, lam_in) into (x_out, u_out, lam_out), device packed arrays
   (in and out may alias).  out: NULL or host [n][3] = (||K||_inf, ||K||_2,
   alpha) of the last iteration.  Synchronizes when out is given. */
int nmpc_plate_iterate(nmpc_plate* h, const double* x0, const double* x_ref, const double* u_ref,
                       const double* x_in, const double* u_in, const double* lam_in,
                       double* x_out, double* u_out, double* lam_out, int n_iter, double* out,
                       void* stream);

/* The handle's current state (the returned iterates after a solve). */
int nmpc_plate_get_state(nmpc_plate* h, double* x, double* u, double* lam, void* stream);

/* The plant of the closed loop (Sec. 5.3): w (device [sum n_s], in place)
   advances by dt in n_sub explicit-Euler sub-steps of the model with the
   actuator points held at the first-stage inputs of the current state.
   BAD_ARG without a solved state. */
int nmpc_plate_plant_step(nmpc_plate* h, double* w, double dt, int n_sub, void* stream);

/* Receding-horizon loop: each of `steps` periods solves from x0 = w (cold
   at the first step unless the handle holds a state, then shifted), applies
   u_1 for one stage length (each instance's own h; n_sub plant sub-steps).  u_hist: NULL or
   device [steps][sum n_u]; iters_hist, res_hist: NULL or host
   [steps][n].  Returns the first non-OK solve code met. */
int nmpc_plate_closed_loop(nmpc_plate* h, double* w, const double* x_ref, const double* u_ref,
                           int steps, int n_sub, double* u_hist, int* iters_hist,
                           double* res_hist, void* stream);

/* Free everything (NULL is a no-op).  Synchronizes. */
void nmpc_plate_destroy(nmpc_plate* h);

#ifdef __cplusplus
}
#endif

#endif /* NMPC_GB300_PLATE_H */
