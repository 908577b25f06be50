/*
 * nmpc_wave.h -- C ABI of the second-order-in-time solver: the double-layer
 * method on PDEs with a w_tt term (Sec. 2, eq. 1 with a != 0), state
 * x = (W, dW/dt) (eq. 5), the lower layer's F_x and F_x^T solves by the
 * elimination of v6 (Sec. 4.3, eq. 25).
 *
 * Problem per instance:
 *   grid    dim = 1 or 2, m points per axis; bc 0: zero Neumann, the points
 *           include the boundary (spacing 1/(m-1)), mirrored fictitious
 *           points (eqs. 2-3); bc 1: zero Dirichlet, interior points
 *           (spacing 1/(m+1));
 *   model   a w_tt + b w_t = c Lap w - kappa w^3 + sum_a gain u_a delta_a,
 *           constants a > 0, b, c, kappa; input a is a point force on the
 *           grid point act_cell[a];
 *   state   x_i = (W_i, V_i), V = dW/dt, n_x = 2 n_g per stage, all W first;
 *           f = [V; g], g = (c L W - b V - kappa W^3 + B u) / a;
 *   NLP     backward Euler x_i = x_{i-1} + h f(u_i, x_i) (eq. 6); stage cost
 *           h (q/2 |W - w_ref|^2 + qv/2 |V|^2 + r/2 |u - u_ref|^2), terminal
 *           h qf/2 |W_N - w_ref|^2, regularization gamma/2 |u_i - u_i^k|^2
 *           (Remark 1); no input bounds (every step is the full step);
 *   solve   K(S) = 0 of eq. 9 by the upper-layer Jacobi iteration (eq. 15) or
 *           its red-black Gauss-Seidel form (eq. 18 in the even-then-odd
 *           stage order), each stage by the lower layer (eqs. 21-24, the
 *           u-iteration of Sec. 5.2): F_x (v6, v7) = (b6, b7) as v6 = h v7 -
 *           b6 with E v7 = b7 + h grad_W g b6, E = h grad_V g - I + h^2
 *           grad_W g (eq. 25); F_x^T (v8, v9) = (b8, b9) as E^T v9 = b9 + h b8,
 *           v8 = h grad_W g^T v9 - b8; E and E^T by n_lo pointwise Jacobi
 *           sweeps from zero (Lemma 1); until ||K(S^k)||_inf <= tol.
 * Arrays, packed per instance in setup order, float64, device pointers:
 *   x0 [sum 2 n_g] (W0 then V0); w_ref [sum n_g]; u_ref [sum n_u];
 *   x, lam [sum N 2 n_g] stage-major, (W, V) per stage; u [sum N n_u].
 * Arithmetic: float64, or with NMPC_MIXED a float32 lower layer.  The
 * caller owns its buffers; the handle owns its workspace (allocated in
 * setup, freed in destroy); solves allocate nothing.  Return codes are the NMPC_* codes of nmpc.h.
 */
#ifndef NMPC_GB300_WAVE_H
#define NMPC_GB300_WAVE_H

#include <stdint.h>

#include "nmpc.h"

#ifdef __cplusplus
extern "C" {
#endif

#define NMPC_WAVE_MAX_POINTS 1024 /* grid points of one instance            */

typedef struct {
  int dim;             /* 1 or 2                                              */
  int m;               /* grid points per axis                                */
  int bc;              /* 0 zero Neumann (boundary points included), 1 zero Dirichlet */
  int horizon;         /* N >= 1                                              */
  int n_u;             /* point forces, 1..NMPC_MAX_NU                        */
  const int* act_cell; /* [n_u] distinct grid point indices (host, read in setup) */
  double h;            /* stage length                                        */
  double a, b, c;      /* a w_tt + b w_t = c Lap w + ...; a > 0               */
  double kappa;        /* cubic term -kappa w^3                               */
  double gain;         /* force per unit input                                */
  double q, qv, r, qf; /* weights: displacement, velocity, input, terminal    */
  double gamma;        /* regularization (>= 0)                               */
} nmpc_wave_desc;

typedef struct {
  double tol;       /* stop at ||K(S^k)||_inf <= tol                         */
  int max_iter;     /* iterations before NMPC_ERR_NOT_CONVERGED              */
  int n_lo;         /* Jacobi sweeps per E, E^T solve (2 as Table 2)         */
  int n_u_it;       /* u fixed-point iterations (Sec. 5.2: 2)                */
  int variant;      /* NMPC_VARIANT_JACOBI or NMPC_VARIANT_REDBLACK           */
  int check_every;  /* iterations between host polls of the running count    */
  int precision;    /* NMPC_FP64 (default), or NMPC_MIXED: the lower layer's
                       sweeps and u-iteration in float32 against the float64
                       residual, coefficients and update (the root is the
                       float64 root)                                         */
} nmpc_wave_opts;

typedef struct nmpc_wave nmpc_wave;

/* Defaults: tol 1e-6, max_iter 5000, n_lo 2, n_u_it 2, Jacobi, check_every 16,
   NMPC_FP64. */
void nmpc_wave_default_opts(nmpc_wave_opts* o);

/* Validate the descriptors (BAD_ARG: dims, a <= 0, negative weights, r <= 0,
   actuator indices out of the grid or repeated; UNSUPPORTED: more than
   NMPC_WAVE_MAX_POINTS points or NMPC_MAX_NU inputs), build the stencil
   tables and allocate the workspace on the current device.  Synchronous. */
int nmpc_wave_setup(const nmpc_wave_desc* descs, int n_instances, const nmpc_wave_opts* opts,
                    nmpc_wave** out);

/* out[0] = sum 2 n_g (x0), out[1] = sum N 2 n_g (x, lam), out[2] = sum N n_u,
   out[3] = sum n_u, out[4] = sum n_g (w_ref). */
int nmpc_wave_sizes(const nmpc_wave* h, int64_t* out);

/* Solve every instance from x0 tracking (w_ref, u_ref) (device).  init:
   NMPC_INIT_COLD (x_i = x0, u = 0, lambda = 0), NMPC_INIT_WARM (the handle's
   current state) or NMPC_INIT_SHIFT (the current state shifted by one
   stage, the last one repeated).  u_out: device [sum N n_u] or NULL; stats:
   host [n].  Synchronizes.  NMPC_OK when every instance converged, else the
   first of NOT_CONVERGED / DIVERGED met. */
int nmpc_wave_solve(nmpc_wave* h, const double* x0, const double* w_ref, const double* u_ref,
                    int init, double* u_out, nmpc_stats* stats, void* stream);

/* n_iter >= 1 iterations (no convergence test) from (x_in, u_in, lam_in)
   into (x_out, u_out, lam_out), device packed arrays (in and out may
   alias).  out: NULL or host [n][3] = (||K||_inf, ||K||_2, step length 1)
   of the last iteration.  Synchronizes when out is given. */
int nmpc_wave_iterate(nmpc_wave* h, const double* x0, const double* w_ref, const double* u_ref,
                      const double* x_in, const double* u_in, const double* lam_in, double* x_out,
                      double* u_out, double* lam_out, int n_iter, double* out, void* stream);

/* The handle's current state (the returned iterates after a solve). */
int nmpc_wave_get_state(nmpc_wave* h, double* x, double* u, double* lam, void* stream);

/* The plant of the closed loop (Sec. 5.3): x = (W, V) (device [sum 2 n_g],
   in place) advances by dt in n_sub semi-implicit (symplectic) Euler steps
   of the model, V <- V + tau g(W, V, u1) then W <- W + tau V, with the
   inputs at the first-stage values u1 of the current state.  BAD_ARG
   without a solved state. */
int nmpc_wave_plant_step(nmpc_wave* h, double* x, double dt, int n_sub, void* stream);

/* Receding-horizon loop: each of `steps` periods solves from x0 = x (cold
   at the first step unless the handle holds a state, then shifted), applies
   u_1 for one stage length (each instance's own h; n_sub plant steps).
   u_hist: NULL or device [steps][sum n_u]; iters_hist, res_hist: NULL or
   host [steps][n].  Returns the first non-OK solve code met. */
int nmpc_wave_closed_loop(nmpc_wave* h, double* x, const double* w_ref, const double* u_ref,
                          int steps, int n_sub, double* u_hist, int* iters_hist,
                          double* res_hist, void* stream);

/* Free everything (NULL is a no-op).  Synchronizes. */
void nmpc_wave_destroy(nmpc_wave* h);

#ifdef __cplusplus
}
#endif

#endif /* NMPC_GB300_WAVE_H */
