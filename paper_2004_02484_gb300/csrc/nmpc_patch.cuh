// Actuator patches of the strip path (included from nmpc_kernels.cuh inside
// namespace nmpc_dev).
//
// The u fixed-point iteration of Sec. 5.2 reads P^{-1} at the actuator cells:
// y_lambda(a) of Y(v3) = P^{-1}(F_u v3 - K1, -K3).  For stages on the strip
// path, k_patch runs first in each iteration: one warp per (instance, stage,
// actuator) evaluates the residual and P^{-1} on the actuator's patch (the
// cells within E = 2 n_lo - 1 of its cell, which is the patch's single own
// cell: the residual is a five-point stencil and one P^{-1} application is
// 2 (n_lo - 1) stencil sweeps after pointwise first sweeps) for
// y0 = Y(0)_lambda(a) and, for n_u_it > 1, the response g = Z(e_a)_lambda(a)
// to a unit control, iterates v3 <- (K2 + h b0 (y0 + g v3)) / A_uu and
// stores v3.  This equals the full-field iteration when no two actuators
// share a cell or lie within 2 (n_lo - 1) cells of each other (the host
// routes other instances to the slab path when n_u_it > 1).

// Region geometry: RW x RH cells; region cell r = rj RW + ri is grid cell
// (gy0 + rj, gx0 + ri); its level is its distance to the region's border.
struct Rgn {
  int RW, RH, nR, gx0, gy0;
};

// Staged float64 inputs of a region (shared memory), one record of SREC
// doubles per cell: x_i, lambda_i, x_{i-1} (x0 at stage 1), lambda_{i+1}
// (unused at the last stage), ref.  All five are zero outside the grid; at
// the region's border only x, lambda are read.
constexpr int SREC = 5;
enum { R_X = 0, R_L = 1, R_XP = 2, R_LN = 3, R_RF = 4 };

// Residual accumulators of a region's own cells: float32 norms and the
// rounding bound's magnitudes (split residual), float64 norms (full).
struct Norms {
  float fmax, fsq;
  float4 mg;
  double vmax, vsq;
  float gm;  // largest neighbour difference of x (difference-form Laplacian)
};

template <int NT>
__device__ __forceinline__ void rgn_sync() {
  if constexpr (NT == 32) __syncwarp();
  else __syncthreads();
}

// The residual and one P^{-1} application on a region by a group of NT
// threads (a CTA, or a warp for an actuator patch); the thread at column tx,
// row ty (tx < RW, ty < nty; other threads idle) carries the region cells
// (ty + q nty, tx), q < NS, in registers through every pass.
//
// Pass 0 covers the whole region; the later passes run on every interior
// cell (level >= 1) with no per-level branches: a slot outside the interior
// recomputes a clamped interior cell and stores nothing, a cell at level
// < m holds values pass m does not need (the own cells, level >= E, depend
// only on cells computed at their proper level), and cells outside the grid
// carry 1/diag F_x = 0, which zeroes every sweep there (the Dirichlet ring).
//
// S: staged records; W0, W1, W2: work arrays of nR float64-sized cells.
// amask: bit q set when slot q's cell holds an actuator.  v3 (per actuator,
// or null for v3 = 0) enters the right-hand side as F_u v3.  With unit2 a
// second right-hand side, a unit control at the region's centre (K = 0), is
// solved with the same coefficients.  out(q, r, c, v5, v4, which) receives
// P^{-1}'s result at every own cell (level >= E inside the grid) for
// right-hand side `which`.  resid_only: stop after the residual.
template <typename T, int NS, int NT, int n_lo, bool UNIT2, typename OUT>
__device__ __forceinline__ void region_solve(const InstDev& I, const Rgn& R, int tx, int ty, int nty,
                                             const double* S, double* W0, double* W1, double* W2,
                                             bool full, bool last, const double* u, const int* act,
                                             const T* v3, unsigned amask, bool norms,
                                             bool resid_only, bool unit2, Norms& nm, OUT out) {
  constexpr int E = 2 * n_lo - 1;
  const int RW = R.RW, RH = R.RH;
  const bool on = tx < RW && ty < nty;
  const int cxc = min(max(tx, 1), RW - 2);  // clamped interior column
  const bool col_in = on && tx >= 1 && tx <= RW - 2;
  const int lvx = min(tx, RW - 1 - tx);
  const int gx = R.gx0 + tx;
  const bool gx_ok = gx >= 0 && gx < I.mx;
  // per slot: interior cell index (clamped), and bit masks of the slots that
  // are interior (st), inside the grid (gd) and own (ow)
  int rr[NS];
  unsigned st = 0u, gd = 0u, ow = 0u;
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const int rj = ty + q * nty;
    rr[q] = min(max(rj, 1), RH - 2) * RW + cxc;
    const bool in = col_in && rj >= 1 && rj <= RH - 2;
    const int gy = R.gy0 + rj;
    const bool g = in && gx_ok && gy >= 0 && gy < I.my;
    const int lv = min(lvx, min(rj, RH - 1 - rj));
    st |= (in ? 1u : 0u) << q;
    gd |= (g ? 1u : 0u) << q;
    ow |= ((g && lv >= E) ? 1u : 0u) << q;
  }
  // ---- pass 0: the residual's stencil inputs on the whole region ----
  float* W0f = reinterpret_cast<float*>(W0);
  float* W1f = reinterpret_cast<float*>(W1);
  float* W2f = reinterpret_cast<float*>(W2);
  if (on) {
    if (full) {
      const double k0 = I.k0, k1h = 0.5 * I.k1;
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const int rj = ty + q * nty;
        if (rj >= RH) break;
        const int r = rj * RW + tx;
        const double x = S[SREC * r + R_X];
        W0[r] = k0 * (x + k1h * x * x);
        W1[r] = S[SREC * r + R_L];
      }
    } else {
      const float fk0 = I.fk0, fk1h = I.fk1h;
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const int rj = ty + q * nty;
        if (rj >= RH) break;
        const int r = rj * RW + tx;
        const float xv = d2f(S[SREC * r + R_X]), lf = d2f(S[SREC * r + R_L]);
        W0f[r] = fk0 * (xv + fk1h * xv * xv);
        W1f[r] = lf;
        // read back by this thread in pass 1 (split residuals only run with
        // T = float, so the float view indexes the same cells as T does)
        W2f[r] = xv;
        if (norms) {
          nm.mg.x = fmaxf(nm.mg.x, fabsf(xv));
          nm.mg.y = fmaxf(nm.mg.y, fabsf(lf));
        }
      }
    }
  }
  rgn_sync<NT>();

  // ---- pass 1: K_i (eq. 9) and the coefficient fields on the interior ----
  const T th = pick<T>(I.h, I.fh), tdc = pick<T>(I.dcoef, I.fdc), tb0 = pick<T>(I.b0, I.fb0);
  const T tcx = pick<T>(I.cx, I.fcx), tcy = pick<T>(I.cy, I.fcy);
  T K3[NS], ax[NS], rg[NS], dp[NS], v1[NS];
  if (full) {
    const double h = I.h, cxd = I.cx, cyd = I.cy, dcd = I.dcoef, k0 = I.k0, k1 = I.k1, qd = I.q;
    const double b0d = I.b0, hqf = I.hqf, axl = last ? I.hqf : 0.0;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const int r = rr[q];
      const double* rec = S + SREC * r;
      // sources of the cell: sum of u (b0 B u in K1) and of v3 (F_u v3)
      double srcd = 0.0;
      T inj = T(0);
      if ((amask >> q) & 1u) {
        const int c = (R.gy0 + ty + q * nty) * I.mx + gx;  // an interior slot (not clamped)
        for (int a = 0; a < I.nu; ++a)
          if (act[a] == c) {
            srcd += u[a];
            if (v3) inj += v3[a];
          }
      }
      const double x = rec[R_X], lam = rec[R_L], xp = rec[R_XP], rc = rec[R_RF];
      const double ln = last ? hqf * (x - rc) : rec[R_LN];
      const double lphi = cxd * (W0[r - 1] + W0[r + 1]) + cyd * (W0[r - RW] + W0[r + RW]) - dcd * W0[r];
      const double mu = cxd * (W1[r - 1] + W1[r + 1]) + cyd * (W1[r - RW] + W1[r + RW]) - dcd * lam;
      const double dphi = k0 * (1.0 + k1 * x);
      const double K1d = xp - x + h * (lphi + b0d * srcd);
      const double K3d = ln - lam + h * (qd * (x - rc) + dphi * mu);
      if (norms && ((ow >> q) & 1u)) {
        nm.vmax = fmax(nm.vmax, fmax(abs_or_inf(K1d), abs_or_inf(K3d)));
        nm.vsq += K1d * K1d + K3d * K3d;
      }
      K3[q] = to_T<T>(K3d);
      dp[q] = to_T<T>(dphi);
      ax[q] = to_T<T>(h * (qd + k0 * k1 * mu) + axl);
      // 1/diag F_x, zero outside the grid (every sweep there stays zero)
      rg[q] = ((gd >> q) & 1u) ? rcp_T(-T(1) - th * tdc * dp[q]) : T(0);
      v1[q] = (th * tb0 * inj - to_T<T>(K1d)) * rg[q];  // first F_x sweep of F_x v5 = F_u v3 - K1
    }
  } else {
    const float fcx = I.fcx, fcy = I.fcy, fdc = I.fdc, fh = I.fh, fk0 = I.fk0, fk1 = I.fk1;
    const float fq = I.fq, fb0 = I.fb0, fk01 = I.fk01;
    const float hqff = last ? I.fhqf : 0.0f;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const int r = rr[q];
      const double* rec = S + SREC * r;
      float srcf = 0.0f;
      T inj = T(0);
      if ((amask >> q) & 1u) {
        const int c = (R.gy0 + ty + q * nty) * I.mx + gx;  // an interior slot (not clamped)
        for (int a = 0; a < I.nu; ++a)
          if (act[a] == c) {
            srcf += d2f(u[a]);
            if (v3) inj += v3[a];
          }
      }
      const double x = rec[R_X], lam = rec[R_L], xp = rec[R_XP], rc = rec[R_RF];
      const float lphi = fcx * (W0f[r - 1] + W0f[r + 1]) + fcy * (W0f[r - RW] + W0f[r + RW]) -
                         fdc * W0f[r];
      const float mu = fcx * (W1f[r - 1] + W1f[r + 1]) + fcy * (W1f[r - RW] + W1f[r + RW]) -
                       fdc * W1f[r];
      const float xv = std::is_same<T, float>::value ? W2f[r] : d2f(x), rv = d2f(rc);
      const float dphi = fk0 * (1.0f + fk1 * xv);
      const float t1 = fh * (lphi + fb0 * srcf);
      const float t3 = fh * (fq * (xv - rv) + dphi * mu);
      const double d3 = last ? -lam : rec[R_LN] - lam;
      const float dx = d2f(xp - x), dl = d2f(d3);
      const float K1f = dx + t1;
      const float K3f = dl + t3 + hqff * (xv - rv);
      if (norms) {
        const bool own = (ow >> q) & 1u;
        const float K1v = own ? K1f : 0.0f, K3v = own ? K3f : 0.0f;
        nm.mg.z = fmaxf(nm.mg.z, own ? fmaxf(fabsf(dx), fabsf(dl)) : 0.0f);
        nm.mg.w = fmaxf(nm.mg.w, own ? fabsf(rv) : 0.0f);
        nm.fmax = fmax_nan(nm.fmax, fmax_nan(fabsf(K1v), fabsf(K3v)));
        nm.fsq += K1v * K1v + K3v * K3v;
      }
      K3[q] = (T)K3f;
      dp[q] = (T)dphi;
      ax[q] = (T)(fh * (fq + fk01 * mu) + hqff);
      // 1/diag F_x, zero outside the grid (every sweep there stays zero)
      rg[q] = ((gd >> q) & 1u) ? rcp_T(-T(1) - th * tdc * dp[q]) : T(0);
      v1[q] = (th * tb0 * inj - (T)K1f) * rg[q];  // first F_x sweep of F_x v5 = F_u v3 - K1
      // one slot's loads at a time: hoisting all slots' loads would spill
      asm volatile("" ::: "memory");
    }
  }
  if (resid_only) return;

  // ---- P^{-1} (eq. 24): n_lo - 1 F_x sweeps, then n_lo - 1 F_x^T sweeps ----
  const int centre = E * RW + E;  // a patch's actuator cell
  // v5 and w1 (the last F_x sweep and the first F_x^T sweep): separate arrays
  // when a second right-hand side reuses the coefficients, else the
  // registers of A_xx and K3, which are dead once they are formed
  T v5a[UNIT2 ? NS : 1], w1a[UNIT2 ? NS : 1];
  auto V5 = [&](int q) -> T& {
    if constexpr (UNIT2) return v5a[q];
    else return ax[q];
  };
  auto WF1 = [&](int q) -> T& {
    if constexpr (UNIT2) return w1a[q];
    else return K3[q];
  };
  auto sweeps = [&](bool unit, int which) {
    T* A = reinterpret_cast<T*>(W2);
    T* Bn = reinterpret_cast<T*>(W0);
    // first sweep: the stored v1, or D^{-1} h b0 e_centre for the unit control
    auto V0 = [&](int q) { return unit ? ((rr[q] == centre) ? th * tb0 * rg[q] : T(0)) : v1[q]; };
    auto K3v = [&](int q) { return unit ? T(0) : K3[q]; };
    if constexpr (n_lo == 1) {
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const T v = V0(q);
        const T w = (-K3v(q) - ax[q] * v) * rg[q];
        if ((ow >> q) & 1u) out(q, rr[q], (R.gy0 + ty + q * nty) * I.mx + gx, v, w, which);
      }
    } else {
#pragma unroll
      for (int q = 0; q < NS; ++q)
        if ((st >> q) & 1u) A[rr[q]] = dp[q] * V0(q);
      rgn_sync<NT>();
      // F_x sweeps 2 .. n_lo; the last one also forms the first F_x^T sweep
#pragma unroll
      for (int m = 2; m <= n_lo; ++m) {
        const bool lastx = (m == n_lo);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          const int r = rr[q];
          const T off = th * (tcx * (A[r - 1] + A[r + 1]) + tcy * (A[r - RW] + A[r + RW]));
          const T v = V0(q) - rg[q] * off;
          if (!lastx) {
            if ((st >> q) & 1u) Bn[r] = dp[q] * v;
          } else {
            const T w = (-K3v(q) - ax[q] * v) * rg[q];
            V5(q) = v;
            WF1(q) = w;
            if ((st >> q) & 1u) Bn[r] = w;
          }
        }
        rgn_sync<NT>();
        T* t = A;
        A = Bn;
        Bn = t;
      }
      // F_x^T sweeps 2 .. n_lo (passes n_lo + 1 .. E)
#pragma unroll
      for (int m = n_lo + 1; m <= E; ++m) {
        const bool fin = (m == E);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          const int r = rr[q];
          const T off = th * dp[q] * (tcx * (A[r - 1] + A[r + 1]) + tcy * (A[r - RW] + A[r + RW]));
          const T v4 = WF1(q) - rg[q] * off;
          if (!fin) {
            if ((st >> q) & 1u) Bn[r] = v4;
          } else if ((ow >> q) & 1u) {
            out(q, r, (R.gy0 + ty + q * nty) * I.mx + gx, V5(q), v4, which);
          }
        }
        if (!fin) {
          rgn_sync<NT>();
          T* t = A;
          A = Bn;
          Bn = t;
        }
      }
    }
  };
  sweeps(false, 0);
  if constexpr (UNIT2) {
    if (unit2) {
      rgn_sync<NT>();  // the first right-hand side's last reads are done
      sweeps(true, 1);
    }
  }
}

// Region thread shape: nty rows of RW threads (at most NT threads).
__host__ __device__ inline int region_rows_of_threads(int RW, int NT) { return NT / RW; }

// Patch cells per lane: a (2E + 1) x (2E + 1) patch, E = 2 n_lo - 1, on a warp
// laid out as rows of 2E + 1 lanes.
template <int n_lo>
__host__ __device__ constexpr int patch_slots() {
  return (4 * n_lo - 1 + 32 / (4 * n_lo - 1) - 1) / (32 / (4 * n_lo - 1));
}

// Shared memory of one k_patch warp: the stage's controls and actuator cells,
// then 8 arrays of (2E + 1)^2 doubles (five staged inputs, three work arrays).
struct PatchShared {
  double u[MAX_NU];
  int act[MAX_NU];
};

// v3 of one actuator: k_patch work item (instance, stage, actuator) per warp.
// The warp stages the patch (radius E around the actuator's cell, zero
// outside the grid), runs the residual and P^{-1} on it for Y(0) (and the
// unit response for n_u_it > 1), and stores v3 of the u fixed-point
// iteration (in T, as float64) at the control's position.
template <typename T, int n_lo>
__global__ void __launch_bounds__(128) k_patch(IterArgs A, int MODE, int j) {
  constexpr int E = 2 * n_lo - 1, P = 2 * E + 1, nP = P * P, NTY = 32 / P;
  constexpr int WPB = 4;  // warps per block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t per_warp = ((sizeof(PatchShared) + 15) & ~size_t(15)) + 8 * nP * sizeof(double);
  PatchShared& ps = *reinterpret_cast<PatchShared*>(smem_raw + warp * per_warp);
  double* S = reinterpret_cast<double*>(smem_raw + warp * per_warp +
                                        ((sizeof(PatchShared) + 15) & ~size_t(15)));
  double* W0 = S + SREC * nP;
  double* W1 = W0 + nP;
  double* W2 = W1 + nP;
  pdl_trigger();
  const int k = (MODE == MODE_SOLVE) ? *(volatile int*)A.iter_k + launch_iter(A, j) : 0;
  const int half = launch_half(A, j);
  const int rd = (MODE == MODE_SOLVE) ? (k & 1) : 0;
  pdl_wait();
  // the running-instance count for the strip launch that follows (no
  // instance finishes between the two: only the strip kernels keep the books)
  if (MODE == MODE_SOLVE && A.n_tail > 0 && blockIdx.x == 0 && threadIdx.x == 0)
    *A.strip_run = *(volatile int*)A.n_active;
  const int item = ((A.rb && half) ? A.n_patches_even : 0) + blockIdx.x * WPB + warp;
  const int item_end = A.rb ? (half ? A.n_patches : A.n_patches_even) : A.n_patches;
  if (item >= item_end) return;  // warp-uniform; no block barriers follow
  const int4 it = A.patches[item];
  const int b = it.x, s = it.y, a = it.z;
  if (!stage_in_half(A, s, half)) return;
  bool full;
  if (MODE == MODE_SOLVE) {
    int skip = 0, fl = 1;
    if (lane == 0) {
      const Decision d = decide(A, b, k);
      skip = d.skip || (k == A.max_iter);  // a residual-only iteration needs no v3
      fl = d.full;
    }
    skip = __shfl_sync(0xffffffffu, skip, 0);
    fl = __shfl_sync(0xffffffffu, fl, 0);
    if (skip) return;
    full = fl != 0;
  } else {
    full = A.full_all != 0;
  }
  const InstDev& I = A.inst[b];
  const int nu = I.nu;
  const bool last = (s == I.N - 1);
  for (int q = lane; q < nu; q += 32) {
    ps.act[q] = A.act[I.act_off + q];
    ps.u[q] = A.uin[rd][I.u_off + (long long)s * nu + q];
  }
  __syncwarp();
  const int ca = ps.act[a], ax0 = ca % I.mx, ay0 = ca / I.mx;
  const Rgn R{P, P, nP, ax0 - E, ay0 - E};
  const long long so = I.s_off + (long long)s * I.ng;
  const double* Xg = A.xin[rd] + so;
  const double* Lg = A.lin[rd] + so;
  // v3 enters the right-hand side only: in red-black half 1 it is formed
  // with x_{i-1}, lambda_{i+1} as updated by half 0 (the buffer being written)
  const bool rbn = A.rb && half == 1;
  const double* XPg = (s == 0) ? A.x0 + I.g_off
                               : (rbn ? A.xout[rd ^ 1] : A.xin[rd]) + so - I.ng;
  const double* LNg = (rbn ? A.lout[rd ^ 1] : A.lin[rd]) + so + I.ng;
  const double* RFg = A.ref + I.g_off;
  for (int r = lane; r < nP; r += 32) {
    const int rj = r / P, ri = r - rj * P;
    const int gy = R.gy0 + rj, gx = R.gx0 + ri;
    if (gx >= 0 && gx < I.mx && gy >= 0 && gy < I.my) {
      const int c = gy * I.mx + gx;
      double* rec = S + SREC * r;
      rec[R_X] = Xg[c];
      rec[R_L] = Lg[c];
      rec[R_XP] = XPg[c];
      rec[R_LN] = last ? 0.0 : LNg[c];
      rec[R_RF] = RFg[c];
    } else {
      double* rec = S + SREC * r;
      rec[R_X] = rec[R_L] = rec[R_XP] = rec[R_LN] = rec[R_RF] = 0.0;
    }
  }
  // this lane's slots that hold an actuator cell at level >= 1
  const int tx = lane % P, ty = lane / P;
  unsigned am = 0u;
  for (int a2 = 0; a2 < nu; ++a2) {
    const int c2 = ps.act[a2];
    const int rx = c2 % I.mx - R.gx0, ry = c2 / I.mx - R.gy0;
    if (rx == tx && ty < NTY && rx >= 1 && rx <= P - 2 && ry >= 1 && ry <= P - 2 &&
        (ry - ty) % NTY == 0 && ry >= ty)
      am |= 1u << ((ry - ty) / NTY);
  }
  __syncwarp();
  Norms nm{};
  T y0 = T(0), g = T(0);
  constexpr int centre = E * P + E;
  region_solve<T, patch_slots<n_lo>(), 32, n_lo, true>(
      I, R, tx, ty, NTY, S, W0, W1, W2, full, last, ps.u, ps.act,
      (const T*)nullptr, am, false, false, A.n_u_it > 1, nm, [&](int, int r, int, T, T v4, int which) {
        if (r == centre) {
          if (which == 0) y0 = v4;
          else g = v4;
        }
      });
  // the centre cell (E, E) belongs to the lane at column E, row E % NTY
  const int cl = (E % NTY) * P + E;
  y0 = __shfl_sync(0xffffffffu, y0, cl);
  g = __shfl_sync(0xffffffffu, g, cl);
  if (lane == 0) {
    const T th = pick<T>(I.h, I.fh), tb0 = pick<T>(I.b0, I.fb0), auu = pick<T>(I.auu, I.fauu);
    const T b3 = (T)(I.h * (I.r * ps.u[a] + I.b0 * S[SREC * centre + R_L]));  // K2, the u row of eq. 9
    T v = T(0);
    for (int q = 0; q < A.n_u_it; ++q) v = (b3 + th * tb0 * (y0 + g * v)) / auu;
    A.v3g[I.u_off + (long long)s * nu + a] = (double)v;
  }
}

#include "nmpc_strip.cuh"
