// Line path of the upper-layer iteration for 1D stages (included from
// nmpc_kernels.cuh inside namespace nmpc_dev, after nmpc_patch.cuh).
//
// One warp of k_line computes one (instance, stage) work item of iteration k
// for a 1D stage of M <= 32 CPL cells: lane l holds the CPL consecutive cells
// l CPL .. l CPL + CPL - 1 in registers, so a three-point stencil reads its
// neighbours from the lane's own registers and, at the lane's two ends, from
// lanes l - 1 and l + 1 by one warp shuffle each.  The work item's float64
// inputs (x_i, lambda_i, x_{i-1}, lambda_{i+1}, the reference) arrive by
// coalesced asynchronous copies into shared memory, cell q at q + q / CPL (the
// padding puts a warp's blocked reads into distinct banks); cells q >= M are
// zero-filled and carry 1/diag F_x = 0, so every sweep stays zero there (the
// Dirichlet ring).  Then, with no block barrier:
//   K_i (eq. 9) in the split or the float64 form, the coefficient fields
//   Phi'(x), A_xx, 1/diag F_x, the norms (warp shuffles);
//   the lower layer (eqs. 22-24) with the full-field u fixed-point iteration
//   of Sec. 5.2: n_u_it + 1 applications of P^{-1}, each n_lo pointwise
//   Jacobi sweeps of F_x and of F_x^T, on registers;
//   S_i <- S_i + alpha Y (eq. 15) in float64, coalesced through the same
//   shared-memory layout.
// The arithmetic is that of the cluster path's 1D slab (same operations in
// the same order), so the two paths agree to rounding.

constexpr int LINE_WARPS = 4;    // warps (stages) per CTA
constexpr int LINE_MAX_CPL = 8;  // cells per lane: M <= 256
constexpr int LINE_SLOTS = 32 * LINE_MAX_CPL + 32;  // padded positions per field
enum LField { L_X = 0, L_L, L_XP, L_LN, L_RF, L_NF };

// Shared memory of one line warp: the staged inputs, and per control its
// cell, value, lambda at its cell, K1 there (b1), K2 (b3) and v3.
struct LineShared {
  double f[L_NF][LINE_SLOTS];
  double u[MAX_NU], lact[MAX_NU];
  int act[MAX_NU];
  float b1[MAX_NU], b3[MAX_NU], v3[MAX_NU];
};

// Padded position of cell q.
template <int CPL>
__device__ __forceinline__ int lpad(int q) {
  return CPL == 1 ? q : q + q / CPL;
}

// out[t] = sum of the two neighbours of the lane's cell t (zero beyond the
// line's ends; cells past M hold zeros themselves).
template <int CPL, typename V>
__device__ __forceinline__ void line_nsum(const V (&v)[CPL], V (&out)[CPL], int lane) {
  V lft = __shfl_up_sync(0xffffffffu, v[CPL - 1], 1);
  V rgt = __shfl_down_sync(0xffffffffu, v[0], 1);
  lft = (lane == 0) ? V(0) : lft;
  rgt = (lane == 31) ? V(0) : rgt;
#pragma unroll
  for (int t = 0; t < CPL; ++t) out[t] = (t > 0 ? v[t - 1] : lft) + (t < CPL - 1 ? v[t + 1] : rgt);
}

// Value of a blocked field at cell c (every lane receives it).
template <int CPL, typename V>
__device__ __forceinline__ V line_at(const V (&v)[CPL], int c) {
  const int tc = c & (CPL - 1);
  V mine = v[0];
#pragma unroll
  for (int t = 1; t < CPL; ++t) mine = (tc == t) ? v[t] : mine;
  return __shfl_sync(0xffffffffu, mine, c / CPL);
}

// The stage of work item (b, s) for one residual form (FULL: float64).
// RBN: red-black half 1 (the right-hand side takes x_{i-1}, lambda_{i+1} as
// updated by half 0, read from the buffer being written; the norms stay
// those of K(S^k)).
template <int CPL, bool FULL, bool RBN>
__device__ __forceinline__ void line_body(const IterArgs& A, LineShared& ws, int lane, int b,
                                          int s, int k, int rd, bool resid_only) {
  using T = float;
  // the instance's constants in registers (the stores below could alias the
  // descriptor table as far as the compiler knows)
  const InstDev I = A.inst[b];
  const int M = I.mx, nu = I.nu;
  const bool last = (s == I.N - 1);
  const long long so = I.s_off + (long long)s * I.ng;
  const double* Xg = A.xin[rd] + so;
  const double* Lg = A.lin[rd] + so;
  const double* XPg = (s == 0) ? A.x0 + I.g_off : A.xin[rd] + so - I.ng;
  const double* LNg = last ? Lg : A.lin[rd] + so + I.ng;
  const double* RFg = A.ref + I.g_off;
  const double* XPNg = (s == 0) ? A.x0 + I.g_off : A.xout[rd ^ 1] + so - I.ng;
  const double* LNNg = A.lout[rd ^ 1] + so + I.ng;
  // coalesced copies: lane l copies cells t 32 + l (zeros past M)
#pragma unroll
  for (int t = 0; t < CPL; ++t) {
    const int q = t * 32 + lane;
    const bool ok = q < M;
    const int qc = ok ? q : 0;
    const int p = lpad<CPL>(q);
    cp_async8_zfill(&ws.f[L_X][p], Xg + qc, ok);
    cp_async8_zfill(&ws.f[L_L][p], Lg + qc, ok);
    cp_async8_zfill(&ws.f[L_XP][p], XPg + qc, ok);
    cp_async8_zfill(&ws.f[L_LN][p], LNg + qc, ok && !last);
    cp_async8_zfill(&ws.f[L_RF][p], RFg + qc, ok);
  }
  asm volatile("cp.async.commit_group;\n" ::);
  const double* uin_s = A.uin[rd] + I.u_off + (long long)s * nu;
  for (int a = lane; a < nu; a += 32) {
    const int c = A.act[I.act_off + a];
    ws.act[a] = c;
    ws.u[a] = uin_s[a];
    ws.lact[a] = __ldcg(Lg + c);
  }
  asm volatile("cp.async.wait_all;\n" ::);
  __syncwarp();

  // blocked registers: lane l's cells l CPL + t
  const int q0 = lane * CPL;
  // red-black half 1: the lane's cells of the updated x_{i-1}, lambda_{i+1}
  double xpn[RBN ? CPL : 1], lnn[RBN ? CPL : 1];
  if constexpr (RBN) {
#pragma unroll
    for (int t = 0; t < CPL; ++t) {
      const bool ok = q0 + t < M;
      xpn[t] = ok ? XPNg[q0 + t] : 0.0;
      lnn[t] = (ok && !last) ? LNNg[q0 + t] : 0.0;
    }
  }
  const int pb0 = lpad<CPL>(q0);  // positions pb0 + t (one lane's cells are contiguous)
  const T th = I.fh, tdc = I.fdc, tcx = I.fcx, tb0 = I.fb0;
  T K1[CPL], K3[CPL], dp[CPL], ax[CPL], rg[CPL];
  double rmax, rsq, e = 0.0;
  if constexpr (FULL) {
    double xd[CPL], ld[CPL], ph[CPL], ns[CPL];
#pragma unroll
    for (int t = 0; t < CPL; ++t) {
      xd[t] = ws.f[L_X][pb0 + t];
      ld[t] = ws.f[L_L][pb0 + t];
      ph[t] = phi_d(xd[t], I.k0, I.k1);
    }
    double vmax = 0.0, vsq = 0.0;
    line_nsum<CPL, double>(ph, ns, lane);
    double lphi[CPL];
#pragma unroll
    for (int t = 0; t < CPL; ++t) lphi[t] = I.cx * ns[t] - I.dcoef * ph[t];
    line_nsum<CPL, double>(ld, ns, lane);
#pragma unroll
    for (int t = 0; t < CPL; ++t) {
      const bool valid = q0 + t < M;
      const double x = xd[t], lam = ld[t];
      const double xp = ws.f[L_XP][pb0 + t], rc = ws.f[L_RF][pb0 + t];
      const double ln = last ? I.hqf * (x - rc) : ws.f[L_LN][pb0 + t];
      const double mu = I.cx * ns[t] - I.dcoef * lam;
      const double dphi = I.k0 * (1.0 + I.k1 * x);
      double srcd = 0.0;  // controls on this cell
      for (int a = 0; a < nu; ++a)
        if (ws.act[a] == q0 + t) srcd += ws.u[a];
      const double t1 = I.h * (lphi[t] + srcd * I.b0);
      const double t3 = I.h * (I.q * (x - rc) + dphi * mu);
      const double K1d = xp - x + t1;
      const double K3d = ln - lam + t3;
      if (valid) {
        vmax = fmax(vmax, fmax(abs_or_inf(K1d), abs_or_inf(K3d)));
        vsq += K1d * K1d + K3d * K3d;
      }
      if constexpr (RBN) {
        K1[t] = to_T<T>(xpn[t] - x + t1);
        K3[t] = to_T<T>(last ? K3d : lnn[t] - lam + t3);
      } else {
        K1[t] = to_T<T>(K1d);
        K3[t] = to_T<T>(K3d);
      }
      dp[t] = to_T<T>(dphi);
      ax[t] = to_T<T>(I.h * (I.q + I.k0 * I.k1 * mu) + (last ? I.hqf : 0.0));
      rg[t] = valid ? rcp_T(-T(1) - th * tdc * dp[t]) : T(0);
    }
    // stage-gradient rows: lane a % 32 takes control a
    for (int a = lane; a < nu; a += 32) {
      const double K2 = I.h * (I.r * ws.u[a] + I.b0 * ws.lact[a]);
      vmax = fmax(vmax, abs_or_inf(K2));
      vsq += K2 * K2;
    }
    for (int o = 16; o > 0; o >>= 1) {
      vmax = dmax_nan(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      vsq += __shfl_xor_sync(0xffffffffu, vsq, o);
    }
    rmax = vmax;
    rsq = vsq;
  } else {
    // controls' sources on the lane's cells
    float srcf[CPL];
#pragma unroll
    for (int t = 0; t < CPL; ++t) srcf[t] = 0.0f;
    for (int a = 0; a < nu; ++a) {
      const int c = ws.act[a];
      if (c / CPL == lane) {
        const int tc = c & (CPL - 1);
#pragma unroll
        for (int t = 0; t < CPL; ++t)
          if (t == tc) srcf[t] += d2f(ws.u[a]);
      }
    }
    float xv[CPL], lv[CPL], ph[CPL], ns[CPL], lphi[CPL];
    float4 mg = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int t = 0; t < CPL; ++t) {
      xv[t] = d2f(ws.f[L_X][pb0 + t]);
      lv[t] = d2f(ws.f[L_L][pb0 + t]);
      ph[t] = I.fk0 * (xv[t] + I.fk1h * xv[t] * xv[t]);
      mg.x = fmaxf(mg.x, fabsf(xv[t]));
      mg.y = fmaxf(mg.y, fabsf(lv[t]));
    }
    line_nsum<CPL, float>(ph, ns, lane);
#pragma unroll
    for (int t = 0; t < CPL; ++t) lphi[t] = I.fcx * ns[t] - I.fdc * ph[t];
    line_nsum<CPL, float>(lv, ns, lane);
    float fm = 0.0f, fs = 0.0f;
    const float hqff = last ? I.fhqf : 0.0f;
#pragma unroll
    for (int t = 0; t < CPL; ++t) {
      const bool valid = q0 + t < M;
      const double x = ws.f[L_X][pb0 + t], lam = ws.f[L_L][pb0 + t];
      const double xp = ws.f[L_XP][pb0 + t];
      const float rv = d2f(ws.f[L_RF][pb0 + t]);
      const float mu = I.fcx * ns[t] - I.fdc * lv[t];
      const float dphi = I.fk0 * (1.0f + I.fk1 * xv[t]);
      const float t1 = I.fh * (lphi[t] + I.fb0 * srcf[t]);
      const float t3 = I.fh * (I.fq * (xv[t] - rv) + dphi * mu);
      // the O(1) differences in float64 (taken in float32 from truncated
      // values they would move in steps of 2^-23 |x|, and the split
      // iteration would stall at that scale above tight tolerances); at the
      // last stage lambda_{N+1} is h qf (x_N - ref), an O(h) term
      const double d3 = last ? -lam : ws.f[L_LN][pb0 + t] - lam;
      const float dx = d2f(xp - x), dl = d2f(d3);
      const float K1f = dx + t1;
      const float K3f = dl + t3 + (last ? hqff * (xv[t] - rv) : 0.0f);
      const float K1v = valid ? K1f : 0.0f, K3v = valid ? K3f : 0.0f;
      mg.z = fmaxf(mg.z, valid ? fmaxf(fabsf(dx), fabsf(dl)) : 0.0f);
      mg.w = fmaxf(mg.w, valid ? fabsf(rv) : 0.0f);
      fm = fmax_nan(fm, fmax_nan(fabsf(K1v), fabsf(K3v)));
      fs += K1v * K1v + K3v * K3v;
      if constexpr (RBN) {
        K1[t] = d2f(xpn[t] - x) + t1;
        K3[t] = last ? K3f : d2f(lnn[t] - lam) + t3;
      } else {
        K1[t] = K1f;
        K3[t] = K3f;
      }
      dp[t] = dphi;
      ax[t] = I.fh * (I.fq + I.fk01 * mu) + hqff;
      rg[t] = valid ? rcp_T(-T(1) - th * tdc * dp[t]) : T(0);
    }
    // stage-gradient rows: lane a % 32 takes control a
    for (int a = lane; a < nu; a += 32) {
      const double K2 = I.h * (I.r * ws.u[a] + I.b0 * ws.lact[a]);
      const float K2f = d2f(K2);
      fm = fmax_nan(fm, fabsf(K2f));
      fs += K2f * K2f;
      mg.z = fmaxf(mg.z, fabsf(K2f));
    }
    for (int o = 16; o > 0; o >>= 1) {
      fm = fmax_nan(fm, __shfl_xor_sync(0xffffffffu, fm, o));
      fs += __shfl_xor_sync(0xffffffffu, fs, o);
      mg.x = fmaxf(mg.x, __shfl_xor_sync(0xffffffffu, mg.x, o));
      mg.y = fmaxf(mg.y, __shfl_xor_sync(0xffffffffu, mg.y, o));
      mg.z = fmaxf(mg.z, __shfl_xor_sync(0xffffffffu, mg.z, o));
      mg.w = fmaxf(mg.w, __shfl_xor_sync(0xffffffffu, mg.w, o));
    }
    rmax = f2d(fm);
    rsq = f2d(fs);
    if (lane == 0) {
      const float mags[4] = {mg.x, mg.y, mg.z, mg.w};
      float usum = 0.0f;
      for (int a = 0; a < nu; ++a) usum += fabsf(d2f(ws.u[a]));
      e = split_bound(I, last, mags, usum);
    }
  }
  if (lane == 0) publish_residual(A, (k % RES_SLOTS) * A.n_inst + b, b, k, rmax, rsq, e, FULL);
  if (resid_only) return;

  // K1 at the control cells (the u-iteration's refresh), K2 (b3)
  for (int a = 0; a < nu; ++a) {
    const T k1a = line_at<CPL, T>(K1, ws.act[a]);
    if (lane == (a & 31)) {
      ws.b1[a] = k1a;
      ws.b3[a] = (T)(I.h * (I.r * ws.u[a] + I.b0 * ws.lact[a]));
      ws.v3[a] = T(0);
    }
  }
  __syncwarp();

  // ---- lower layer: n_u_it + 1 applications of P^{-1} ----
  const T auu = I.fauu;
  T v1[CPL], y5[CPL], y4[CPL], w1[CPL], ns[CPL];
#pragma unroll
  for (int t = 0; t < CPL; ++t) v1[t] = -K1[t] * rg[t];  // first F_x sweep (v3 = 0)
  const int n_lo = A.n_lo;
  for (int it = 0; it <= A.n_u_it; ++it) {
    if (it > 0) {
      // F_u v3 - K1 changes only on the control cells: refresh v1 there (the
      // first control on a cell carries the cell's total v3)
      for (int a = 0; a < nu; ++a) {
        const int c = ws.act[a];
        bool first = true;
        for (int a2 = 0; a2 < a; ++a2) first = first && (ws.act[a2] != c);
        if (!first || c / CPL != lane) continue;
        T inj = T(0);
        for (int a2 = 0; a2 < nu; ++a2)
          if (ws.act[a2] == c) inj += ws.v3[a2];
        const int tc = c & (CPL - 1);
#pragma unroll
        for (int t = 0; t < CPL; ++t)
          if (t == tc) v1[t] = (th * tb0 * inj - ws.b1[a]) * rg[t];
      }
    }
    // F_x v5 = F_u v3 - K1: sweep m + 1 = v1 - D^{-1} h (offdiag) (Phi' sweep m)
#pragma unroll
    for (int t = 0; t < CPL; ++t) y5[t] = v1[t];
    for (int sw = 1; sw < n_lo; ++sw) {
      T pw[CPL];
#pragma unroll
      for (int t = 0; t < CPL; ++t) pw[t] = dp[t] * y5[t];
      line_nsum<CPL, T>(pw, ns, lane);
#pragma unroll
      for (int t = 0; t < CPL; ++t) y5[t] = v1[t] - rg[t] * (th * (tcx * ns[t]));
    }
    // F_x^T v4 = -K3 - A_xx v5
#pragma unroll
    for (int t = 0; t < CPL; ++t) {
      w1[t] = (-K3[t] - ax[t] * y5[t]) * rg[t];
      y4[t] = w1[t];
    }
    for (int sw = 1; sw < n_lo; ++sw) {
      line_nsum<CPL, T>(y4, ns, lane);
#pragma unroll
      for (int t = 0; t < CPL; ++t) y4[t] = w1[t] - rg[t] * (th * dp[t] * (tcx * ns[t]));
    }
    if (it < A.n_u_it) {
      // A_uu v3 = K2 + F_u^T y_lambda (A_ux = 0)
      for (int a = 0; a < nu; ++a) {
        const T y = line_at<CPL, T>(y4, ws.act[a]);
        if (lane == (a & 31)) ws.v3[a] = (ws.b3[a] + th * tb0 * y) / auu;
      }
      __syncwarp();
    }
  }

  // ---- S_i <- S_i - alpha Delta s_i (float64), coalesced ----
  float* Y5 = reinterpret_cast<float*>(ws.f[L_XP]);
  float* Y4 = reinterpret_cast<float*>(ws.f[L_LN]);
#pragma unroll
  for (int t = 0; t < CPL; ++t) {
    Y5[pb0 + t] = y5[t];
    Y4[pb0 + t] = y4[t];
  }
  __syncwarp();
  const double alpha = A.alpha;
  double* Xo = A.xout[rd ^ 1] + so;
  double* Lo = A.lout[rd ^ 1] + so;
#pragma unroll
  for (int t = 0; t < CPL; ++t) {
    // every position q < 32 CPL exists (zeros past M): only the stores are
    // predicated
    const int q = t * 32 + lane;
    const int p = lpad<CPL>(q);
    const double xn = fma(alpha, f2d(Y5[p]), ws.f[L_X][p]);
    const double ln = fma(alpha, f2d(Y4[p]), ws.f[L_L][p]);
    if (q < M) {
      Xo[q] = xn;
      Lo[q] = ln;
    }
  }
  double* Uo = A.uout[rd ^ 1] + I.u_off + (long long)s * nu;
  for (int a = lane; a < nu; a += 32) Uo[a] = ws.u[a] - alpha * (double)ws.v3[a];
}

// One upper-layer iteration over the line work list (MODE_SOLVE: iteration
// *iter_k + j with the convergence bookkeeping, over the items of the
// instances running at the start of the chunk, compacted to the front of the
// list and followed by empty items; MODE_ONESHOT: one residual or iteration
// from the given buffers, over every item).  Item (b, s, CPL); one item per
// warp, warps on an empty item return at once.
template <bool RBN>
__global__ void __launch_bounds__(LINE_WARPS * 32, 4) k_line(IterArgs A, int MODE, int j_launch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  LineShared& ws = *reinterpret_cast<LineShared*>(
      smem_raw + warp * ((sizeof(LineShared) + 15) & ~size_t(15)));
  pdl_trigger();
  const int k = (MODE == MODE_SOLVE) ? *(volatile int*)A.iter_k + launch_iter(A, j_launch) : 0;
  const int half = launch_half(A, j_launch);
  const int rd = (MODE == MODE_SOLVE) ? (k & 1) : 0;
  pdl_wait();  // the previous iteration's state, residuals and control words
  const int item = blockIdx.x * LINE_WARPS + warp;
  if (item >= A.n_lines) return;  // warp-uniform; no block barriers in this kernel
  const int4* list = (MODE == MODE_SOLVE) ? A.lines_act : A.lines;
  const int4 it = list[item];
  if (it.x < 0) return;  // past the running items (solve mode)
  const int b = it.x, s = it.y, cpl = it.z;
  if (!stage_in_half(A, s, half)) return;

  bool resid_only, full;
  if (MODE == MODE_ONESHOT) {
    resid_only = (A.resid_only != 0);
    full = resid_only || (A.full_all != 0);
  } else {
    int skip = 0, fl = 1;
    if (lane == 0) {
      Cl cl;
      cl.C = 1;
      cl.rank = 0;  // one warp per stage: stage 0's warp keeps the books
      control_decision(A, b, s, k, cl, skip, fl);
    }
    skip = __shfl_sync(0xffffffffu, skip, 0);
    fl = __shfl_sync(0xffffffffu, fl, 0);
    if (skip) return;
    full = fl != 0;
    resid_only = (k == A.max_iter);
  }
  if (full) {
    switch (cpl) {
      case 1: line_body<1, true, RBN>(A, ws, lane, b, s, k, rd, resid_only); break;
      case 2: line_body<2, true, RBN>(A, ws, lane, b, s, k, rd, resid_only); break;
      case 4: line_body<4, true, RBN>(A, ws, lane, b, s, k, rd, resid_only); break;
      default: line_body<8, true, RBN>(A, ws, lane, b, s, k, rd, resid_only); break;
    }
  } else {
    switch (cpl) {
      case 1: line_body<1, false, RBN>(A, ws, lane, b, s, k, rd, resid_only); break;
      case 2: line_body<2, false, RBN>(A, ws, lane, b, s, k, rd, resid_only); break;
      case 4: line_body<4, false, RBN>(A, ws, lane, b, s, k, rd, resid_only); break;
      default: line_body<8, false, RBN>(A, ws, lane, b, s, k, rd, resid_only); break;
    }
  }
}

// The items of the line list whose instance is running, in list order (one
// CTA: per round of blockDim items, ballots and a prefix over the warps'
// counts), then empty items (instance -1) up to the list's length, and the
// running items' number.  Runs at the start of every chunk of solve
// iterations, so an instance that finishes inside a chunk keeps its items
// (its stage-0 warp records the finish) until the next chunk.
constexpr int COMPACT_THREADS = 1024;
__global__ void __launch_bounds__(COMPACT_THREADS) k_compact_lines(IterArgs A) {
  __shared__ int wofs[32];
  __shared__ int total;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int base = 0;  // every thread keeps the same running count
  for (int i0 = 0; i0 < A.n_lines; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    int4 it = make_int4(0, 0, 0, 0);
    bool keep = false;
    if (i < A.n_lines) {
      it = A.lines[i];
      keep = __ldcg(A.status + it.x) == ST_RUNNING;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wofs[w] = __popc(m);
    __syncthreads();
    if (w == 0) {
      const int c = (lane < nw) ? wofs[lane] : 0;
      int incl = c;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane < nw) wofs[lane] = incl - c;
      if (lane == 31) total = incl;
    }
    __syncthreads();
    if (keep) A.lines_act[base + wofs[w] + __popc(m & ((1u << lane) - 1u))] = it;
    base += total;
    __syncthreads();  // wofs and total are rewritten by the next round
  }
  for (int i = base + threadIdx.x; i < A.n_lines; i += blockDim.x)
    A.lines_act[i] = make_int4(-1, 0, 0, 0);
  if (threadIdx.x == 0) *A.n_lines_act = base;
}

// Persistent solve over the line list (Jacobi upper layer): in every
// iteration k = *iter_k .. max_iter the resident CTAs' warps claim items of
// the whole list from a per-iteration counter (an item of a finished
// instance costs one control read), with a grid barrier between iterations
// (one arrival per CTA; the last arrival clears the next iteration's counter
// and ends the launch when no instance is running).  Its own inlined copy of
// the stage body, so its float32 arithmetic may differ from k_line's by the
// compiler's multiply-add contraction (rounding level).  A barrier wait longer than A.grid_wait cycles raises
// the error word gsync[3] and ends the launch; the host then restarts the
// solve with one launch per iteration.  Launched cooperatively with at most
// the resident number of CTAs.
constexpr int LINE_CLAIM = 1;  // items per claim of the persistent line launch (larger claims balance worse)

__global__ void __launch_bounds__(LINE_WARPS * 32, 4) k_line_solve(IterArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int bar_code;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  LineShared& ws = *reinterpret_cast<LineShared*>(
      smem_raw + warp * ((sizeof(LineShared) + 15) & ~size_t(15)));
  unsigned* ctr = A.gsync + 4;  // item counters, one per iteration parity
  unsigned gen = 0u;
  if (threadIdx.x == 0) gen = ld_acquire_u32(&A.gsync[1]);
  for (int k = *(volatile int*)A.iter_k; k <= A.max_iter; ++k) {
    const int rd = k & 1;
    for (;;) {
      // claim LINE_CLAIM consecutive items; their lanes read the instances'
      // status at once, and the warp runs the items of running instances
      int base = 0;
      if (lane == 0) base = (int)atomicAdd(&ctr[k & 1], (unsigned)LINE_CLAIM);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= A.n_lines) break;
      int4 mine = make_int4(-1, 0, 0, 0);
      bool run = false;
      if (lane < LINE_CLAIM && base + lane < A.n_lines) {
        mine = A.lines[base + lane];
        run = __ldcg(A.status + mine.x) == ST_RUNNING;
      }
      unsigned m = __ballot_sync(0xffffffffu, run);
      while (m) {
        const int l = __ffs(m) - 1;
        m &= m - 1u;
        const int b = __shfl_sync(0xffffffffu, mine.x, l);
        const int s = __shfl_sync(0xffffffffu, mine.y, l);
        const int cpl = __shfl_sync(0xffffffffu, mine.z, l);
        int skip = 0, fl = 1;
        if (lane == 0) {
          Cl cl;
          cl.C = 1;
          cl.rank = 0;  // one warp per stage: stage 0's warp keeps the books
          control_decision(A, b, s, k, cl, skip, fl);
        }
        skip = __shfl_sync(0xffffffffu, skip, 0);
        fl = __shfl_sync(0xffffffffu, fl, 0);
        if (skip) continue;
        const bool resid_only = (k == A.max_iter);
        if (fl) {
          switch (cpl) {
            case 1: line_body<1, true, false>(A, ws, lane, b, s, k, rd, resid_only); break;
            case 2: line_body<2, true, false>(A, ws, lane, b, s, k, rd, resid_only); break;
            case 4: line_body<4, true, false>(A, ws, lane, b, s, k, rd, resid_only); break;
            default: line_body<8, true, false>(A, ws, lane, b, s, k, rd, resid_only); break;
          }
        } else {
          switch (cpl) {
            case 1: line_body<1, false, false>(A, ws, lane, b, s, k, rd, resid_only); break;
            case 2: line_body<2, false, false>(A, ws, lane, b, s, k, rd, resid_only); break;
            case 4: line_body<4, false, false>(A, ws, lane, b, s, k, rd, resid_only); break;
            default: line_body<8, false, false>(A, ws, lane, b, s, k, rd, resid_only); break;
          }
        }
      }
    }
    // grid barrier: the CTA's warps meet (after publishing their global
    // writes), thread 0 arrives, the last arrival decides whether to stop
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      unsigned* gs = A.gsync;
      const unsigned target = gen + 1u;
      if (atomicAdd(&gs[0], 1u) == gridDim.x - 1u) {
        gs[0] = 0u;
        ctr[(k + 1) & 1] = 0u;  // every claim of iteration k - 1 is done
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
      bar_code = (int)(ld_acquire_u32(&gs[2]) | (ld_acquire_u32(&gs[3]) << 1));
      gen = target;
    }
    __syncthreads();
    if (bar_code != 0) break;
  }
}
