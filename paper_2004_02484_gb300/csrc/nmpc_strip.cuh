// Strip path of the upper-layer iteration for large 2D stages (included from
// nmpc_kernels.cuh inside namespace nmpc_dev, after nmpc_patch.cuh).
//
// One warp of k_strip computes one strip of one (instance, stage) work item
// of iteration k: 32 - 2E own columns (lane = region column, E = 2 n_lo - 1
// on each side) and a run of own rows, from a region extended by E rows above
// and below.  The warp walks down the region's rows; at step j, pass m works
// on row j - m:
//   pass 0       the stencil inputs Phi(x), lambda of row j;
//   pass 1       K_i (eq. 9), Phi'(x), A_xx, 1/diag F_x and the first F_x
//                sweep of row j - 1;
//   pass 2..n_lo the F_x sweeps of P^{-1} (eq. 24), the last one also the
//                first F_x^T sweep;
//   pass n_lo+1..E the F_x^T sweeps; pass E updates the own cells of row
//                j - E (S <- S + alpha Y, eq. 15, float64).
// A pass reads its stencil neighbours from the previous pass: the rows above
// and below from a three-row register window, the columns left and right by
// warp shuffles.  Cells at level < m of pass m (lanes or rows near the
// region's border) hold values no own cell depends on.  Cells outside the
// grid carry 1/diag F_x = 0, so every sweep is zero there (the Dirichlet
// ring).  Inputs arrive by asynchronous copies into a four-row ring in
// shared memory, two rows ahead.  No block barrier and no shared-memory
// stencil traffic.  The actuators' v3 come from k_patch (same iteration).

constexpr int STRIP_WARPS = 4;  // warps (strips) per CTA
constexpr int STRIP_AHEAD = 2;  // rows copied ahead
// CTAs per SM the register allocation must allow (4 warps each)
#ifndef STRIP_MIN_BLOCKS
#define STRIP_MIN_BLOCKS 5
#endif

// An actuator inside a strip's region: region row, lane, control index.
struct StripAct {
  int row, lane, a, pad;
};

// Rows of a warp's input ring: from the row pass E updates (j - E) to the
// row being copied (j + STRIP_AHEAD), so the update reads x, lambda from
// shared memory.
__host__ __device__ constexpr int strip_ring_rows(int n_lo) {
  return 2 * n_lo - 1 + STRIP_AHEAD + 1;
}

// Shared memory of one strip warp: the input rings (float64, 32 lanes) and
// the actuators in reach sorted by row.  x_i and lambda_i stay RING rows
// (the update of row j - E reads them); the fields only pass 1 reads
// (x_{i-1}, lambda_{i+1}, ref, and for red-black half 1 x_{i-1}, lambda_{i+1}
// as updated by half 0) need rows j - 1 .. j + 2 only: a ring of
// STRIP_AHEAD + 2 rows with NF = 3 or 5 fields.
enum { RB_X = 0, RB_L = 1 };                                      // RING rows
enum { RS_XP = 0, RS_LN = 1, RS_RF = 2, RS_XPN = 3, RS_LNN = 4 };  // short ring
constexpr int STRIP_SHORT = STRIP_AHEAD + 2;
static_assert((STRIP_SHORT & (STRIP_SHORT - 1)) == 0, "the short ring is indexed by j & (rows - 1)");
__host__ __device__ constexpr int strip_fields(bool rbn) { return rbn ? 5 : 3; }
template <int RING, int NF = 3>
struct StripShared {
  double ring[RING * 2 * 32];
  double sring[STRIP_SHORT * NF * 32];
  StripAct act[MAX_NU];
  int n_act;
};

// A three-row window of a stencil field: w0 = row above, w1 = centre,
// w2 = row below the consumer's row.
template <typename V>
struct Win {
  V w0, w1, w2;
  __device__ __forceinline__ void push(V v) {
    w0 = w1;
    w1 = w2;
    w2 = v;
  }
  // centre's horizontal neighbours plus the vertical ones, weighted
  __device__ __forceinline__ V nsum(V cx, V cy) const {
    const V l = __shfl_up_sync(0xffffffffu, w1, 1), r = __shfl_down_sync(0xffffffffu, w1, 1);
    return cx * (l + r) + cy * (w0 + w2);
  }
};

// Shift register of per-row values: at step j, d[k] holds the value pass 1
// formed k + 1 steps earlier (row j - 2 - k).
template <typename V, int D>
struct Shift {
  V d[D > 0 ? D : 1];
  __device__ __forceinline__ void push(V v) {
    if constexpr (D > 0) {
#pragma unroll
      for (int k = D - 1; k > 0; --k) d[k] = d[k - 1];
      d[0] = v;
    }
  }
};

// The strip of work item (b, s, x0, y0) for one residual form (FULL: the
// float64 residual; else the split one): a separate instantiation per form,
// so neither form's arithmetic is issued in the other's iterations.  RBN:
// red-black half 1 (the right-hand side takes x_{i-1}, lambda_{i+1} as
// updated by half 0; the norms stay those of K(S^k)).  GSN: red-black half 1
// in the split form of a solve, where the norms are only the trigger of the
// float64 residual: x_{i-1}, lambda_{i+1} as updated by half 0 serve both the
// right-hand side and the norms (the Gauss-Seidel residual K_i of the
// half-updated iterate), so the values of iterate k at the neighbours are
// not read.
template <typename T, int n_lo, bool FULL, bool RBN, bool GSN = false>
__device__ __forceinline__ void strip_body(const IterArgs& A,
                                           StripShared<strip_ring_rows(n_lo), strip_fields(RBN)>& ws,
                                           int lane, int b, int s, int k, int rd, int x0, int y0,
                                           bool resid_only) {
  constexpr int E = 2 * n_lo - 1;
  constexpr int RING = strip_ring_rows(n_lo);
  constexpr int NF = strip_fields(RBN);
  constexpr bool full = FULL;
  const InstDev& I = A.inst[b];
  const int nu = I.nu;
  const bool last = (s == I.N - 1);
  const long long so = I.s_off + (long long)s * I.ng;
  // region: columns x0 - E + lane, rows y0 - E .. y0 + own_rows + E - 1
  const int own_rows = min(A.strip_y, I.my - y0);
  const int RH = own_rows + 2 * E;
  const int gx = x0 - E + lane;
  const bool gx_ok = gx >= 0 && gx < I.mx;
  const bool own_lane = lane >= E && lane < 32 - E && gx_ok;
  const int gy0 = y0 - E;

  // actuators in reach, sorted by (row, lane, index): lane l looks at
  // actuators l and l + 32 (n_u <= 64), each candidate's rank is the number
  // of smaller keys across the warp
  {
    const float inv_mx = 1.0f / (float)I.mx;
    long long key[2];
    int rr[2], rl[2];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int a = lane + 32 * h2;
      key[h2] = 0x7fffffffffffffffLL;
      rr[h2] = rl[h2] = 0;
      if (a < nu) {
        const int c = A.act[I.act_off + a];
        const int cy = fdiv(c, I.mx, inv_mx), cx = c - cy * I.mx;
        rl[h2] = cx - (x0 - E);
        rr[h2] = cy - gy0;
        if (rl[h2] >= 0 && rl[h2] < 32 && rr[h2] >= 0 && rr[h2] < RH)
          key[h2] = ((long long)rr[h2] * 32 + rl[h2]) * MAX_NU + a;
      }
    }
    int rank[2] = {0, 0};
    for (int l = 0; l < 32; ++l) {
      const long long k0 = __shfl_sync(0xffffffffu, key[0], l);
      const long long k1 = __shfl_sync(0xffffffffu, key[1], l);
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) rank[h2] += (k0 < key[h2]) + (k1 < key[h2]);
    }
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2)
      if (key[h2] != 0x7fffffffffffffffLL)
        ws.act[rank[h2]] = StripAct{rr[h2], rl[h2], lane + 32 * h2, 0};
    const int n = __popc(__ballot_sync(0xffffffffu, key[0] != 0x7fffffffffffffffLL)) +
                  __popc(__ballot_sync(0xffffffffu, key[1] != 0x7fffffffffffffffLL));
    if (lane == 0) ws.n_act = n;
  }
  __syncwarp();
  const int n_act = ws.n_act;
  int na = 0;  // next actuator entry (rows increase along the strip; all rows >= 0)
  int next_row = n_act > 0 ? ws.act[0].row : 0x7fffffff;

  // asynchronous copies of region row rj into its ring slot (zero outside the grid)
  const double* Xg = A.xin[rd] + so;
  const double* Lg = A.lin[rd] + so;
  const double* XPg = (s == 0) ? A.x0 + I.g_off : (GSN ? A.xout[rd ^ 1] : A.xin[rd]) + so - I.ng;
  const double* LNg = (GSN ? A.lout[rd ^ 1] : A.lin[rd]) + so + I.ng;
  const double* RFg = A.ref + I.g_off;
  const double* XPNg = (s == 0) ? A.x0 + I.g_off : A.xout[rd ^ 1] + so - I.ng;
  const double* LNNg = A.lout[rd ^ 1] + so + I.ng;
  double* ring = ws.ring + lane;
  // the short ring follows the long one in the same structure: addressed
  // from the same base (no second pointer register)
  using SS = StripShared<RING, NF>;
  static_assert(offsetof(SS, sring) == offsetof(SS, ring) + sizeof(double) * RING * 2 * 32,
                "short ring right after the long one");
  // ring row of j + d for the current step j (sj = j mod RING), -RING < d < RING
  int sj = 0;
  auto slot_at = [&](int d, int f) -> double* {
    int q = sj + d;
    q = q < 0 ? q + RING : (q >= RING ? q - RING : q);
    return ring + (q * 2 + f) * 32;
  };
  // short-ring row of region row r (any r >= -1: rows j - 1 .. j + 2 of step j)
  auto sslot_row = [&](int r, int f) -> double* {
    return ring + RING * 2 * 32 + (((r + STRIP_SHORT) & (STRIP_SHORT - 1)) * NF + f) * 32;
  };
  // row rj's five inputs; cells outside the grid and rows past the region
  // are zero-filled by the copies themselves (source size 0, from a clamped
  // address inside the grid)
  const int gxc = min(max(gx, 0), I.mx - 1);
  const int mx = I.mx, my = I.my;
  // row rj = j + dj of the current step j
  auto fetch = [&](int rj, int dj) {
    const int gy = gy0 + rj;
    const bool ok = gx_ok && gy >= 0 && gy < my && rj < RH;
    const int c = min(max(gy, 0), my - 1) * mx + gxc;
    double* d = slot_at(dj, 0);
    double* e = sslot_row(rj, 0);
    cp_async8_zfill(d + RB_X * 32, Xg + c, ok);
    cp_async8_zfill(d + RB_L * 32, Lg + c, ok);
    cp_async8_zfill(e + RS_XP * 32, XPg + c, ok);
    cp_async8_zfill(e + RS_LN * 32, (last ? Lg : LNg) + c, ok && !last);
    cp_async8_zfill(e + RS_RF * 32, RFg + c, ok);
    if constexpr (RBN) {
      cp_async8_zfill(e + RS_XPN * 32, XPNg + c, ok);
      cp_async8_zfill(e + RS_LNN * 32, (last ? Lg : LNNg) + c, ok && !last);
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
#pragma unroll
  for (int q = 0; q < STRIP_AHEAD; ++q) fetch(q, q);  // before step 0 (sj = 0)

  const T th = pick<T>(I.h, I.fh), tdc = pick<T>(I.dcoef, I.fdc), tb0 = pick<T>(I.b0, I.fb0);
  const T tcx = pick<T>(I.cx, I.fcx), tcy = pick<T>(I.cy, I.fcy);
  const double alpha = A.alpha;
  double* __restrict__ Xo = A.xout[rd ^ 1] + so;
  double* __restrict__ Lo = A.lout[rd ^ 1] + so;
  const double* Lin = Lg;
  // the instance's constants in registers (the loop's stores could alias the
  // descriptor table as far as the compiler knows)
  const double cxd = I.cx, cyd = I.cy, dcd = I.dcoef, hd = I.h, k0d = I.k0, k1d = I.k1;
  const double qd = I.q, b0d = I.b0, hqfd = I.hqf;
  const float fcx = I.fcx, fcy = I.fcy, fdc = I.fdc, fh = I.fh, fk0 = I.fk0, fk1 = I.fk1;
  const float fk1h = I.fk1h, fq = I.fq, fb0 = I.fb0, fk01 = I.fk01;
  const float hqff = last ? I.fhqf : 0.0f;
  const double* uin_s = A.uin[rd] + I.u_off + (long long)s * nu;
  const double* v3_s = A.v3g + I.u_off + (long long)s * nu;

  Norms nm{0.0f, 0.0f, make_float4(0.f, 0.f, 0.f, 0.f), 0.0, 0.0, 0.0f};
  // pass 0 windows (float64 in the full residual, float32 in the split one)
  Win<double> phd{0.0, 0.0, 0.0}, lad{0.0, 0.0, 0.0};
  Win<float> laf{0.f, 0.f, 0.f}, xvf{0.f, 0.f, 0.f};
  // sweep fields: pw[m] is the window of pass m + 1's output (m = 0 .. E - 2)
  Win<T> pw[E > 1 ? E - 1 : 1];
#pragma unroll
  for (int m = 0; m < (E > 1 ? E - 1 : 1); ++m) pw[m] = Win<T>{T(0), T(0), T(0)};
  // per-row values of pass 1 for the later passes
  Shift<T, E - 1> sdp, srg;        // Phi', 1/diag F_x  (passes 2 .. E)
  Shift<T, n_lo - 1> sk3, sax, sv1;  // K3, A_xx, v1     (passes 2 .. n_lo)
  Shift<T, n_lo - 1> sv5, sw1;     // v5, w1 of pass n_lo (passes n_lo + 1 .. E)

  const int steps = RH + E;
  for (int j = 0; j < steps; ++j) {
    fetch(j + STRIP_AHEAD, STRIP_AHEAD);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(STRIP_AHEAD));
    // ---- pass 0: row j ----
    {
      const double x = *slot_at(0, RB_X), l = *slot_at(0, RB_L);
      if constexpr (full) {
        phd.push(k0d * (x + 0.5 * k1d * x * x));
        lad.push(l);
      } else {
        const float xv = d2f(x), lf = d2f(l);
        laf.push(lf);
        xvf.push(xv);
        if (j < RH) {
          nm.mg.x = fmaxf(nm.mg.x, fabsf(xv));
          nm.mg.y = fmaxf(nm.mg.y, fabsf(lf));
        }
      }
    }
    // ---- pass 1: row j - 1 ----
    T K3 = T(0), ax = T(0), rg = T(0), dp = T(0), v1 = T(0);
    {
      const int rj = j - 1;
      const int gy = gy0 + rj;
      const bool in_grid = gx_ok && gy >= 0 && gy < my;
      const bool own = own_lane && rj >= E && rj < RH - E && gy < my;
      // sources of the cell: sum of u (b0 B u in K1) and of v3 (F_u v3)
      double srcd = 0.0;
      float srcf = 0.0f;
      T inj = T(0);
      if (rj == next_row) {  // warp-uniform
        while (na < n_act && ws.act[na].row == rj) {
          const StripAct e = ws.act[na];
          if (e.lane == lane) {
            const double ua = uin_s[e.a];
            if constexpr (full) srcd += ua;
            else srcf += d2f(ua);
            inj += (T)v3_s[e.a];
          }
          ++na;
        }
        next_row = na < n_act ? ws.act[na].row : 0x7fffffff;
      }
      const double* rs = slot_at(-1, 0);
      const double* qs = sslot_row(j - 1, 0);
      const double x = rs[RB_X * 32], lam = rs[RB_L * 32], xp = qs[RS_XP * 32], rc = qs[RS_RF * 32];
      T K1;
      if constexpr (full) {
        const double ln = last ? hqfd * (x - rc) : qs[RS_LN * 32];
        const double lphi = phd.nsum(cxd, cyd) - dcd * phd.w1;
        const double mu = lad.nsum(cxd, cyd) - dcd * lad.w1;
        const double dphi = k0d * (1.0 + k1d * x);
        const double t1 = hd * (lphi + b0d * srcd);
        const double t3 = hd * (qd * (x - rc) + dphi * mu);
        const double K1d = xp - x + t1;
        const double K3d = ln - lam + t3;
        if (own) {
          nm.vmax = fmax(nm.vmax, fmax(abs_or_inf(K1d), abs_or_inf(K3d)));
          nm.vsq += K1d * K1d + K3d * K3d;
        }
        if constexpr (RBN) {
          K1 = to_T<T>(qs[RS_XPN * 32] - x + t1);
          K3 = to_T<T>(last ? K3d : qs[RS_LNN * 32] - lam + t3);
        } else {
          K1 = to_T<T>(K1d);
          K3 = to_T<T>(K3d);
        }
        dp = to_T<T>(dphi);
        ax = to_T<T>(hd * (qd + k0d * k1d * mu) + (last ? hqfd : 0.0));
      } else {
        // Lap Phi(x) in difference form, sum_n c_n k0 (x_n - x_c)(1 + k1/2
        // (x_n + x_c)): no cancellation of the O(dcoef Phi) terms, so its
        // rounding bound scales with the neighbour differences
        const float xv = xvf.w1, rv = d2f(rc);
        const float xl = __shfl_up_sync(0xffffffffu, xv, 1), xr = __shfl_down_sync(0xffffffffu, xv, 1);
        const float dlx = xl - xv, drx = xr - xv, dux = xvf.w0 - xv, ddx = xvf.w2 - xv;
        const float lphi =
            fk0 * (fcx * (dlx * (1.0f + fk1h * (xl + xv)) + drx * (1.0f + fk1h * (xr + xv))) +
                   fcy * (dux * (1.0f + fk1h * (xvf.w0 + xv)) + ddx * (1.0f + fk1h * (xvf.w2 + xv))));
        const float mu = laf.nsum(fcx, fcy) - fdc * laf.w1;
        const float dphi = fk0 * (1.0f + fk1 * xv);
        const float t1 = fh * (lphi + fb0 * srcf);
        const float t3 = fh * (fq * (xv - rv) + dphi * mu);
        // the O(1) differences in float32 from the truncated values (the
        // float64 pipe issues 2 lanes per clock per SM; their rounding enters
        // the bound, and the float64 residual certifies convergence); at the
        // last stage lambda_{N+1} = h qf (x_N - ref) is an O(h) term
        const float xpf = d2f(xp), lnf = last ? 0.0f : d2f(qs[RS_LN * 32]);
        const float dx = xpf - xv, dl = lnf - laf.w1;
        const float K1f = dx + t1;
        const float K3f = dl + t3 + hqff * (xv - rv);
        const float K1v = own ? K1f : 0.0f, K3v = own ? K3f : 0.0f;
        nm.gm = fmaxf(nm.gm, own ? fmaxf(fmaxf(fabsf(dlx), fabsf(drx)), fmaxf(fabsf(dux), fabsf(ddx)))
                                 : 0.0f);
        nm.mg.x = fmaxf(nm.mg.x, own ? fabsf(xpf) : 0.0f);
        nm.mg.y = fmaxf(nm.mg.y, own ? fabsf(lnf) : 0.0f);
        nm.mg.z = fmaxf(nm.mg.z, own ? fmaxf(fabsf(dx), fabsf(dl)) : 0.0f);
        nm.mg.w = fmaxf(nm.mg.w, own ? fabsf(rv) : 0.0f);
        nm.fmax = fmax_nan(nm.fmax, fmax_nan(fabsf(K1v), fabsf(K3v)));
        nm.fsq += K1v * K1v + K3v * K3v;
        if constexpr (RBN) {
          K1 = (T)((d2f(qs[RS_XPN * 32]) - xv) + t1);
          K3 = last ? (T)K3f : (T)((d2f(qs[RS_LNN * 32]) - laf.w1) + t3);
        } else {
          K1 = (T)K1f;
          K3 = (T)K3f;
        }
        dp = (T)dphi;
        ax = (T)(fh * (fq + fk01 * mu) + hqff);
      }
      // 1/diag F_x, zero outside the grid (every sweep there stays zero)
      rg = in_grid ? rcp_T(-T(1) - th * tdc * dp) : T(0);
      v1 = (th * tb0 * inj - K1) * rg;  // first F_x sweep of F_x v5 = F_u v3 - K1
    }
    if (!resid_only) {
      if constexpr (n_lo == 1) {
        // pass 1 is the last pass: v5 = v1, v4 = w1
        const int rj = j - 1;
        const int gy = gy0 + rj;
        if (own_lane && rj >= E && rj < RH - E && gy < my) {
          const int c = gy * mx + gx;
          const T w = (-K3 - ax * v1) * rg;
          const double* rs = slot_at(-1, 0);
          Xo[c] = fma(alpha, to_double(v1), rs[RB_X * 32]);
          Lo[c] = fma(alpha, to_double(w), rs[RB_L * 32]);
        }
      } else {
        // ---- pass 1's output: the first F_x sweep's field (or w1 for n_lo = 1) ----
        pw[0].push(dp * v1);
        // ---- passes 2 .. n_lo: F_x sweeps of row j - m ----
        T v5n = T(0), w1n = T(0);
#pragma unroll
        for (int m = 2; m <= n_lo; ++m) {
          // row j - m: pass 1 values of m - 1 steps ago
          const T dpm = sdp.d[m - 2], rgm = srg.d[m - 2], v1m = sv1.d[m - 2];
          const T off = th * pw[m - 2].nsum(tcx, tcy);
          const T v = v1m - rgm * off;
          if (m < n_lo) {
            pw[m - 1].push(dpm * v);
          } else {
            const T w = (-sk3.d[m - 2] - sax.d[m - 2] * v) * rgm;
            v5n = v;
            w1n = w;
            pw[m - 1].push(w);
          }
        }
        // ---- passes n_lo + 1 .. E: F_x^T sweeps of row j - m ----
#pragma unroll
        for (int m = n_lo + 1; m <= E; ++m) {
          const T dpm = sdp.d[m - 2], rgm = srg.d[m - 2];
          const T w1m = sw1.d[m - n_lo - 1];
          const T off = th * dpm * pw[m - 2].nsum(tcx, tcy);
          const T v4 = w1m - rgm * off;
          if (m < E) {
            pw[m - 1].push(v4);
          } else {
            // ---- update of the own cells of row j - E ----
            const int rj = j - E;
            const int gy = gy0 + rj;
            if (own_lane && rj >= E && rj < RH - E && gy < my) {
              const int c = gy * mx + gx;
              const T v5m = sv5.d[E - n_lo - 1];
              const double* rs = slot_at(-E, 0);  // still in the ring
              Xo[c] = fma(alpha, to_double(v5m), rs[RB_X * 32]);
              Lo[c] = fma(alpha, to_double(v4), rs[RB_L * 32]);
            }
          }
        }
        sv5.push(v5n);
        sw1.push(w1n);
      }
    }
    sdp.push(dp);
    srg.push(rg);
    sk3.push(K3);
    sax.push(ax);
    sv1.push(v1);
    sj = (sj + 1 == RING) ? 0 : sj + 1;
  }
  asm volatile("cp.async.wait_all;\n" ::);

  // u rows (K2) and updates of the actuators whose cell is an own cell
  for (int e = 0; e < n_act; ++e) {
    const StripAct a = ws.act[e];
    const int gy = gy0 + a.row;
    if (a.lane != lane || !own_lane || a.row < E || a.row >= RH - E || gy >= I.my) continue;
    const double ua = A.uin[rd][I.u_off + (long long)s * nu + a.a];
    const double K2 = I.h * (I.r * ua + I.b0 * Lin[gy * I.mx + gx]);
    if constexpr (full) {
      nm.vmax = fmax(nm.vmax, abs_or_inf(K2));
      nm.vsq += K2 * K2;
    } else {
      const float K2f = d2f(K2);
      nm.fmax = fmax_nan(nm.fmax, fabsf(K2f));
      nm.fsq += K2f * K2f;
      nm.mg.z = fmaxf(nm.mg.z, fabsf(K2f));
    }
    if (!resid_only)
      A.uout[rd ^ 1][I.u_off + (long long)s * nu + a.a] =
          ua - alpha * (double)(T)A.v3g[I.u_off + (long long)s * nu + a.a];
  }
  // warp reduction of the norms, then one publication per strip
  double rmax, rsq;
  float mags[4];
  if constexpr (full) {
    double vm = nm.vmax, vs = nm.vsq;
    for (int o = 16; o > 0; o >>= 1) {
      vm = dmax_nan(vm, __shfl_xor_sync(0xffffffffu, vm, o));
      vs += __shfl_xor_sync(0xffffffffu, vs, o);
    }
    rmax = vm;
    rsq = vs;
  } else {
    float fm = nm.fmax, fs = nm.fsq, gm = nm.gm;
    float4 mg = nm.mg;
    for (int o = 16; o > 0; o >>= 1) {
      gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
      fm = fmax_nan(fm, __shfl_xor_sync(0xffffffffu, fm, o));
      fs += __shfl_xor_sync(0xffffffffu, fs, o);
      mg.x = fmaxf(mg.x, __shfl_xor_sync(0xffffffffu, mg.x, o));
      mg.y = fmaxf(mg.y, __shfl_xor_sync(0xffffffffu, mg.y, o));
      mg.z = fmaxf(mg.z, __shfl_xor_sync(0xffffffffu, mg.z, o));
      mg.w = fmaxf(mg.w, __shfl_xor_sync(0xffffffffu, mg.w, o));
    }
    rmax = f2d(fm);
    rsq = f2d(fs);
    mags[0] = mg.x;
    mags[1] = mg.y;
    mags[2] = mg.z;
    mags[3] = mg.w;
    nm.gm = gm;
  }
  if (lane == 0) {
    const int slot_k = (k % RES_SLOTS) * A.n_inst + b;
    double e = 0.0;
    if constexpr (!full) {
      float usum = 0.0f;
      for (int a = 0; a < nu; ++a) usum += fabsf(d2f(A.uin[rd][I.u_off + (long long)s * nu + a]));
      e = split_bound(I, last, mags, usum, true, nm.gm);
    }
    publish_residual(A, slot_k, b, k, rmax, rsq, e, full);
  }
}

// One upper-layer iteration over the strip work list (MODE_SOLVE: iteration
// *iter_k + j with the convergence bookkeeping; MODE_ONESHOT: one residual or
// iteration from the given buffers), after k_patch of the same iteration.
template <typename T, int n_lo, bool RBN>
__global__ void __launch_bounds__(STRIP_WARPS * 32, STRIP_MIN_BLOCKS) k_strip(IterArgs A, int MODE, int j_launch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  using WS = StripShared<strip_ring_rows(n_lo), strip_fields(RBN)>;
  using WS3 = StripShared<strip_ring_rows(n_lo), strip_fields(false)>;  // fits in WS
  unsigned char* wbase = smem_raw + warp * ((sizeof(WS) + 15) & ~size_t(15));
  WS& ws = *reinterpret_cast<WS*>(wbase);
  pdl_trigger();
  const int k = (MODE == MODE_SOLVE) ? *(volatile int*)A.iter_k + launch_iter(A, j_launch) : 0;
  const int half = launch_half(A, j_launch);
  const int rd = (MODE == MODE_SOLVE) ? (k & 1) : 0;
  pdl_wait();  // the previous iteration's state, residuals and control words; this one's v3
  const int item = ((A.rb && half) ? A.n_strips_even : 0) + blockIdx.x * STRIP_WARPS + warp;
  const int item_end = A.rb ? (half ? A.n_strips : A.n_strips_even) : A.n_strips;
  if (item >= item_end) return;  // warp-uniform; no block barriers in this kernel
  const int4 it = A.strips[item];
  const int b = it.x, s = it.y, x0 = it.z, y0 = it.w;
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
      cl.rank = (x0 == 0 && y0 == 0) ? 0 : 1;  // the stage's first strip keeps the books
      control_decision(A, b, s, k, cl, skip, fl);
    }
    skip = __shfl_sync(0xffffffffu, skip, 0);
    fl = __shfl_sync(0xffffffffu, fl, 0);
    if (skip) return;
    full = fl != 0;
    resid_only = (k == A.max_iter);
  }
  if (full || std::is_same<T, double>::value)
    strip_body<T, n_lo, true, RBN>(A, ws, lane, b, s, k, rd, x0, y0, resid_only);
  else if (RBN && MODE == MODE_SOLVE)
    strip_body<T, n_lo, false, false, true>(A, *reinterpret_cast<WS3*>(wbase), lane, b, s, k, rd,
                                            x0, y0, resid_only);
  else
    strip_body<T, n_lo, false, RBN>(A, ws, lane, b, s, k, rd, x0, y0, resid_only);
}
#include "nmpc_strip2.cuh"
