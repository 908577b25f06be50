// Strip path with two grid columns per lane (included from nmpc_strip.cuh
// inside namespace nmpc_dev): the same computation as k_strip (residual,
// coefficient fields, the lower layer's sweeps and the update pipelined down
// a strip's rows in registers, see nmpc_strip.cuh), for the mixed-precision
// path with n_lo <= 2, on 64-column regions: lane l holds region columns 2l
// and 2l + 1, and the float32 arithmetic of a column pair runs as packed
// .f32x2 instructions.  A region of 64 columns keeps 64 - 2P of them as own
// columns (P = 2 n_lo >= E + 1 on each side, even so that column pairs are
// 16-byte aligned), against 32 - 2E in k_strip: 56 of 64 for n_lo = 2
// instead of 26 of 32.  Stencil neighbours across a lane boundary come from
// one shuffle per field (the left neighbour of column 2l is lane l - 1's
// second column, the right neighbour of column 2l + 1 lane l + 1's first);
// the inputs arrive as 16-byte asynchronous copies of column pairs (a pair
// is entirely inside or outside the grid: even grid width, even region
// origin) and the update stores column pairs.
//
// Requirements checked by the host: float32 lower layer, n_lo <= 2, every
// strip instance with an even grid width and even offsets of its state and
// x0 / ref arrays (16-byte aligned pairs).

constexpr int STRIP2_WARPS = 4;  // warps (strips) per CTA
#ifndef STRIP2_MIN_BLOCKS
#define STRIP2_MIN_BLOCKS 3
#endif

// left / right region padding of the two-column strips: E + 1 (E odd)
__host__ __device__ constexpr int strip2_pad(int n_lo) { return 2 * n_lo; }

// Packed float32 pairs: .f32x2 arithmetic (round to nearest per component).
struct __align__(8) F2 {
  float x, y;
};
__device__ __forceinline__ unsigned long long f2_bits(F2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ F2 f2_from(unsigned long long r) {
  F2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(d);
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(d);
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(d);
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
  return f2_from(d);
}
__device__ __forceinline__ F2 bc2(float v) { return F2{v, v}; }
__device__ __forceinline__ F2 sel2(bool p, F2 a, F2 b) { return p ? a : b; }
__device__ __forceinline__ F2 d2f2(double2 v) { return F2{d2f(v.x), d2f(v.y)}; }

// float -> double for the update's increments in a few integer operations (no
// subnormal or Inf/NaN cases): exact for normal floats and +-0; a subnormal
// maps to within 2^-125 of its value; Inf and NaN map to finite values of
// magnitude 2^128 and more, which the next residual reads as infinite
// (divergence).
__device__ __forceinline__ double f2d_upd(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned a = b & 0x7fffffffu;
  const unsigned hi = (a == 0u) ? 0u : (a >> 3) + 0x38000000u;  // exponent rebiased
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)(b << 29));
}

// A column pair of float64 values (the float64 residual's fields).
struct D2 {
  double x, y;
};
__device__ __forceinline__ D2 operator+(D2 a, D2 b) { return D2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ D2 operator-(D2 a, D2 b) { return D2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ D2 operator*(double s, D2 a) { return D2{s * a.x, s * a.y}; }

// Three-row window of a column-pair field: w0 = row above, w1 = centre, w2 =
// row below the consumer's row.
template <typename V>
struct Win2 {
  V w0, w1, w2;
  __device__ __forceinline__ void push(V v) {
    w0 = w1;
    w1 = w2;
    w2 = v;
  }
  // the centre's left and right neighbours (one shuffle each: lane l - 1's
  // second column, lane l + 1's first column)
  __device__ __forceinline__ V left() const {
    return V{__shfl_up_sync(0xffffffffu, w1.y, 1), w1.x};
  }
  __device__ __forceinline__ V right() const {
    return V{w1.y, __shfl_down_sync(0xffffffffu, w1.x, 1)};
  }
};
__device__ __forceinline__ F2 nsum2(const Win2<F2>& w, F2 cx, F2 cy) {
  return fma2(cx, w.left() + w.right(), cy * (w.w0 + w.w2));
}
__device__ __forceinline__ D2 nsum2(const Win2<D2>& w, double cx, double cy) {
  const D2 l = w.left(), r = w.right();
  return D2{cx * (l.x + r.x) + cy * (w.w0.x + w.w2.x), cx * (l.y + r.y) + cy * (w.w0.y + w.w2.y)};
}

// Shared memory of one two-column strip warp: input rings of 64 doubles per
// row and field (x, lambda: RING rows; the fields only pass 1 reads: the
// short ring), the actuators in reach.
template <int RING, int NF = 3>
struct StripShared2 {
  __align__(16) double ring[RING * 2 * 64];
  __align__(16) double sring[STRIP_SHORT * NF * 64];
  StripAct act[MAX_NU];
  int n_act;
};

// 16-byte asynchronous copy (zeros when !valid; src must still be a valid address)
__device__ __forceinline__ void cp_async16_zfill(void* dst_smem, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(valid ? 16 : 0));
}

template <int n_lo, bool FULL, bool RBN, bool GSN = false>
__device__ __forceinline__ void strip2_body(const IterArgs& A,
                                            StripShared2<strip_ring_rows(n_lo), strip_fields(RBN)>& ws,
                                            int lane, int b, int s, int k, int rd, int x0, int y0,
                                            int strip_y, bool resid_only) {
  constexpr int E = 2 * n_lo - 1;
  constexpr int P = strip2_pad(n_lo);
  constexpr int RING = strip_ring_rows(n_lo);
  constexpr int NF = strip_fields(RBN);
  constexpr bool full = FULL;
  const InstDev& I = A.inst[b];
  const int nu = I.nu;
  const bool last = (s == I.N - 1);
  const long long so = I.s_off + (long long)s * I.ng;
  // region: columns x0 - P + 2 lane (+1), rows y0 - E .. y0 + own_rows + E - 1
  const int own_rows = min(strip_y, I.my - y0);
  const int RH = own_rows + 2 * E;
  const int gx = x0 - P + 2 * lane;               // even; the pair is gx, gx + 1
  const bool gx_ok = gx >= 0 && gx < I.mx;        // both columns (even width)
  const bool own_lane = lane >= n_lo && lane < 32 - n_lo && gx_ok;
  const int gy0 = y0 - E;

  // actuators in reach, sorted by (row, region column, index)
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
        rl[h2] = cx - (x0 - P);
        rr[h2] = cy - gy0;
        if (rl[h2] >= 0 && rl[h2] < 64 && rr[h2] >= 0 && rr[h2] < RH)
          key[h2] = ((long long)rr[h2] * 64 + rl[h2]) * MAX_NU + a;
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
  int na = 0;
  int next_row = n_act > 0 ? ws.act[0].row : 0x7fffffff;

  const double* Xg = A.xin[rd] + so;
  const double* Lg = A.lin[rd] + so;
  const double* XPg = (s == 0) ? A.x0 + I.g_off : (GSN ? A.xout[rd ^ 1] : A.xin[rd]) + so - I.ng;
  const double* LNg = (GSN ? A.lout[rd ^ 1] : A.lin[rd]) + so + I.ng;
  const double* RFg = A.ref + I.g_off;
  const float* RFf = A.ref_f + I.g_off;  // the split form reads ref as float32 pairs
  const double* XPNg = (s == 0) ? A.x0 + I.g_off : A.xout[rd ^ 1] + so - I.ng;
  const double* LNNg = A.lout[rd ^ 1] + so + I.ng;
  double* ring = ws.ring + 2 * lane;
  using SS = StripShared2<RING, NF>;
  static_assert(offsetof(SS, sring) == offsetof(SS, ring) + sizeof(double) * RING * 2 * 64,
                "short ring right after the long one");
  int sj = 0;
  auto slot_at = [&](int d, int f) -> double* {
    int q = sj + d;
    q = q < 0 ? q + RING : (q >= RING ? q - RING : q);
    return ring + (q * 2 + f) * 64;
  };
  auto sslot_row = [&](int r, int f) -> double* {
    return ring + RING * 2 * 64 + (((r + STRIP_SHORT) & (STRIP_SHORT - 1)) * NF + f) * 64;
  };
  auto ld2 = [](const double* p) { return *reinterpret_cast<const double2*>(p); };
  const int gxc = min(max(gx, 0), I.mx - 2);
  const int mx = I.mx, my = I.my;
  auto fetch = [&](int rj, int dj) {
    const int gy = gy0 + rj;
    const bool ok = gx_ok && gy >= 0 && gy < my && rj < RH;
    const int c = min(max(gy, 0), my - 1) * mx + gxc;
    double* d = slot_at(dj, 0);
    double* e = sslot_row(rj, 0);
    cp_async16_zfill(d + RB_X * 64, Xg + c, ok);
    cp_async16_zfill(d + RB_L * 64, Lg + c, ok);
    cp_async16_zfill(e + RS_XP * 64, XPg + c, ok);
    cp_async16_zfill(e + RS_LN * 64, (last ? Lg : LNg) + c, ok && !last);
    if constexpr (full)
      cp_async16_zfill(e + RS_RF * 64, RFg + c, ok);
    else  // the first 8 bytes of the pair's slot
      cp_async8_zfill(e + RS_RF * 64, RFf + c, ok);
    if constexpr (RBN) {
      cp_async16_zfill(e + RS_XPN * 64, XPNg + c, ok);
      cp_async16_zfill(e + RS_LNN * 64, (last ? Lg : LNNg) + c, ok && !last);
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
#pragma unroll
  for (int q = 0; q < STRIP_AHEAD; ++q) fetch(q, q);

  const F2 th = bc2(I.fh), tdc = bc2(I.fdc), tb0 = bc2(I.fb0);
  const F2 tcx = bc2(I.fcx), tcy = bc2(I.fcy);
  const double alpha = A.alpha;
  double* __restrict__ Xo = A.xout[rd ^ 1] + so;
  double* __restrict__ Lo = A.lout[rd ^ 1] + so;
  const double* Lin = Lg;
  const double cxd = I.cx, cyd = I.cy, dcd = I.dcoef, hd = I.h, k0d = I.k0, k1d = I.k1;
  const double qd = I.q, b0d = I.b0, hqfd = I.hqf;
  const F2 fcx = bc2(I.fcx), fcy = bc2(I.fcy), fdc = bc2(I.fdc), fh = bc2(I.fh);
  const F2 fk0 = bc2(I.fk0), fk1 = bc2(I.fk1), fk1h = bc2(I.fk1h), fq = bc2(I.fq);
  const F2 fb0 = bc2(I.fb0), fk01 = bc2(I.fk01), one = bc2(1.0f);
  const F2 hqff = bc2(last ? I.fhqf : 0.0f);
  const double* uin_s = A.uin[rd] + I.u_off + (long long)s * nu;
  const double* v3_s = A.v3g + I.u_off + (long long)s * nu;

  Norms nm{0.0f, 0.0f, make_float4(0.f, 0.f, 0.f, 0.f), 0.0, 0.0, 0.0f};
  Win2<D2> phd{}, lad{};
  Win2<F2> laf{}, xvf{};
  Win2<F2> pw[E > 1 ? E - 1 : 1];
#pragma unroll
  for (int m = 0; m < (E > 1 ? E - 1 : 1); ++m) pw[m] = Win2<F2>{};
  Shift<F2, E - 1> sdp, srg;
  Shift<F2, n_lo - 1> sk3, sax, sv1;
  Shift<F2, n_lo - 1> sv5, sw1;

  const int steps = RH + E;
  for (int j = 0; j < steps; ++j) {
    fetch(j + STRIP_AHEAD, STRIP_AHEAD);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(STRIP_AHEAD));
    // ---- pass 0: row j ----
    {
      const double2 x = ld2(slot_at(0, RB_X)), l = ld2(slot_at(0, RB_L));
      if constexpr (full) {
        phd.push(D2{k0d * (x.x + 0.5 * k1d * x.x * x.x), k0d * (x.y + 0.5 * k1d * x.y * x.y)});
        lad.push(D2{l.x, l.y});
      } else {
        const F2 xv = d2f2(x), lf = d2f2(l);
        laf.push(lf);
        xvf.push(xv);
        if (j < RH) {
          nm.mg.x = fmaxf(nm.mg.x, fmaxf(fabsf(xv.x), fabsf(xv.y)));
          nm.mg.y = fmaxf(nm.mg.y, fmaxf(fabsf(lf.x), fabsf(lf.y)));
        }
      }
    }
    // ---- pass 1: row j - 1 ----
    F2 K3 = F2{0.f, 0.f}, ax = F2{0.f, 0.f}, rg = F2{0.f, 0.f}, dp = F2{0.f, 0.f},
       v1 = F2{0.f, 0.f};
    {
      const int rj = j - 1;
      const int gy = gy0 + rj;
      const bool in_grid = gx_ok && gy >= 0 && gy < my;
      const bool own = own_lane && rj >= E && rj < RH - E && gy < my;
      // sources of the column pair: sums of u (b0 B u in K1) and of v3 (F_u v3)
      D2 srcd{0.0, 0.0};
      F2 srcf{0.f, 0.f}, inj{0.f, 0.f};
      if (rj == next_row) {  // warp-uniform
        while (na < n_act && ws.act[na].row == rj) {
          const StripAct e = ws.act[na];
          if ((e.lane >> 1) == lane) {
            const double ua = uin_s[e.a];
            const float v3a = (float)v3_s[e.a];
            if (e.lane & 1) {
              srcd.y += ua;
              srcf.y += d2f(ua);
              inj.y += v3a;
            } else {
              srcd.x += ua;
              srcf.x += d2f(ua);
              inj.x += v3a;
            }
          }
          ++na;
        }
        next_row = na < n_act ? ws.act[na].row : 0x7fffffff;
      }
      const double* rs = slot_at(-1, 0);
      const double* qs = sslot_row(j - 1, 0);
      const double2 x = ld2(rs + RB_X * 64), lam = ld2(rs + RB_L * 64);
      const double2 xp = ld2(qs + RS_XP * 64);
      F2 K1;
      if constexpr (full) {
        const double2 rc = ld2(qs + RS_RF * 64);
        const double2 lnv = last ? make_double2(hqfd * (x.x - rc.x), hqfd * (x.y - rc.y))
                                 : ld2(qs + RS_LN * 64);
        const D2 lphi = nsum2(phd, cxd, cyd) - dcd * phd.w1;
        const D2 mu = nsum2(lad, cxd, cyd) - dcd * lad.w1;
        const double dphx = k0d * (1.0 + k1d * x.x), dphy = k0d * (1.0 + k1d * x.y);
        const double t1x = hd * (lphi.x + b0d * srcd.x), t1y = hd * (lphi.y + b0d * srcd.y);
        const double t3x = hd * (qd * (x.x - rc.x) + dphx * mu.x);
        const double t3y = hd * (qd * (x.y - rc.y) + dphy * mu.y);
        const double K1x = xp.x - x.x + t1x, K1y = xp.y - x.y + t1y;
        const double K3x = lnv.x - lam.x + t3x, K3y = lnv.y - lam.y + t3y;
        if (own) {
          nm.vmax = fmax(nm.vmax, fmax(fmax(abs_or_inf(K1x), abs_or_inf(K3x)),
                                       fmax(abs_or_inf(K1y), abs_or_inf(K3y))));
          nm.vsq += K1x * K1x + K3x * K3x + K1y * K1y + K3y * K3y;
        }
        if constexpr (RBN) {
          const double2 xpn = ld2(qs + RS_XPN * 64);
          K1 = F2{d2f(xpn.x - x.x + t1x), d2f(xpn.y - x.y + t1y)};
          if (last) {
            K3 = F2{d2f(K3x), d2f(K3y)};
          } else {
            const double2 lnn = ld2(qs + RS_LNN * 64);
            K3 = F2{d2f(lnn.x - lam.x + t3x), d2f(lnn.y - lam.y + t3y)};
          }
        } else {
          K1 = F2{d2f(K1x), d2f(K1y)};
          K3 = F2{d2f(K3x), d2f(K3y)};
        }
        dp = F2{d2f(dphx), d2f(dphy)};
        const double hq = last ? hqfd : 0.0;
        ax = F2{d2f(hd * (qd + k0d * k1d * mu.x) + hq), d2f(hd * (qd + k0d * k1d * mu.y) + hq)};
      } else {
        // Lap Phi(x) in difference form (see k_strip)
        const F2 xv = xvf.w1, rv = *reinterpret_cast<const F2*>(qs + RS_RF * 64);
        const F2 xl = xvf.left(), xr = xvf.right();
        const F2 dlx = xl - xv, drx = xr - xv, dux = xvf.w0 - xv, ddx = xvf.w2 - xv;
        const F2 sx = fma2(dlx, fma2(fk1h, xl + xv, one), drx * fma2(fk1h, xr + xv, one));
        const F2 sy = fma2(dux, fma2(fk1h, xvf.w0 + xv, one), ddx * fma2(fk1h, xvf.w2 + xv, one));
        const F2 lphi = fk0 * fma2(fcx, sx, fcy * sy);
        const F2 mu = nsum2(laf, fcx, fcy) - fdc * laf.w1;
        const F2 dphi = fk0 * fma2(fk1, xv, one);
        const F2 t1 = fh * fma2(fb0, srcf, lphi);
        const F2 t3 = fh * fma2(fq, xv - rv, dphi * mu);
        const F2 xpf = d2f2(xp);
        const F2 lnf = last ? F2{0.f, 0.f} : d2f2(ld2(qs + RS_LN * 64));
        const F2 dx = xpf - xv, dl = lnf - laf.w1;
        const F2 K1f = dx + t1;
        const F2 K3f = fma2(hqff, xv - rv, dl + t3);
        const F2 K1v = sel2(own, K1f, F2{0.f, 0.f}), K3v = sel2(own, K3f, F2{0.f, 0.f});
        const float gmx = fmaxf(fmaxf(fabsf(dlx.x), fabsf(drx.x)), fmaxf(fabsf(dux.x), fabsf(ddx.x)));
        const float gmy = fmaxf(fmaxf(fabsf(dlx.y), fabsf(drx.y)), fmaxf(fabsf(dux.y), fabsf(ddx.y)));
        nm.gm = fmaxf(nm.gm, own ? fmaxf(gmx, gmy) : 0.0f);
        nm.mg.x = fmaxf(nm.mg.x, own ? fmaxf(fabsf(xpf.x), fabsf(xpf.y)) : 0.0f);
        nm.mg.y = fmaxf(nm.mg.y, own ? fmaxf(fabsf(lnf.x), fabsf(lnf.y)) : 0.0f);
        nm.mg.z = fmaxf(nm.mg.z, own ? fmaxf(fmaxf(fabsf(dx.x), fabsf(dl.x)),
                                             fmaxf(fabsf(dx.y), fabsf(dl.y)))
                                     : 0.0f);
        nm.mg.w = fmaxf(nm.mg.w, own ? fmaxf(fabsf(rv.x), fabsf(rv.y)) : 0.0f);
        nm.fmax = fmax_nan(nm.fmax, fmax_nan(fmax_nan(fabsf(K1v.x), fabsf(K3v.x)),
                                             fmax_nan(fabsf(K1v.y), fabsf(K3v.y))));
        const F2 sq2 = fma2(K1v, K1v, K3v * K3v);
        nm.fsq += sq2.x + sq2.y;
        if constexpr (RBN) {
          K1 = (d2f2(ld2(qs + RS_XPN * 64)) - xv) + t1;
          K3 = last ? K3f : (d2f2(ld2(qs + RS_LNN * 64)) - laf.w1) + t3;
        } else {
          K1 = K1f;
          K3 = K3f;
        }
        dp = dphi;
        ax = fma2(fh, fma2(fk01, mu, fq), hqff);
      }
      // 1/diag F_x, zero outside the grid (every sweep there stays zero)
      const F2 dg = F2{-1.0f, -1.0f} - th * tdc * dp;
      rg = in_grid ? F2{__frcp_rn(dg.x), __frcp_rn(dg.y)} : F2{0.f, 0.f};
      v1 = (th * tb0 * inj - K1) * rg;  // first F_x sweep of F_x v5 = F_u v3 - K1
    }
    if (!resid_only) {
      if constexpr (n_lo == 1) {
        const int rj = j - 1;
        const int gy = gy0 + rj;
        if (own_lane && rj >= E && rj < RH - E && gy < my) {
          const int c = gy * mx + gx;
          const F2 w = (F2{0.f, 0.f} - K3 - ax * v1) * rg;
          const double* rs = slot_at(-1, 0);
          const double2 xo = ld2(rs + RB_X * 64), lo = ld2(rs + RB_L * 64);
          *reinterpret_cast<double2*>(Xo + c) =
              make_double2(fma(alpha, f2d_upd(v1.x), xo.x), fma(alpha, f2d_upd(v1.y), xo.y));
          *reinterpret_cast<double2*>(Lo + c) =
              make_double2(fma(alpha, f2d_upd(w.x), lo.x), fma(alpha, f2d_upd(w.y), lo.y));
        }
      } else {
        pw[0].push(dp * v1);
        F2 v5n = F2{0.f, 0.f}, w1n = F2{0.f, 0.f};
#pragma unroll
        for (int m = 2; m <= n_lo; ++m) {
          const F2 dpm = sdp.d[m - 2], rgm = srg.d[m - 2], v1m = sv1.d[m - 2];
          const F2 off = th * nsum2(pw[m - 2], tcx, tcy);
          const F2 v = v1m - rgm * off;
          if (m < n_lo) {
            pw[m - 1].push(dpm * v);
          } else {
            const F2 w = (F2{0.f, 0.f} - sk3.d[m - 2] - sax.d[m - 2] * v) * rgm;
            v5n = v;
            w1n = w;
            pw[m - 1].push(w);
          }
        }
#pragma unroll
        for (int m = n_lo + 1; m <= E; ++m) {
          const F2 dpm = sdp.d[m - 2], rgm = srg.d[m - 2];
          const F2 w1m = sw1.d[m - n_lo - 1];
          const F2 off = th * dpm * nsum2(pw[m - 2], tcx, tcy);
          const F2 v4 = w1m - rgm * off;
          if (m < E) {
            pw[m - 1].push(v4);
          } else {
            // ---- update of the own column pair of row j - E ----
            const int rj = j - E;
            const int gy = gy0 + rj;
            if (own_lane && rj >= E && rj < RH - E && gy < my) {
              const int c = gy * mx + gx;
              const F2 v5m = sv5.d[E - n_lo - 1];
              const double* rs = slot_at(-E, 0);  // still in the ring
              const double2 xo = ld2(rs + RB_X * 64), lo = ld2(rs + RB_L * 64);
              *reinterpret_cast<double2*>(Xo + c) =
                  make_double2(fma(alpha, f2d_upd(v5m.x), xo.x), fma(alpha, f2d_upd(v5m.y), xo.y));
              *reinterpret_cast<double2*>(Lo + c) =
                  make_double2(fma(alpha, f2d_upd(v4.x), lo.x), fma(alpha, f2d_upd(v4.y), lo.y));
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
    if ((a.lane >> 1) != lane || !own_lane || a.row < E || a.row >= RH - E || gy >= I.my) continue;
    const double ua = A.uin[rd][I.u_off + (long long)s * nu + a.a];
    const double K2 = I.h * (I.r * ua + I.b0 * Lin[gy * I.mx + gx + (a.lane & 1)]);
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
          ua - alpha * (double)(float)A.v3g[I.u_off + (long long)s * nu + a.a];
  }
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

// One upper-layer iteration over the strip work list with two columns per
// lane (the strip list's x0 advance by 64 - 2 strip2_pad(n_lo)); control flow
// as k_strip.
template <int n_lo, bool RBN>
__global__ void __launch_bounds__(STRIP2_WARPS * 32, STRIP2_MIN_BLOCKS)
    k_strip2(IterArgs A, int MODE, int j_launch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  using WS = StripShared2<strip_ring_rows(n_lo), strip_fields(RBN)>;
  using WS3 = StripShared2<strip_ring_rows(n_lo), strip_fields(false)>;  // fits in WS
  unsigned char* wbase = smem_raw + warp * ((sizeof(WS) + 15) & ~size_t(15));
  WS& ws = *reinterpret_cast<WS*>(wbase);
  pdl_trigger();
  const int k = (MODE == MODE_SOLVE) ? *(volatile int*)A.iter_k + launch_iter(A, j_launch) : 0;
  const int half = launch_half(A, j_launch);
  const int rd = (MODE == MODE_SOLVE) ? (k & 1) : 0;
  pdl_wait();
  // the tail plan once few instances run (the count k_patch recorded before
  // this launch: the same value for every warp)
  const bool tail = MODE == MODE_SOLVE && A.n_tail > 0 && *A.strip_run <= A.tail_below;
  const int n_all = tail ? A.n_tail : A.n_strips, n_even = tail ? A.n_tail_even : A.n_strips_even;
  const int item = ((A.rb && half) ? n_even : 0) + blockIdx.x * STRIP2_WARPS + warp;
  const int item_end = A.rb ? (half ? n_all : n_even) : n_all;
  if (item >= item_end) return;  // warp-uniform; no block barriers in this kernel
  const int4 it = (tail ? A.tail : A.strips)[item];
  const int sy = tail ? A.tail_y : A.strip_y;
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
  if (full)
    strip2_body<n_lo, true, RBN>(A, ws, lane, b, s, k, rd, x0, y0, sy, resid_only);
  else if (RBN && MODE == MODE_SOLVE)
    strip2_body<n_lo, false, false, true>(A, *reinterpret_cast<WS3*>(wbase), lane, b, s, k, rd,
                                          x0, y0, sy, resid_only);
  else
    strip2_body<n_lo, false, RBN>(A, ws, lane, b, s, k, rd, x0, y0, sy, resid_only);
}
