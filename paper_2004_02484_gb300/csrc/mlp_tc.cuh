// Blackwell (sm_103a) tensor-core GEMM of the learned warm start:
//   C[M, N] = sum_k A[m, k] B[n, k]   (+ bias[n], optional GELU)
// A and B BF16, row-major with K contiguous (K-major operands), FP32
// accumulation in tensor memory (TMEM).  Included from mlp_kernels.cuh inside
// namespace mlp_dev.
//
// One CTA of 128 threads computes a 128 x 128 tile of C over a range of K
// blocks (all of K, or one slice of a split-K launch):
//   warp 0, one lane: TMA loads (cp.async.bulk.tensor.2d, 128-byte swizzle)
//     of the A and B tiles of each 64-wide K block into a ring of STAGES
//     shared-memory stages; a "full" mbarrier per stage counts the bytes;
//   warp 1, one lane: per K block, four tcgen05.mma (kind::f16, BF16 x BF16,
//     FP32 accumulator of 128 lanes x 128 columns in TMEM, M = 128, N = 128,
//     K = 16 each), then tcgen05.commit onto the stage's "empty" mbarrier so
//     the producer may refill it; after the last block a commit onto "done";
//   warp 0 allocates the 128 TMEM columns before the loop and frees them at
//   the end;
//   epilogue, all four warps: warp w reads TMEM lanes 32 w .. 32 w + 31 (the
//     tile's rows) with tcgen05.ld (32 columns per load), adds the bias,
//     applies GELU and stores FP32 and/or BF16 rows; in a split-K launch it
//     stores the raw FP32 partial tile to a workspace slice instead, and
//     k_splitk_epilogue sums the slices in a fixed order.
// Operand tiles are read by TMA from this GPU's own memory only (no
// multicast).  Rows or K columns past the matrix are zero-filled by the TMA
// unit.  Every mbarrier wait is bounded: a wait that runs out raises the
// error word, the CTA stops issuing work, waits (bounded) for what it issued,
// frees its TMEM and returns.
#pragma once

// three stages (96 KB) so that two CTAs fit per SM: one CTA's epilogue then
// overlaps the other's main loop (TMEM: 2 x 128 of 512 columns)
constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 3;
constexpr int TC_THREADS = 128;
constexpr int TC_TILE_A = TC_BM * TC_BK * 2;  // bytes of one A stage (16 KB)
constexpr int TC_TILE_B = TC_BN * TC_BK * 2;  // bytes of one B stage (16 KB)
constexpr int TC_SMEM = TC_STAGES * (TC_TILE_A + TC_TILE_B) + 1024 /* alignment */ + 256;
constexpr long long TC_WAIT_TRIES = 1LL << 24;  // bounded mbarrier waits

struct TcArgs {
  int M, N, K;          // problem
  int kb_per_split;     // K blocks of 64 per CTA (grid.z slices)
  int n_kb;             // K blocks in all
  const float* bias;    // [N] or null (no split)
  float* C;             // [M, ldc] or null
  __nv_bfloat16* Cb;    // [M, ldc] or null
  int ldc, epi;
  int vec_ok;           // C / Cb rows 16-byte aligned (ldc % 8 == 0, aligned bases)
  float* ws;            // split-K partials [split][M][N] (split > 1) or null
  int* err;             // raised when a bounded wait ran out
};

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Wait until the phase of parity `parity` of the mbarrier at `bar` has
// completed, for at most TC_WAIT_TRIES polls; false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long t = 0; t < TC_WAIT_TRIES; ++t) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle (rows of 128 bytes, 8-row groups 1024 bytes apart): start
// address, stride between 8-row groups 1024 B, the fixed version bits, and
// the 128-byte swizzle mode.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);           // start address
  d |= (uint64_t)(16u >> 4) << 16;                     // leading byte offset (unused here)
  d |= (uint64_t)(1024u >> 4) << 32;                   // stride byte offset
  d |= (uint64_t)1 << 46;                              // descriptor version
  d |= (uint64_t)2 << 61;                              // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = TC_BN, M = TC_BM.
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(tc_idesc()), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
      : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(TC_THREADS, 2)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              TcArgs g) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // 1024-byte aligned stage ring (the 128-byte swizzle repeats every 1024 B)
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t sA = base;                              // STAGES x 16 KB
  const uint32_t sB = base + TC_STAGES * TC_TILE_A;      // STAGES x 16 KB
  const uint32_t bars = sB + TC_STAGES * TC_TILE_B;      // full[S], empty[S], done
  const uint32_t full0 = bars, empty0 = bars + 8 * TC_STAGES, done = bars + 16 * TC_STAGES;
  const uint32_t tslot = done + 8;                       // TMEM base address (written by alloc)
  unsigned char* gen_base = tc_smem_raw + (base - raw);
  volatile uint32_t* tslot_ptr =
      reinterpret_cast<volatile uint32_t*>(gen_base + (tslot - base));
  __shared__ int s_fail;
  __shared__ int s_issued;  // K blocks whose TMA loads the producer issued

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * TC_BN, m0 = blockIdx.y * TC_BM;
  const int kb0 = blockIdx.z * g.kb_per_split;
  const int kb1 = min(g.n_kb, kb0 + g.kb_per_split);
  const int nk = max(0, kb1 - kb0);

  if (threadIdx.x == 0) {
    s_fail = 0;
    s_issued = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tslot),
                 "r"(TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot_ptr;

  if (warp == 0 && lane == 0) {
    // producer: wait for a free stage, then both tiles of the next K block
    for (int i = 0; i < nk; ++i) {
      const int s = i % TC_STAGES;
      const uint32_t ph = (uint32_t)((i / TC_STAGES) & 1);
      if (!mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
        atomicExch(&s_fail, 1);
        break;
      }
      if (*(volatile int*)&s_fail) break;
      mbar_expect_tx(full0 + 8 * s, (uint32_t)(TC_TILE_A + TC_TILE_B));
      const int kc = (kb0 + i) * TC_BK;
      tma_load_2d(sA + s * TC_TILE_A, &tmA, full0 + 8 * s, kc, m0);
      tma_load_2d(sB + s * TC_TILE_B, &tmB, full0 + 8 * s, kc, n0);
      s_issued = i + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: four K = 16 steps per stage, the stage freed by a commit
    for (int i = 0; i < nk; ++i) {
      const int s = i % TC_STAGES;
      const uint32_t ph = (uint32_t)((i / TC_STAGES) & 1);
      if (!mbar_wait(full0 + 8 * s, ph)) {
        atomicExch(&s_fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a = sA + s * TC_TILE_A, b = sB + s * TC_TILE_B;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk)
        tc_mma(tmem, smem_desc_sw128(a + 32 * kk), smem_desc_sw128(b + 32 * kk),
               (i > 0 || kk > 0) ? 1u : 0u);
      tc_commit(empty0 + 8 * s);
    }
    // the accumulator is complete once every issued MMA is (a commit with no
    // MMA outstanding arrives at once)
    tc_commit(done);
  }
  __syncwarp();
  // epilogue: every warp waits for the accumulator
  const bool ok = mbar_wait(done, 0u);
  if (!ok && lane == 0) atomicExch(&s_fail, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  __syncthreads();
  const bool failed = s_fail != 0;
  if (!failed && nk > 0) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < TC_BN; c0 += 32) {
      float v[32];
      tmem_ld32(lane_base + (uint32_t)c0, v);
      const int n = n0 + c0;
      if (row < g.M && n < g.N) {
        const bool whole = (n + 32 <= g.N);
        if (g.ws) {
          float* dst = g.ws + ((long long)blockIdx.z * g.M + row) * g.N + n;
          if (whole && ((g.N & 3) == 0)) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (n + j < g.N) dst[j] = v[j];
          }
        } else if (whole && g.vec_ok) {
          // 32 whole columns with 16-byte aligned rows: vector stores
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float x = v[j];
            if (g.bias) x += g.bias[n + j];
            v[j] = x;
          }
          const long long o = (long long)row * g.ldc + n;
          if (g.C) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              float4 q;
              q.x = (g.epi == EPI_GELU) ? gelu(v[j]) : v[j];
              q.y = (g.epi == EPI_GELU) ? gelu(v[j + 1]) : v[j + 1];
              q.z = (g.epi == EPI_GELU) ? gelu(v[j + 2]) : v[j + 2];
              q.w = (g.epi == EPI_GELU) ? gelu(v[j + 3]) : v[j + 3];
              *reinterpret_cast<float4*>(g.C + o + j) = q;
            }
          }
          if (g.Cb) {
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
              uint4 q;
              uint32_t* w = reinterpret_cast<uint32_t*>(&q);
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                float a = v[j + 2 * t], b = v[j + 2 * t + 1];
                if (g.epi != EPI_NONE) {
                  a = gelu(a);
                  b = gelu(b);
                }
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
                w[t] = *reinterpret_cast<const uint32_t*>(&h2);
              }
              *reinterpret_cast<uint4*>(g.Cb + o + j) = q;
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (n + j < g.N) epilogue_store(v[j], row, n + j, g.bias, g.epi, g.C, g.Cb, g.ldc);
        }
      }
    }
  } else if (failed && threadIdx.x == 0 && g.err) {
    atomicExch(g.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (failed && warp == 0 && lane == 0) {
    // bounded wait for the TMA copies this CTA issued (the last load into
    // each stage completes its full barrier's phase) before shared memory is
    // released
    const int issued = s_issued;
    for (int s = 0; s < TC_STAGES && s < issued; ++s) {
      const int last = ((issued - 1 - s) / TC_STAGES) * TC_STAGES + s;
      mbar_wait(full0 + 8 * s, (uint32_t)((last / TC_STAGES) & 1));
    }
  }
  __syncwarp();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_BN));
}

// Split-K: C = sum over the slices of the workspace (fixed order) + bias,
// optional GELU; FP32 and/or BF16 outputs.
__global__ void k_splitk_epilogue(const float* ws, int split, int M, int N, const float* bias,
                                  int epi, float* C, __nv_bfloat16* Cb, int ldc) {
  const long long total = (long long)M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    float x = 0.0f;
    for (int s = 0; s < split; ++s) x += ws[(long long)s * total + i];
    const int m = (int)(i / N), n = (int)(i - (long long)m * N);
    epilogue_store(x, m, n, bias, epi, C, Cb, ldc);
  }
}
