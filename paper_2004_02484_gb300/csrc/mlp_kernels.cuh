// Kernels of the learned warm start: a multilayer perceptron with BF16
// operands and FP32 accumulation on the tensor cores, its backward pass, Adam,
// and the POD decode of predicted coefficients into state/costate guesses.
//
// GEMM convention (all layers, forward and backward):
//   C[M, N] = sum_k A[m, k] * B[n, k]   (+ bias[n], optional GELU)
// with A and B row-major and K contiguous, BF16; accumulation in FP32 by
// mma.sync.m16n8k16.row.col.f32.bf16.bf16.f32.  The CTA tile is 128 x 128 x 32
// (8 warps as 2 x 4, warp tile 64 x 32), operands staged in shared memory by
// cp.async with a double buffer and read into fragments by ldmatrix.  Rows and
// columns outside the matrix are zero-filled, so M, N are arbitrary and K only
// needs to be a multiple of 8 (16-byte chunks).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace mlp_dev {

constexpr int BM = 128, BN = 128, BK = 32, PAD = 8, LDS = BK + PAD;  // bf16 elements
constexpr int GEMM_THREADS = 256;
enum { EPI_NONE = 0, EPI_GELU = 1, EPI_Z_GELU = 2 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;  // src-size 0 writes zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t& r0, uint32_t& r1,
                                            uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad(float z) {
  const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
  return cdf + z * pdf;
}

// Output (m, n) of an accumulated product x: + bias; EPI_NONE / EPI_GELU store
// the (activated) value to C and/or Cb; EPI_Z_GELU stores the pre-activation
// to C and BF16 GELU of it to Cb (a hidden layer's z and activation from one
// product).
__device__ __forceinline__ void epilogue_store(float x, int m, int n, const float* bias, int epi,
                                               float* C, __nv_bfloat16* Cb, int ldc) {
  if (bias) x += bias[n];
  const long long o = (long long)m * ldc + n;
  if (epi == EPI_Z_GELU) {
    if (C) C[o] = x;
    if (Cb) Cb[o] = __float2bfloat16_rn(gelu(x));
    return;
  }
  if (epi == EPI_GELU) x = gelu(x);
  if (C) C[o] = x;
  if (Cb) Cb[o] = __float2bfloat16_rn(x);
}

struct GemmArgs {
  const __nv_bfloat16* A;  // [M, lda]
  const __nv_bfloat16* B;  // [N, ldb]
  const float* bias;       // [N] or null
  float* C;                // [M, ldc] fp32 or null
  __nv_bfloat16* Cb;       // [M, ldc] bf16 or null (after the epilogue)
  int M, N, K, lda, ldb, ldc;
  int epi;
};

__global__ void __launch_bounds__(GEMM_THREADS) k_gemm_bf16(GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 sA[2][BM * LDS];
  __shared__ __align__(16) __nv_bfloat16 sB[2][BN * LDS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

  // each tile is 128 rows x 4 chunks of 16 bytes; 256 threads x 2 chunks
  auto load_tile = [&](int stage, int k0) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int chunk = tid + t * GEMM_THREADS;
      const int row = chunk >> 2, kc = (chunk & 3) * 8;
      const int gk = k0 + kc;
      {
        const int gm = m0 + row;
        const bool ok = (gm < g.M) && (gk < g.K);
        const __nv_bfloat16* src = g.A + (ok ? ((long long)gm * g.lda + gk) : 0);
        cp_async16(smem_u32(&sA[stage][row * LDS + kc]), src, ok);
      }
      {
        const int gn = n0 + row;
        const bool ok = (gn < g.N) && (gk < g.K);
        const __nv_bfloat16* src = g.B + (ok ? ((long long)gn * g.ldb + gk) : 0);
        cp_async16(smem_u32(&sB[stage][row * LDS + kc]), src, ok);
      }
    }
  };

  const int ktiles = (g.K + BK - 1) / BK;
  load_tile(0, 0);
  cp_async_commit();
  for (int kt = 0; kt < ktiles; ++kt) {
    const int st = kt & 1;
    if (kt + 1 < ktiles) load_tile(st ^ 1, (kt + 1) * BK);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[4][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int j = lane >> 3, r = lane & 7;
        const int row = wm + i * 16 + (j & 1) * 8 + r;
        const int col = kk + (j >> 1) * 8;
        ldmatrix_x4(smem_u32(&sA[st][row * LDS + col]), af[i][0], af[i][1], af[i][2], af[i][3]);
      }
#pragma unroll
      for (int jp = 0; jp < 2; ++jp) {
        const int j = lane >> 3, r = lane & 7;
        const int row = wn + jp * 16 + (j >> 1) * 8 + r;
        const int col = kk + (j & 1) * 8;
        uint32_t r0, r1, r2, r3;
        ldmatrix_x4(smem_u32(&sB[st][row * LDS + col]), r0, r1, r2, r3);
        bf[2 * jp][0] = r0;
        bf[2 * jp][1] = r1;
        bf[2 * jp + 1][0] = r2;
        bf[2 * jp + 1][1] = r3;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
  cp_async_wait<0>();

  // epilogue: bias, GELU, fp32 and/or bf16 stores
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + i * 16 + (lane >> 2) + ((q >> 1) ? 8 : 0);
        const int n = n0 + wn + j * 8 + (lane & 3) * 2 + (q & 1);
        if (m < g.M && n < g.N) {
          epilogue_store(acc[i][j][q], m, n, g.bias, g.epi, g.C, g.Cb, g.ldc);
        }
      }
}

// The same product for few rows (M <= 8, e.g. single-instance inference):
// one warp per output column n, 16-byte loads of B's row and of the M rows of
// A (shared by all warps through L1), FP32 accumulation, warp-shuffle sums.
constexpr int GEMV_MAX_M = 8;

__global__ void __launch_bounds__(256) k_gemv_bf16(GemmArgs g) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = blockIdx.x * 8 + warp;
  if (n >= g.N) return;
  float acc[GEMV_MAX_M];
#pragma unroll
  for (int m = 0; m < GEMV_MAX_M; ++m) acc[m] = 0.0f;
  const __nv_bfloat16* brow = g.B + (long long)n * g.ldb;
  for (int k = lane * 8; k < g.K; k += 256) {
    const uint4 bv = *reinterpret_cast<const uint4*>(brow + k);
    const __nv_bfloat162* b2 = reinterpret_cast<const __nv_bfloat162*>(&bv);
    float bf[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 f = __bfloat1622float2(b2[q]);
      bf[2 * q] = f.x;
      bf[2 * q + 1] = f.y;
    }
#pragma unroll
    for (int m = 0; m < GEMV_MAX_M; ++m) {
      if (m < g.M) {
        const uint4 av = *reinterpret_cast<const uint4*>(g.A + (long long)m * g.lda + k);
        const __nv_bfloat162* a2 = reinterpret_cast<const __nv_bfloat162*>(&av);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 f = __bfloat1622float2(a2[q]);
          acc[m] = fmaf(f.x, bf[2 * q], acc[m]);
          acc[m] = fmaf(f.y, bf[2 * q + 1], acc[m]);
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < GEMV_MAX_M; ++m) {
    float v = acc[m];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && m < g.M) epilogue_store(v, m, n, g.bias, g.epi, g.C, g.Cb, g.ldc);
  }
}

// out[c, r] = in[r, c] (bf16), 32 x 32 tiles through shared memory
__global__ void k_transpose_bf16(const __nv_bfloat16* in, __nv_bfloat16* out, int rows, int cols) {
  __shared__ __nv_bfloat16 t[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int r = blockIdx.y * 32 + dy;
    if (r < rows && c < cols) t[dy][threadIdx.x] = in[(long long)r * cols + c];
  }
  __syncthreads();
  const int r2 = blockIdx.y * 32 + threadIdx.x;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int c2 = blockIdx.x * 32 + dy;
    if (c2 < cols && r2 < rows) out[(long long)c2 * rows + r2] = t[threadIdx.x][dy];
  }
}

// out = in (a kernel rather than a copy node, so that the forward pass can be
// captured into any graph, conditional bodies included)
__global__ void k_copy_f32(const float* in, float* out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = in[e];
}

__global__ void k_cast_bf16(const float* in, __nv_bfloat16* out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = __float2bfloat16_rn(in[e]);
}

__global__ void k_cast_f64(const float* in, double* out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (double)in[e];
}

__global__ void k_cast_f64_f32(const double* in, float* out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

// Average pooling of n_img row-major my x mx float64 fields by f x f blocks
// into float32 [n_img][(my/f) (mx/f)] (sums in float64).
__global__ void k_pool_avg(const double* src, float* dst, int n_img, int mx, int my, int f,
                           long long dst_stride) {
  const int ox = mx / f, oy = my / f;
  const long long n = (long long)n_img * ox * oy;
  const double inv = 1.0 / ((double)f * f);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long img = e / ((long long)ox * oy);
    const int o = (int)(e - img * ox * oy);
    const int oyi = o / ox, oxi = o - oyi * ox;
    const double* s = src + img * (long long)mx * my + (long long)oyi * f * mx + (long long)oxi * f;
    double acc = 0.0;
    for (int a = 0; a < f; ++a)
      for (int c = 0; c < f; ++c) acc += s[(long long)a * mx + c];
    dst[img * dst_stride + o] = (float)(acc * inv);
  }
}

// loss = mean((y - t)^2) over B*N; dy = 2 (y - t) / (B*N) written as bf16 (and fp32)
__global__ void k_mse(const float* y, const float* t, long long n, float* dy32,
                      __nv_bfloat16* dy16, float* loss_acc) {
  float acc = 0.0f;
  const float scale = 2.0f / (float)n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float d = y[e] - t[e];
    acc += d * d;
    const float gval = scale * d;
    if (dy32) dy32[e] = gval;
    dy16[e] = __float2bfloat16_rn(gval);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, acc / (float)n);
}

// dz = da * GELU'(z) (hidden layers); written as bf16 for the next GEMMs and fp32
__global__ void k_gelu_backward(const float* da, const float* z, float* dz32,
                                __nv_bfloat16* dz16, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float v = da[e] * gelu_grad(z[e]);
    dz32[e] = v;
    dz16[e] = __float2bfloat16_rn(v);
  }
}

// db[n] = sum_b dz[b, n]
__global__ void k_bias_grad(const float* dz, float* db, int B, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int b = 0; b < B; ++b) s += dz[(long long)b * N + n];
  db[n] = s;
}

// Adam (Kingma & Ba 2015) on fp32 master weights, then the bf16 copy
__global__ void k_adam(float* w, const float* g, float* m, float* v, __nv_bfloat16* wb,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float gv = g[e];
    const float mv = b1 * m[e] + (1.0f - b1) * gv;
    const float vv = b2 * v[e] + (1.0f - b2) * gv * gv;
    m[e] = mv;
    v[e] = vv;
    const float upd = lr * (mv / c1) / (sqrtf(vv / c2) + eps);
    const float nw = w[e] - upd;
    w[e] = nw;
    if (wb) wb[e] = __float2bfloat16_rn(nw);
  }
}

#include "mlp_tc.cuh"

}  // namespace mlp_dev
