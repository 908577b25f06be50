// Host side of the learned-warm-start network (include/nmpc_mlp.h): a
// fully connected network with GELU hidden layers, BF16 tensor-core GEMMs with
// FP32 accumulation, MSE loss, backward pass and Adam on FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/nmpc_mlp.h"
#include "mlp_kernels.cuh"

namespace {

#define MCK(call)                                                  \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      fprintf(stderr, "nmpc_mlp: %s failed: %s (%s:%d)\n", #call,  \
              cudaGetErrorString(e_), __FILE__, __LINE__);         \
      return NMPC_MLP_ERR_CUDA;                                    \
    }                                                              \
  } while (0)

int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (int)std::min<long long>(std::max<long long>(b, 1), 4096);
}

// ---------------------------------------------------------------------------
// GEMM dispatch: GEMV for M <= 8; the tcgen05 kernel (TMA operand tiles) when
// both operands meet the tensor-map rules (16-byte aligned base, rows a
// multiple of 16 bytes apart); the mma.sync kernel otherwise (or when forced).
// ---------------------------------------------------------------------------
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

int g_gemm_path = 0;  // 0 automatic, 1 the mma.sync kernel only

// error word of the tcgen05 kernel's bounded waits (one per device and process)
__device__ int g_tc_error;

int* tc_error_ptr() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_tc_error) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return static_cast<int*>(p);
}

// Tensor map of a row-major BF16 matrix [rows][ld] read in boxes of
// 128 rows x 64 elements with the 128-byte swizzle (zero fill past the end).
bool make_map(CUtensorMap* m, const __nv_bfloat16* ptr, int rows, int K, int ld) {
  EncodeTiled enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)mlp_dev::TC_BK, (cuuint32_t)mlp_dev::TC_BM};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tma_ok(const void* p, int ld, int K) {
  return ((uintptr_t)p % 16 == 0) && (ld % 8 == 0) && (K % 8 == 0) && K >= 8;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n < 1) n = 1;
  }
  return n;
}

// ws: FP32 workspace of ws_elems for split-K partial products (null: no split).
cudaError_t gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias, float* C,
                 __nv_bfloat16* Cb, int M, int N, int K, int lda, int ldb, int ldc, int epi,
                 cudaStream_t st, float* ws = nullptr, size_t ws_elems = 0) {
  mlp_dev::GemmArgs g{A, B, bias, C, Cb, M, N, K, lda, ldb, ldc, epi};
  if (M <= mlp_dev::GEMV_MAX_M) {
    mlp_dev::k_gemv_bf16<<<(N + 7) / 8, 256, 0, st>>>(g);
    return cudaGetLastError();
  }
  CUtensorMap ta, tb;
  if (g_gemm_path == 0 && tma_ok(A, lda, K) && tma_ok(B, ldb, K) && make_map(&ta, A, M, K, lda) &&
      make_map(&tb, B, N, K, ldb)) {
    static bool configured = false;
    if (!configured) {
      cudaError_t e = cudaFuncSetAttribute(mlp_dev::k_gemm_tc,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           mlp_dev::TC_SMEM);
      if (e != cudaSuccess) return e;
      configured = true;
    }
    const int tiles_m = (M + mlp_dev::TC_BM - 1) / mlp_dev::TC_BM;
    const int tiles_n = (N + mlp_dev::TC_BN - 1) / mlp_dev::TC_BN;
    const int tiles = tiles_m * tiles_n;
    const int n_kb = (K + mlp_dev::TC_BK - 1) / mlp_dev::TC_BK;
    // split K over more CTAs while the tiles alone leave most SMs idle (at
    // least two K blocks per slice; the partials must fit the workspace)
    int split = 1;
    if (ws && tiles * 2 < num_sms() && n_kb >= 4) {
      split = std::min((num_sms() + tiles - 1) / tiles, n_kb / 2);
      const size_t per = (size_t)M * N;
      split = (int)std::min<size_t>((size_t)split, ws_elems / std::max<size_t>(per, 1));
      split = std::max(split, 1);
    }
    const int kb_per = (n_kb + split - 1) / split;
    split = (n_kb + kb_per - 1) / kb_per;  // no empty slice
    const int vec_ok = (ldc % 8 == 0) && ((uintptr_t)C % 16 == 0) && ((uintptr_t)Cb % 16 == 0);
    mlp_dev::TcArgs t{M, N, K, kb_per, n_kb, bias, C, Cb, ldc, epi, vec_ok,
                      split > 1 ? ws : nullptr, tc_error_ptr()};
    dim3 grid(tiles_n, tiles_m, split);
    mlp_dev::k_gemm_tc<<<grid, mlp_dev::TC_THREADS, mlp_dev::TC_SMEM, st>>>(ta, tb, t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || split == 1) return e;
    const long long total = (long long)M * N;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    mlp_dev::k_splitk_epilogue<<<blocks, 256, 0, st>>>(ws, split, M, N, bias, epi, C, Cb, ldc);
    return cudaGetLastError();
  }
  dim3 grid((N + mlp_dev::BN - 1) / mlp_dev::BN, (M + mlp_dev::BM - 1) / mlp_dev::BM);
  mlp_dev::k_gemm_bf16<<<grid, mlp_dev::GEMM_THREADS, 0, st>>>(g);
  return cudaGetLastError();
}

// Launches gemm() issues for these operands (for launch accounting).
int gemm_launches(const void* A, const void* B, int M, int N, int K, int lda, int ldb,
                  bool has_ws) {
  if (M <= mlp_dev::GEMV_MAX_M || g_gemm_path != 0 || !tma_ok(A, lda, K) || !tma_ok(B, ldb, K) ||
      !encode_fn())
    return 1;
  const int tiles = ((M + 127) / 128) * ((N + 127) / 128);
  const int n_kb = (K + 63) / 64;
  return (has_ws && tiles * 2 < num_sms() && n_kb >= 4) ? 2 : 1;
}

cudaError_t transpose(const __nv_bfloat16* in, __nv_bfloat16* out, int rows, int cols,
                      cudaStream_t st) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  mlp_dev::k_transpose_bf16<<<grid, dim3(32, 8), 0, st>>>(in, out, rows, cols);
  return cudaGetLastError();
}

}  // namespace

struct nmpc_mlp {
  int L = 0;                    // layers
  std::vector<int> w;           // widths, L + 1
  int max_batch = 0;
  long long n_params = 0;
  // per layer device buffers
  std::vector<float*> W, b, gW, gb, mW, vW, mb, vb;   // fp32
  std::vector<__nv_bfloat16*> Wb, WTb;                  // bf16 [out,in] and [in,out]
  std::vector<float*> z;         // pre-activation [B, out] fp32
  std::vector<__nv_bfloat16*> a;  // activations [B, width] bf16, a[0] = input
  std::vector<__nv_bfloat16*> aT; // transposes for the weight gradient
  float* da = nullptr;            // [B, max width] fp32
  float* dz = nullptr;
  __nv_bfloat16* dz16 = nullptr;
  __nv_bfloat16* dzT = nullptr;
  float* y = nullptr;             // [B, out]
  float* loss = nullptr;
  float* h_loss = nullptr;
  float* ws = nullptr;  // split-K partial products of the tensor-core GEMM
  size_t ws_elems = 0;
  int step = 0;
  long long launches = 0;
};

extern "C" {

int nmpc_gemm_set_path(int path) {
  if (path != 0 && path != 1) return NMPC_MLP_ERR_BAD_ARG;
  g_gemm_path = path;
  return NMPC_MLP_OK;
}

int nmpc_gemm_error(int clear) {
  int* p = tc_error_ptr();
  if (!p) return NMPC_MLP_ERR_CUDA;
  int v = 0;
  MCK(cudaDeviceSynchronize());
  MCK(cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost));
  if (clear) MCK(cudaMemset(p, 0, sizeof(int)));
  return v;
}

int nmpc_gemm_bf16(const void* A, const void* B, const float* bias, float* C, void* Cb, int M,
                   int N, int K, int lda, int ldb, int ldc, int gelu, void* stream) {
  if (!A || !B || (!C && !Cb) || M < 1 || N < 1 || K < 1 || (K % 8) != 0 || lda < K || ldb < K ||
      ldc < N || (lda % 8) || (ldb % 8))
    return NMPC_MLP_ERR_BAD_ARG;
  if (((uintptr_t)A | (uintptr_t)B) & 15) return NMPC_MLP_ERR_BAD_ARG;
  MCK(gemm((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, bias, C, (__nv_bfloat16*)Cb, M, N, K,
           lda, ldb, ldc, gelu ? mlp_dev::EPI_GELU : mlp_dev::EPI_NONE, (cudaStream_t)stream));
  return NMPC_MLP_OK;
}

int nmpc_cast_f32_bf16(const float* in, void* out, int64_t n, void* stream) {
  if (!in || !out || n < 0) return NMPC_MLP_ERR_BAD_ARG;
  if (n == 0) return NMPC_MLP_OK;
  mlp_dev::k_cast_bf16<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
      in, (__nv_bfloat16*)out, n);
  MCK(cudaGetLastError());
  return NMPC_MLP_OK;
}

int nmpc_transpose_bf16(const void* in, void* out, int rows, int cols, void* stream) {
  if (!in || !out || rows < 1 || cols < 1) return NMPC_MLP_ERR_BAD_ARG;
  MCK(transpose((const __nv_bfloat16*)in, (__nv_bfloat16*)out, rows, cols, (cudaStream_t)stream));
  return NMPC_MLP_OK;
}

int nmpc_cast_f32_f64(const float* in, double* out, int64_t n, void* stream) {
  if (!in || !out || n < 0) return NMPC_MLP_ERR_BAD_ARG;
  if (n == 0) return NMPC_MLP_OK;
  mlp_dev::k_cast_f64<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(in, out, n);
  MCK(cudaGetLastError());
  return NMPC_MLP_OK;
}

int nmpc_cast_f64_f32(const double* in, float* out, int64_t n, void* stream) {
  if (!in || !out || n < 0) return NMPC_MLP_ERR_BAD_ARG;
  if (n == 0) return NMPC_MLP_OK;
  mlp_dev::k_cast_f64_f32<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(in, out, n);
  MCK(cudaGetLastError());
  return NMPC_MLP_OK;
}

int nmpc_pool_avg(const double* src, float* dst, int n_img, int mx, int my, int factor,
                  int64_t dst_stride, void* stream) {
  if (!src || !dst || n_img < 0 || mx < 1 || my < 1 || factor < 1 || (mx % factor) != 0 ||
      (my % factor) != 0)
    return NMPC_MLP_ERR_BAD_ARG;
  const long long per = (long long)(mx / factor) * (my / factor);
  if (dst_stride == 0) dst_stride = per;
  if (dst_stride < per) return NMPC_MLP_ERR_BAD_ARG;
  const long long n = (long long)n_img * per;
  if (n == 0) return NMPC_MLP_OK;
  mlp_dev::k_pool_avg<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(src, dst, n_img, mx, my,
                                                                          factor, dst_stride);
  MCK(cudaGetLastError());
  return NMPC_MLP_OK;
}

int nmpc_mlp_create(int n_layers, const int* widths, int max_batch, uint64_t seed,
                    nmpc_mlp** out) {
  if (!out || !widths || n_layers < 1 || n_layers > 16 || max_batch < 1) return NMPC_MLP_ERR_BAD_ARG;
  for (int l = 0; l <= n_layers; ++l)
    if (widths[l] < 1 || (widths[l] % 8) != 0) return NMPC_MLP_ERR_BAD_ARG;
  *out = nullptr;
  nmpc_mlp* m = new (std::nothrow) nmpc_mlp();
  if (!m) return NMPC_MLP_ERR_CUDA;
  m->L = n_layers;
  m->w.assign(widths, widths + n_layers + 1);
  m->max_batch = max_batch;
  const int B = max_batch;
  int wmax = 0;
  for (int v : m->w) wmax = std::max(wmax, v);
  bool ok = true;
  auto A = [&](cudaError_t e) { ok = ok && (e == cudaSuccess); };
  auto fal = [&](float** p, size_t n) { *p = nullptr; A(cudaMalloc((void**)p, std::max<size_t>(n, 1) * 4)); };
  auto bal = [&](__nv_bfloat16** p, size_t n) { *p = nullptr; A(cudaMalloc((void**)p, std::max<size_t>(n, 1) * 2)); };
  m->W.resize(n_layers); m->b.resize(n_layers); m->gW.resize(n_layers); m->gb.resize(n_layers);
  m->mW.resize(n_layers); m->vW.resize(n_layers); m->mb.resize(n_layers); m->vb.resize(n_layers);
  m->Wb.resize(n_layers); m->WTb.resize(n_layers); m->z.resize(n_layers);
  m->a.resize(n_layers + 1); m->aT.resize(n_layers + 1);
  for (int l = 0; l < n_layers; ++l) {
    const size_t nin = m->w[l], nout = m->w[l + 1];
    fal(&m->W[l], nin * nout); fal(&m->gW[l], nin * nout); fal(&m->mW[l], nin * nout);
    fal(&m->vW[l], nin * nout); fal(&m->b[l], nout); fal(&m->gb[l], nout);
    fal(&m->mb[l], nout); fal(&m->vb[l], nout);
    bal(&m->Wb[l], nin * nout); bal(&m->WTb[l], nin * nout);
    fal(&m->z[l], (size_t)B * nout);
    m->n_params += (long long)nin * nout + nout;
  }
  for (int l = 0; l <= n_layers; ++l) {
    bal(&m->a[l], (size_t)B * m->w[l]);
    bal(&m->aT[l], (size_t)B * m->w[l]);
  }
  fal(&m->da, (size_t)B * wmax);
  fal(&m->dz, (size_t)B * wmax);
  bal(&m->dz16, (size_t)B * wmax);
  bal(&m->dzT, (size_t)B * wmax);
  fal(&m->y, (size_t)B * m->w[n_layers]);
  fal(&m->loss, 1);
  // split-K partial products: up to 8 Mi floats (32 MiB)
  m->ws_elems = std::min<size_t>(size_t(8) << 20, (size_t)B * wmax * 16);
  fal(&m->ws, m->ws_elems);
  A(cudaMallocHost((void**)&m->h_loss, sizeof(float)));
  if (!ok) {
    nmpc_mlp_destroy(m);
    return NMPC_MLP_ERR_CUDA;
  }
  // initial weights: U(-1/sqrt(in), 1/sqrt(in)) from SplitMix64(seed), biases 0
  std::vector<float> host((size_t)m->n_params);
  uint64_t state = seed;
  size_t o = 0;
  for (int l = 0; l < n_layers; ++l) {
    const int nin = m->w[l], nout = m->w[l + 1];
    const float bound = 1.0f / std::sqrt((float)nin);
    for (long long e = 0; e < (long long)nin * nout; ++e) {
      state += 0x9E3779B97F4A7C15ull;
      uint64_t z = state;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
      host[o++] = (float)((2.0 * u - 1.0) * bound);
    }
    for (int e = 0; e < nout; ++e) host[o++] = 0.0f;
  }
  int rc = nmpc_mlp_set_params(m, host.data());
  if (rc != NMPC_MLP_OK) {
    nmpc_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return NMPC_MLP_OK;
}

int64_t nmpc_mlp_num_params(const nmpc_mlp* m) { return m ? m->n_params : 0; }

int nmpc_mlp_set_params(nmpc_mlp* m, const float* host) {
  if (!m || !host) return NMPC_MLP_ERR_BAD_ARG;
  size_t o = 0;
  for (int l = 0; l < m->L; ++l) {
    const size_t nin = m->w[l], nout = m->w[l + 1];
    MCK(cudaMemcpy(m->W[l], host + o, nin * nout * 4, cudaMemcpyHostToDevice));
    o += nin * nout;
    MCK(cudaMemcpy(m->b[l], host + o, nout * 4, cudaMemcpyHostToDevice));
    o += nout;
    MCK(cudaMemset(m->mW[l], 0, nin * nout * 4));
    MCK(cudaMemset(m->vW[l], 0, nin * nout * 4));
    MCK(cudaMemset(m->mb[l], 0, nout * 4));
    MCK(cudaMemset(m->vb[l], 0, nout * 4));
    mlp_dev::k_cast_bf16<<<grid_for(nin * nout, 256), 256>>>(m->W[l], m->Wb[l], nin * nout);
    MCK(cudaGetLastError());
    MCK(transpose(m->Wb[l], m->WTb[l], (int)nout, (int)nin, 0));
  }
  m->step = 0;
  MCK(cudaDeviceSynchronize());
  return NMPC_MLP_OK;
}

static int copy_out(nmpc_mlp* m, float* host, bool grads) {
  size_t o = 0;
  MCK(cudaDeviceSynchronize());
  for (int l = 0; l < m->L; ++l) {
    const size_t nin = m->w[l], nout = m->w[l + 1];
    MCK(cudaMemcpy(host + o, grads ? m->gW[l] : m->W[l], nin * nout * 4, cudaMemcpyDeviceToHost));
    o += nin * nout;
    MCK(cudaMemcpy(host + o, grads ? m->gb[l] : m->b[l], nout * 4, cudaMemcpyDeviceToHost));
    o += nout;
  }
  return NMPC_MLP_OK;
}

int nmpc_mlp_get_params(nmpc_mlp* m, float* host) {
  if (!m || !host) return NMPC_MLP_ERR_BAD_ARG;
  return copy_out(m, host, false);
}

int nmpc_mlp_get_grads(nmpc_mlp* m, float* host) {
  if (!m || !host) return NMPC_MLP_ERR_BAD_ARG;
  return copy_out(m, host, true);
}

int nmpc_mlp_set_grads(nmpc_mlp* m, const float* host) {
  if (!m || !host) return NMPC_MLP_ERR_BAD_ARG;
  MCK(cudaDeviceSynchronize());
  size_t o = 0;
  for (int l = 0; l < m->L; ++l) {
    const size_t nin = m->w[l], nout = m->w[l + 1];
    MCK(cudaMemcpy(m->gW[l], host + o, nin * nout * 4, cudaMemcpyHostToDevice));
    o += nin * nout;
    MCK(cudaMemcpy(m->gb[l], host + o, nout * 4, cudaMemcpyHostToDevice));
    o += nout;
  }
  return NMPC_MLP_OK;
}

static int forward_impl(nmpc_mlp* m, const float* x, int B, float* y, cudaStream_t st) {
  const int n_in = m->w[0];
  mlp_dev::k_cast_bf16<<<grid_for((long long)B * n_in, 256), 256, 0, st>>>(x, m->a[0],
                                                                        (long long)B * n_in);
  MCK(cudaGetLastError());
  m->launches++;
  for (int l = 0; l < m->L; ++l) {
    const int nin = m->w[l], nout = m->w[l + 1];
    const bool last = (l == m->L - 1);
    // z = a W^T + b (fp32 kept for the backward pass) and, for a hidden
    // layer, GELU(z) as bf16: both from one product
    MCK(gemm(m->a[l], m->Wb[l], m->b[l], m->z[l], last ? nullptr : m->a[l + 1], B, nout, nin, nin,
             nin, nout, last ? mlp_dev::EPI_NONE : mlp_dev::EPI_Z_GELU, st, m->ws, m->ws_elems));
    m->launches += gemm_launches(m->a[l], m->Wb[l], B, nout, nin, nin, nin, m->ws != nullptr);
  }
  const int nout = m->w[m->L];
  if (y != m->z[m->L - 1]) {
    const long long ny = (long long)B * nout;
    mlp_dev::k_copy_f32<<<grid_for(ny, 256), 256, 0, st>>>(m->z[m->L - 1], y, ny);
    MCK(cudaGetLastError());
    m->launches++;
  }
  return NMPC_MLP_OK;
}

int nmpc_mlp_forward(nmpc_mlp* m, const float* x, int B, float* y, void* stream) {
  if (!m || !x || !y || B < 1 || B > m->max_batch) return NMPC_MLP_ERR_BAD_ARG;
  return forward_impl(m, x, B, y, (cudaStream_t)stream);
}

int nmpc_mlp_backward(nmpc_mlp* m, const float* x, const float* target, int B, float* loss_host,
                      void* stream) {
  if (!m || !x || !target || B < 1 || B > m->max_batch || (B % 8) != 0) return NMPC_MLP_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = forward_impl(m, x, B, m->y, st);
  if (rc != NMPC_MLP_OK) return rc;
  const int nout_all = m->w[m->L];
  MCK(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
  const long long ny = (long long)B * nout_all;
  mlp_dev::k_mse<<<grid_for(ny, 256), 256, 0, st>>>(m->y, target, ny, m->dz, m->dz16, m->loss);
  MCK(cudaGetLastError());
  m->launches++;
  for (int l = m->L - 1; l >= 0; --l) {
    const int nin = m->w[l], nout = m->w[l + 1];
    // dz (fp32 in m->dz, bf16 in m->dz16) holds dL/dz_l, [B, nout]
    mlp_dev::k_bias_grad<<<(nout + 127) / 128, 128, 0, st>>>(m->dz, m->gb[l], B, nout);
    MCK(cudaGetLastError());
    // gW[o, i] = sum_b dz[b, o] a_l[b, i]: A = dz^T [nout, B], B-operand = a_l^T [nin, B]
    MCK(transpose(m->dz16, m->dzT, B, nout, st));
    MCK(transpose(m->a[l], m->aT[l], B, nin, st));
    MCK(gemm(m->dzT, m->aT[l], nullptr, m->gW[l], nullptr, nout, nin, B, B, B, nin,
             mlp_dev::EPI_NONE, st, m->ws, m->ws_elems));
    m->launches += 3 + gemm_launches(m->dzT, m->aT[l], nout, nin, B, B, B, m->ws != nullptr);
    if (l > 0) {
      // da[b, i] = sum_o dz[b, o] W[o, i]: A = dz [B, nout], B-operand = W^T [nin, nout]
      MCK(gemm(m->dz16, m->WTb[l], nullptr, m->da, nullptr, B, nin, nout, nout, nout, nin,
               mlp_dev::EPI_NONE, st, m->ws, m->ws_elems));
      const long long n = (long long)B * nin;
      mlp_dev::k_gelu_backward<<<grid_for(n, 256), 256, 0, st>>>(m->da, m->z[l - 1], m->dz,
                                                                m->dz16, n);
      MCK(cudaGetLastError());
      m->launches += 1 + gemm_launches(m->dz16, m->WTb[l], B, nin, nout, nout, nout,
                                       m->ws != nullptr);
    }
  }
  if (loss_host) {
    MCK(cudaMemcpyAsync(m->h_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    *loss_host = *m->h_loss;
  }
  return NMPC_MLP_OK;
}

int nmpc_mlp_adam_step(nmpc_mlp* m, float lr, void* stream) {
  if (!m || !(lr > 0)) return NMPC_MLP_ERR_BAD_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  m->step++;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - std::pow(b1, (float)m->step), c2 = 1.0f - std::pow(b2, (float)m->step);
  for (int l = 0; l < m->L; ++l) {
    const long long nw = (long long)m->w[l] * m->w[l + 1];
    mlp_dev::k_adam<<<grid_for(nw, 256), 256, 0, st>>>(m->W[l], m->gW[l], m->mW[l], m->vW[l],
                                                       m->Wb[l], nw, lr, b1, b2, eps, c1, c2);
    mlp_dev::k_adam<<<grid_for(m->w[l + 1], 256), 256, 0, st>>>(
        m->b[l], m->gb[l], m->mb[l], m->vb[l], nullptr, m->w[l + 1], lr, b1, b2, eps, c1, c2);
    MCK(cudaGetLastError());
    MCK(transpose(m->Wb[l], m->WTb[l], m->w[l + 1], m->w[l], st));
    m->launches += 3;
  }
  return NMPC_MLP_OK;
}

int nmpc_mlp_train_step(nmpc_mlp* m, const float* x, const float* target, int B, float lr,
                        float* loss_host, void* stream) {
  int rc = nmpc_mlp_backward(m, x, target, B, loss_host, stream);
  if (rc != NMPC_MLP_OK) return rc;
  return nmpc_mlp_adam_step(m, lr, stream);
}

int64_t nmpc_mlp_launch_count(const nmpc_mlp* m) { return m ? m->launches : 0; }

void nmpc_mlp_destroy(nmpc_mlp* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  auto F = [](void* p) { if (p) cudaFree(p); };
  for (int l = 0; l < (int)m->W.size(); ++l) {
    F(m->W[l]); F(m->b[l]); F(m->gW[l]); F(m->gb[l]); F(m->mW[l]); F(m->vW[l]);
    F(m->mb[l]); F(m->vb[l]); F(m->Wb[l]); F(m->WTb[l]); F(m->z[l]);
  }
  for (size_t l = 0; l < m->a.size(); ++l) { F(m->a[l]); F(m->aT[l]); }
  F(m->da); F(m->dz); F(m->dz16); F(m->dzT); F(m->y); F(m->loss); F(m->ws);
  if (m->h_loss) cudaFreeHost(m->h_loss);
  delete m;
}

}  // extern "C"
