/*
 * nmpc_mlp.h -- C ABI of the learned warm start for the NMPC solver.
 *
 * The paper has no learned component; its method needs only a starting
 * iterate S^0 that is feasible (Sec. 4.2: S^0 with G(u_i, x_i) > 0) and
 * converges from one close enough to the root (Theorem 1, point of
 * attraction).  This network predicts such a starting iterate from the
 * current field and reference: the control trajectory plus per-stage
 * coefficients of the state and costate in a fixed spatial POD basis.  The
 * solver's own cold/shift start stays the fallback (nmpc_solve with
 * NMPC_INIT_COLD, or the residual comparison done by the caller).
 *
 * Network: layers l = 0..L-1, z_l = a_l W_l^T + b_l, a_{l+1} = GELU(z_l) for
 * hidden layers (GELU(z) = z Phi(z), Phi the standard normal CDF, via erff),
 * linear output.  GEMM operands are BF16 with FP32 accumulation on the tensor
 * cores; FP32 master weights; MSE loss mean((y - t)^2); Adam (Kingma & Ba
 * 2015, beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 *
 * Parameter packing (host float32 arrays): for l = 0..L-1, W_l row-major
 * [out][in] followed by b_l [out].  Device arrays are float32 row-major
 * [batch][width] unless stated.  Functions return NMPC_MLP_OK or a negative
 * code; calls are asynchronous on `stream` except where stated.
 */
#ifndef NMPC_GB300_MLP_H
#define NMPC_GB300_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NMPC_MLP_OK 0
#define NMPC_MLP_ERR_BAD_ARG (-1)
#define NMPC_MLP_ERR_CUDA (-2)

typedef struct nmpc_mlp nmpc_mlp;

/* C[M,N] = sum_k A[m,k] B[n,k] (+ bias[n]) (then GELU if gelu != 0), A and B
   BF16 row-major with leading dimensions lda, ldb >= K (multiples of 8, 16-byte
   aligned rows), FP32 accumulation; C (FP32, ldc) and/or Cb (BF16, ldc) may be
   NULL but not both.  K must be a multiple of 8. */
int nmpc_gemm_bf16(const void* A, const void* B, const float* bias, float* C, void* Cb, int M,
                   int N, int K, int lda, int ldb, int ldc, int gelu, void* stream);

/* GEMM implementation (no counterpart in the paper): path 0 (default) runs
   the tcgen05 tensor-core kernel (operand tiles by TMA with the 128-byte
   swizzle, FP32 accumulator in tensor memory, split-K inside the network's
   passes) whenever both operands meet the tensor-map rules (16-byte aligned
   base, leading dimension a multiple of 8 elements), else the mma.sync
   kernel; path 1 always the mma.sync kernel (for comparisons).  GEMMs of at
   most 8 rows take a GEMV kernel either way.  Process-wide setting.
   NMPC_MLP_ERR_BAD_ARG for another value. */
int nmpc_gemm_set_path(int path);

/* 1 if a tensor-core GEMM on the current device gave up on one of its
   bounded waits since the last clear (its outputs are then invalid), else 0;
   clear != 0 resets the word.  Synchronizes the device.  Negative on a CUDA
   error. */
int nmpc_gemm_error(int clear);

/* out[i] = bf16(in[i]), round to nearest even. */
int nmpc_cast_f32_bf16(const float* in, void* out, int64_t n, void* stream);

/* out[c][r] = in[r][c] for a BF16 [rows][cols] matrix. */
int nmpc_transpose_bf16(const void* in, void* out, int rows, int cols, void* stream);

/* out[i] = (double)in[i] and out[i] = (float)in[i] (nearest). */
int nmpc_cast_f32_f64(const float* in, double* out, int64_t n, void* stream);
int nmpc_cast_f64_f32(const double* in, float* out, int64_t n, void* stream);

/* Average pooling (no counterpart in the paper: the input reduction of the
   learned warm start for large grids): src device float64 [n_img][my][mx]
   row-major, dst device float32 [n_img][my/factor][mx/factor], each output
   the mean of a factor x factor block (summed in float64).  mx and my must be
   multiples of factor, else NMPC_MLP_ERR_BAD_ARG.  Image i's pooled cells
   start at dst + i * dst_stride (dst_stride >= (mx / factor) (my / factor);
   0 means exactly that), so pooled fields can land interleaved in feature
   rows. */
int nmpc_pool_avg(const double* src, float* dst, int n_img, int mx, int my, int factor,
                  int64_t dst_stride, void* stream);

/* Network with widths[0..n_layers] (each a multiple of 8), batches up to
   max_batch; weights U(-1/sqrt(in), 1/sqrt(in)) from SplitMix64(seed), biases
   0.  Synchronous. */
int nmpc_mlp_create(int n_layers, const int* widths, int max_batch, uint64_t seed,
                    nmpc_mlp** out);
int64_t nmpc_mlp_num_params(const nmpc_mlp* m);
/* Host parameter copies in the packing above (set resets the Adam state). */
int nmpc_mlp_set_params(nmpc_mlp* m, const float* host);
int nmpc_mlp_get_params(nmpc_mlp* m, float* host);
/* y[B][out] = network(x[B][in]); 1 <= B <= max_batch. */
int nmpc_mlp_forward(nmpc_mlp* m, const float* x, int B, float* y, void* stream);
/* Forward, MSE against target[B][out], backward: gradients kept in the handle
   (nmpc_mlp_get_grads).  B a multiple of 8.  loss_host: NULL or the loss
   (then the call synchronizes). */
int nmpc_mlp_backward(nmpc_mlp* m, const float* x, const float* target, int B,
                      float* loss_host, void* stream);
int nmpc_mlp_get_grads(nmpc_mlp* m, float* host);
/* Replace the handle's gradients by a host copy in the parameter packing (no
   counterpart in the paper: for a loss computed elsewhere, and for testing
   Adam on given gradients).  Synchronous. */
int nmpc_mlp_set_grads(nmpc_mlp* m, const float* host);
/* One Adam update with the current gradients, learning rate lr. */
int nmpc_mlp_adam_step(nmpc_mlp* m, float lr, void* stream);
/* backward + adam_step. */
int nmpc_mlp_train_step(nmpc_mlp* m, const float* x, const float* target, int B, float lr,
                        float* loss_host, void* stream);
int64_t nmpc_mlp_launch_count(const nmpc_mlp* m);
void nmpc_mlp_destroy(nmpc_mlp* m);

#ifdef __cplusplus
}
#endif

#endif /* NMPC_GB300_MLP_H */
