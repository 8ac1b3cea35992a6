// Internal interface of the warm-start MLP kernels (qp_mlp.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qp {
namespace mlp {

enum EpiMode {
  kEpiBiasRelu = 0,   // out_bf16 = bf16(relu(acc + bias))
  kEpiBiasF32 = 1,    // out_f32 = acc + bias
  kEpiPartialF32 = 4, // out_f32 + z * M * ldo = acc for split z (sum_splits adds them in order)
  kEpiReluMask = 3,   // out_bf16 = bf16(relu_ref > 0 ? acc : 0)
};

// D[M x N] (+)= A[M x K] B[N x K]^T; A, B bf16 row-major with K contiguous.
// N in [16, 256] and a multiple of 16; K, lda, ldb multiples of 16 / 8.
struct GemmArgs {
  const __nv_bfloat16 *A;
  int lda;
  const __nv_bfloat16 *B;
  int ldb;
  int M, N, K;
  int k_per_split;  // set by gemm()
  int mode;
  const float *bias;
  float *out_f32;
  __nv_bfloat16 *out_bf16;
  int ldo;
  const __nv_bfloat16 *relu_ref;
  int ldr;
  int *err;  // set to 1 if a bounded wait gave up
};

cudaError_t gemm(const GemmArgs &g, int splits, cudaStream_t st);
// The number of K-splits gemm() launches for K and the requested splits.
int gemm_splits(int K, int splits);
// out[i] = sum over z = 0 .. splits-1, in that order, of ws[z * n + i]: the
// split-K partials of a kEpiPartialF32 gemm, added the same way on every run.
cudaError_t sum_splits(const float *ws, int splits, int n, float *out, cudaStream_t st);

// The network's whole forward pass in one launch, one CTA per 128-row tile:
// x0 bf16 [Mp x 16] (Mp a multiple of 128), weights w[l] bf16 [256 x K_l]
// row-major (K_0 = 16, else 256), bias[l] fp32 [256], hidden activations
// h[l] bf16 [Mp x 256] (null: not written), logits z fp32 [Mp x 256].
struct FwdArgs {
  const __nv_bfloat16 *x0;
  const float *bias[4];
  __nv_bfloat16 *h[3];
  float *z;
  int Mp;
  int *err;  // set to 1 if a bounded wait gave up
};
cudaError_t forward(const FwdArgs &g, const __nv_bfloat16 *const w[4], cudaStream_t st);
// loss_rows[m] = -log p[label] of row m (0 for a padding row); loss_sum[0]
// = their sum, added in a fixed order.
cudaError_t softmax_ce(const float *Z, int ldz, const int32_t *label, const int32_t *steps, int M, float inv_rows,
                       __nv_bfloat16 *dZ, int ldd, float *loss_rows, float *loss_sum, cudaStream_t st);
// out[n] = sum_m Y[m][n], in a fixed order: per slab of rows into partial
// (kColsumSlabs x N floats), then the slabs in order.
constexpr int kColsumSlabs = 64;
cudaError_t colsum(const __nv_bfloat16 *Y, int ld, int M, int N, float *partial, float *out, cudaStream_t st);
cudaError_t transpose(const __nv_bfloat16 *in, int R, int C, int ldi, __nv_bfloat16 *out, int ldo, cudaStream_t st);
cudaError_t adam(float *w, float *m, float *v, const float *g, int rows, int cols, float lr, float b1, float b2,
                 float eps, int step, __nv_bfloat16 *wb, __nv_bfloat16 *wt, cudaStream_t st);
cudaError_t to_bf16(const float *in, __nv_bfloat16 *out, int n, cudaStream_t st);

}  // namespace mlp
}  // namespace qp
