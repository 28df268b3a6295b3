// Internal interface of the tensor-core MLP kernels (gd_mlp.cu).  Not part of the ABI.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gd {

// D = A * B^T (BF16 inputs, FP32 accumulation in TMEM), then per element
// x = D + bias[n]; x = relu(x) if relu; C (FP32) and/or Cb (BF16) receive x;
// with dotw, dot_out[m] = sum_n bf16(x[m][n]) * dotw[n] + dot_bias (requires N <= 256).
// A is M x K (transA: stored K x M), B is N x K (transB: stored K x N); K and N are
// multiples of 16.
struct GemmArgs {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  int lda, ldb, ldc;
  int M, N, K;
  bool transA, transB;
  const float* bias;
  bool relu;
  float* C;
  __nv_bfloat16* Cb;
  const float* dotw;
  float dot_bias;
  const float* dot_bias_dev;  // added to dot_bias when non-null (device scalar)
  float* dot_out;
  int* err;  // set to 1 if a bounded wait ran out (may be null)
  int hold;  // test: the first MMA commit is withheld, so that the wait on it runs out
  // split K (partial set): CTA z < ksplit of the grid's third dimension sums K range
  // [z kslice, min(K, (z + 1) kslice)) into partial[z][M][N] (raw FP32, no epilogue);
  // reduce_splits then adds the ranges in order into C
  int ksplit, kslice;
  float* partial;
};
// C[m][n] (row stride ldc) = sum over z < S of partial[z][m][n], in order of z.
cudaError_t reduce_splits(const float* partial, int S, int M, int N, float* C, int ldc, cudaStream_t stream);

size_t gemm_smem_bytes();
// Fused two-layer forward of the proposer network (persistent, one CTA per SM).
cudaError_t infer_launch(const __nv_bfloat16* X, int M, const __nv_bfloat16* W1b, const __nv_bfloat16* W2b,
                         const float* b1, const float* b2, const float* w3r, const float* b3, float* y, int* err,
                         int hold, int num_sms, cudaStream_t stream);
cudaError_t gemm_launch(const GemmArgs& g, cudaStream_t stream);

}  // namespace gd
