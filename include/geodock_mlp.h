/* geodock_mlp.h -- C ABI of the learned orientation proposer in libgeodock.so.
 *
 * The paper has no learned component: GeoDock evaluates every restart (Listing 1).
 * This proposer sits beside the search: a BF16 multilayer perceptron 48 -> 256 -> 256
 * -> 1 (ReLU, FP32 accumulation) predicts each restart's final score from features of
 * the ligand and its restart pose, and only the best-predicted restarts get the full
 * fragment optimisation of Sec. 3.1.  Its matrix products run on the tensor cores
 * (tcgen05.mma, accumulators in tensor memory).
 *
 * All pointers here are device pointers unless stated otherwise.
 */
#ifndef GEODOCK_MLP_H
#define GEODOCK_MLP_H

#include "geodock.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Matrix product on the tensor cores: D = A * B^T with A (M x K, or K x M when transA)
 * and B (N x K, or K x N when transB) BF16 row-major with leading dimensions lda / ldb
 * (elements; multiples of 8 when not transposed), K and N multiples of 16.  Epilogue per
 * element: x = D + bias[n] (bias may be NULL), x = max(x, 0) if relu; C (FP32) and Cb
 * (BF16) receive x if non-NULL (leading dimension ldc); if dotw is non-NULL (N <= 256),
 * dot_out[m] = sum_n bf16(x[m][n]) * dotw[n] + dot_bias.  dev_err (device int, may be
 * NULL) is set to 1 if a bounded device wait ran out.  Asynchronous on `stream`. */
gd_status gd_mlp_gemm(const void* A, int lda, int transA, const void* B, int ldb, int transB, float* C,
                      void* Cb, int ldc, int M, int N, int K, const float* bias, int relu,
                      const float* dotw, float dot_bias, float* dot_out, int* dev_err, void* stream);

/* Features of every (ligand, restart) of a prepared job: 48 numbers per row, row
 * li * O + o (input ligand order), written as BF16 (x_bf16, the network's input) and/or
 * FP32 (x_f32); either may be NULL.  Row layout:
 *   0..3   unit quaternion (w, x, y, z) of the restart rotation Rz(a) Ry(b) Rz(g), w >= 0
 *   4, 5   atoms / 250, rotamers / 60
 *   6      radius of gyration of the input coordinates / 10 A
 *   7..22  fraction of atoms at distance [0.75 b, 0.75 (b+1)) A from the centroid
 *   23..47 pocket value / 255 under 25 atoms of the placed restart pose, chosen by
 *          farthest-point sampling from the atom farthest from the centroid (ties to
 *          the smaller preorder id), cyclic for ligands of fewer than 25 atoms.
 * Runs on `stream` after the job's upload (use the stream the job was prepared on). */
gd_status gd_job_features(gd_ctx* ctx, gd_job* job, void* x_bf16, float* x_f32, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GEODOCK_MLP_H */
