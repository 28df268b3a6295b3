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

/* ---- the network ------------------------------------------------------------------
 * Parameters, FP32 masters in this order: W1[256][48] | b1[256] | W2[256][256] | b2[256]
 * | w3[256] | b3 (gd_mlp_param_count() floats).  The forward pass multiplies BF16
 * roundings of the weights and stores activations as BF16:
 *   H1 = bf16(relu(X W1^T + b1)), H2 = bf16(relu(H1 W2^T + b2)), y = H2 . bf16(w3) + b3.
 * Training minimises the mean squared error with Adam (beta 0.9 / 0.999, eps 1e-8);
 * gradients follow the same rounding points (products of BF16 operands, FP32 sums). */
typedef struct gd_mlp gd_mlp;
int gd_mlp_param_count(void);
/* Allocate a model on `device` (He-uniform initialisation from `seed`) able to train on
 * batches of up to max_batch rows (a multiple of 16). */
gd_status gd_mlp_create(int device, uint64_t seed, int max_batch, gd_mlp** out);
gd_status gd_mlp_destroy(gd_mlp* model);
/* Parameters to / from host FP32 arrays (set also resets the Adam state). */
gd_status gd_mlp_set_params(gd_mlp* model, const float* host);
gd_status gd_mlp_get_params(gd_mlp* model, float* host);
/* y[M] = network(X[M x 48] BF16), device pointers, asynchronous on `stream`. */
gd_status gd_mlp_predict(gd_mlp* model, const void* x_bf16, long long M, float* y, void* stream);
/* Gradients (device FP32 array in the parameter layout) and loss (device float) of the
 * MSE over B rows (a multiple of 16, <= max_batch): rows idx[0..B) of X / t, or the
 * first B rows when idx is NULL.  No update. */
gd_status gd_mlp_gradients(gd_mlp* model, const void* x_bf16, const float* t, const int32_t* idx, int B,
                           float* grad, float* loss, void* stream);
/* One Adam step on that loss with learning rate lr; loss (device float, may be NULL). */
gd_status gd_mlp_train_step(gd_mlp* model, const void* x_bf16, const float* t, const int32_t* idx, int B,
                            float lr, float* loss, void* stream);
/* 1 if a bounded device wait of the model's kernels ran out since creation. */
gd_status gd_mlp_error(gd_mlp* model, int* host_err);
/* Test of the bounded waits (no fault, no hang): on = 1 makes the model's next
 * tensor-core launch (the predict's fused kernel, or the first GEMM of gradients /
 * train_step) withhold its first MMA commit, so that the wait on it runs out after about
 * two seconds; the kernel then drains its MMAs with one more commit before it frees its
 * tensor memory, sets the error flag and returns (its outputs are undefined).  on = 0
 * clears a hold not yet taken and the error flag (synchronises the device). */
gd_status gd_mlp_test_hold(gd_mlp* model, int on);

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

/* Pruned search of a prepared job: pred[L x O] (device, e.g. gd_mlp_predict on the
 * job's features) ranks the restarts of every ligand; the k best (ties to the smaller
 * restart id) get the full search of Sec. 3.1, except that a ligand falls back to every
 * restart when the spread s = pred(1st) - pred(k-th) is below `margin` (rule 0) or
 * above it (rule 1).  The best pose is then taken over the searched restarts only;
 * evals[] counts them.  Needs O <= 256.  Queue gd_job_download + gd_fetch_results. */
gd_status gd_job_launch_proposed(gd_ctx* ctx, gd_job* job, const float* pred, int k, float margin, int rule,
                                 void* stream);
/* The same with a bounded fallback: a ligand that falls back searches its k_fallback
 * best-predicted restarts (ties to the smaller restart id), k <= k_fallback <= O;
 * k_fallback = O is gd_job_launch_proposed.  GD_EINVAL outside that range. */
gd_status gd_job_launch_proposed_fb(gd_ctx* ctx, gd_job* job, const float* pred, int k, int k_fallback, float margin,
                                    int rule, void* stream);
/* Restarts searched per ligand (k, or the fallback count) and the prediction spreads of the last proposed
 * launch (host arrays of L; either may be NULL; waits for the job). */
gd_status gd_job_selection(gd_ctx* ctx, gd_job* job, int32_t* counts, float* spreads);

#ifdef __cplusplus
}
#endif
#endif /* GEODOCK_MLP_H */
