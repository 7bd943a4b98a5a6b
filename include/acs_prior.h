/*
 * acs_prior.h -- learned edge prior for the candidate lists of libacs.
 *
 * The paper has no learned component: its candidate set is the cl nearest
 * neighbours and eta = 1/d (Sec. 3, Alg. 2). This extension scores every
 * candidate edge (i, nn[i][k]) with a small MLP over 8 edge features and
 * uses the score p in (0,1) to reweight the heuristic, w' = w * p, and to
 * prune each list to its `keep` best-scored candidates. The full-scan
 * fallback of Alg. 2 keeps the plain heuristic. The MLP is trained on the
 * GPU on the edge frequencies of best-so-far tours found by plain ACS.
 *
 * Network: x[8] -> h1 = relu(x W1 + b1)[64] -> h2 = relu(h1 W2 + b2)[64]
 *          -> z = h2 w3 + b3 -> p = sigmoid(z).
 * The two hidden layers run on the tensor cores with BF16 operands
 * (features, W1, h1, W2) and FP32 accumulation; biases, h2, w3 and the last
 * layer stay FP32. Scoring (acs_mlp_forward) and training
 * (acs_mlp_train_batch) issue tcgen05.mma with the accumulators in tensor
 * memory; training rounds dh2 and dh1 to BF16 as the operands of the
 * backward GEMMs and sums the bias and w3 gradients in FP32.
 *
 * Parameters are one FP32 device vector of ACS_MLP_PARAMS floats:
 *   W1 [8][64] at 0, b1 [64] at 512, W2 [64][64] at 576 (W2[in][out]),
 *   b2 [64] at 4672, w3 [64] at 4736, b3 at 4800.
 * Features: BF16 (stored as uint16_t) [rows][8], rows = n*32 per instance,
 * row i*32+k is the edge (i, nn[i][k]); rows with k >= cl are zero.
 *
 * All pointers named dev_* are device pointers; the caller owns them. Calls
 * are stream-ordered on `stream` (a cudaStream_t; NULL = legacy default) and
 * return ACS_EINVAL for bad arguments, ACS_ESTATE for a context that an
 * earlier failure left unusable (or, for acs_prior_count_best_edges, one that
 * has not run an iteration yet), ACS_ECUDA for launch failures. Calls taking
 * a context first wait for the work queued on the context's own stream.
 */
#ifndef ACS_PRIOR_H
#define ACS_PRIOR_H
#include <stdint.h>

#include "acs.h"

#ifdef __cplusplus
extern "C" {
#endif

#define ACS_MLP_FEATURES 8
#define ACS_MLP_HIDDEN 64
#define ACS_MLP_PARAMS 4801

/* The 8 features of every candidate edge of instance `instance`, from the
 * context's plain candidate lists (call before acs_apply_prior):
 * (1) rank/cl, (2) d_ij / mean candidate distance of i, (3) d_ij / d_i,last,
 * (4) (x_j-x_i)/d_i,last, (5) (y_j-y_i)/d_i,last, (6) rank of i in j's list
 * / cl or 1 when absent, (7) d_ij / d_j,last, (8) in-degree of j / cl;
 * d_i,last = distance to i's last candidate (at least 1), the mean also at
 * least 1. Computed in FP32, rounded once to BF16. dev_feat: [n*32][8]. */
acs_status acs_prior_features(acs_ctx* ctx, int32_t instance, uint16_t* dev_feat, void* stream);

/* Adds to dev_count [n*32] (FP32) the number of times each candidate edge of
 * `instance` appears, in either direction, in the context's best-so-far tour.
 * Summing over R independent runs and dividing by R gives the training label
 * (the edge's frequency in best tours). */
acs_status acs_prior_count_best_edges(acs_ctx* ctx, int32_t instance, float* dev_count,
                                      void* stream);

/* Scores p = sigmoid(z) of `rows` feature rows (dev_feat [rows][8] BF16,
 * 16-byte aligned, else ACS_EINVAL) into dev_p [rows] FP32. The kernel's
 * only wait (for the tensor core's completion signal) is bounded; if it ever
 * gives up, the rows that were not scored hold NaN, the device status word
 * records it (acs_mlp_sync then returns ACS_ETIMEOUT) and tensor memory is
 * freed only after the MMA already issued has completed. */
acs_status acs_mlp_forward(const float* dev_params, const uint16_t* dev_feat, int64_t rows,
                           float* dev_p, void* stream);

/* One training pass over a mini-batch: rows b = 0..batch-1 read feature row
 * and label perm(first + b) with perm(i) = (perm_a * i + perm_c) mod total
 * (perm_a coprime with total). Writes the mean BCE loss to dev_loss[0] and
 * the gradient of that mean to dev_grad [ACS_MLP_PARAMS] (both overwritten).
 * dev_feat 16-byte aligned. If a bounded wait for the tensor core gives up,
 * the loss is NaN, the gradient incomplete and acs_mlp_sync reports
 * ACS_ETIMEOUT. */
acs_status acs_mlp_train_batch(const float* dev_params, const uint16_t* dev_feat,
                               const float* dev_label, int64_t total, int64_t first,
                               int64_t batch, int64_t perm_a, int64_t perm_c, float* dev_grad,
                               float* dev_loss, void* stream);

/* Waits for the work queued on `stream`, then reports whether a bounded
 * tensor-core wait of an acs_mlp_forward / acs_mlp_train_batch launch on the
 * current device has given up: ACS_ETIMEOUT the first time (that launch's
 * scores or gradient are incomplete), ACS_OK if none has. After a give-up the
 * tensor-core path of the process is closed: acs_mlp_forward,
 * acs_mlp_train_batch, acs_mlp_adam, acs_apply_prior and this call return
 * ACS_ESTATE. acs_apply_prior runs the same check before using its scores
 * (ACS_ETIMEOUT, and the context is poisoned). ACS_ECUDA if the stream
 * reports an error. */
acs_status acs_mlp_sync(void* stream);

/* Test hook of the bounded waits (no counterpart in the paper; for tests of
 * the failure path, never needed otherwise): wait_ns sets the bound of one
 * tensor-core wait (0 restores the default of 200 ms); phantom = 1 makes the
 * first wait of every tile poll a second mbarrier that nothing arrives on,
 * so the bound is reached while the tensor core still completes normally.
 * Process-wide; ACS_EINVAL for a negative bound or a phantom other than 0/1. */
acs_status acs_mlp_test_wait_hook(int64_t wait_ns, int32_t phantom);

/* One Adam step (Kingma & Ba) on all parameters, step >= 1, in place:
 * m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, p -= lr mhat / (sqrt(vhat)+eps). */
acs_status acs_mlp_adam(float* dev_params, const float* dev_grad, float* dev_m, float* dev_v,
                        int32_t step, float lr, float beta1, float beta2, float eps,
                        void* stream);

/* Replaces the candidate rows of `instance` with the `keep` best-scored of
 * its cl candidates (dev_p [n*32], scores of the current rows; ties -> lower
 * rank), kept in their original rank order, with weights w' = w * p (FP32).
 * The full-scan fallback keeps the plain heuristic. 1 <= keep <= cl. */
acs_status acs_apply_prior(acs_ctx* ctx, int32_t instance, const float* dev_p, int32_t keep,
                           void* stream);

/* Replaces the candidate rows of `instance` with caller tables (host nn
 * [n][cl], w [n][cl], 1 <= cl <= 32, entries in [0,n) and != own node). */
acs_status acs_set_candidates(acs_ctx* ctx, int32_t instance, const int32_t* nn, const float* w,
                              int32_t cl);

#ifdef __cplusplus
}
#endif
#endif
