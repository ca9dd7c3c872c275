/*
 * gdi_mpnn.h -- C ABI of the learned warm start in libgdi.so: a small message-passing network
 * that predicts an initial spin assignment for gdi_anneal, trained on partitions the annealer
 * itself produces.  The paper has no counterpart (its annealer always starts from random spins,
 * Algorithms 2 and 3); the network only chooses where annealing starts, and the plain annealer
 * judges the result.
 *
 * Conventions (all entry points):
 *   - every pointer is a device pointer on the current CUDA device; buffers are owned by the
 *     caller; work is enqueued on `stream` (cudaStream_t, NULL = legacy default) without waiting;
 *   - a batch of graphs is one disjoint-union CSR: row_ptr int64 [N + 1], col int32 [nnz]
 *     (symmetric, no self-loops), graph_ptr int64 [G + 1] vertex offsets of the graphs;
 *   - activations are float32 row-major [N x d]; weights are BF16 (uint16 bit patterns,
 *     row-major [din x 64]) with float32 master copies for the optimiser;
 *   - return 0 or a negative GDI_ERR_* code (invalid sizes, or a failed launch).
 *
 * Network: H_l = ReLU(H_{l-1} Ws_l + (A_mean H_{l-1}) Wn_l + b_l), l = 1..3, hidden 64,
 * A_mean = D^-1 A; logits z = H_3 wo + bo.  Input features: 16 channels (8 channels of Philox +-1
 * noise diffused by lazy normalised-walk steps, centred and scaled per graph and optionally
 * sign-aligned to the first channel; log(1 + deg); deg / mean degree; 6 zeros).
 */
#ifndef GDI_MPNN_H
#define GDI_MPNN_H

#include <stdint.h>

#include "gdi.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GDI_MPNN_HIDDEN 64
#define GDI_MPNN_FEATURES 16

/* feature flags */
#define GDI_MPNN_ALIGN    1   /* noise channel c >= 1 times the sign of its inner product with channel 0 */
#define GDI_MPNN_NO_NOISE 2   /* the 8 noise channels are 0 (ablation: degree features only)            */

/* Input features X [N x 16].  Vertex i of graph g draws channel c from Philox counter
 * (i - graph_ptr[g], c, graph_id[g], 0x4D504E4E) under key (seed low, seed high), word 0, bit 31;
 * the 8 noise channels are diffused by `steps` lazy walk steps, centred and scaled per graph, and
 * (GDI_MPNN_ALIGN) sign-aligned to channel 0 per graph.  scratch: float [2 * N * 8]. */
int gdi_mpnn_features(int64_t N, int32_t G, const int64_t *graph_ptr, const uint32_t *graph_id,
                      const int64_t *row_ptr, const int32_t *col, uint64_t seed, int32_t steps,
                      int32_t flags, float *X, float *scratch, void *stream);

/* Y [N x d] (d <= 64) from X [N x d]: mode 0 = A_mean X, mode 1 = A_mean^T X (transpose, used by
 * the backward pass), mode 2 = one lazy normalised-walk step 0.5 X + 0.5 D^-1/2 A D^-1/2 X.
 * accumulate != 0 adds into Y. */
int gdi_mpnn_aggregate(int64_t N, const int64_t *row_ptr, const int32_t *col, const float *X, int32_t d,
                       float *Y, int32_t mode, int32_t accumulate, void *stream);

/* H [N x 64] = ReLU(X Ws + AGG Wn + b); X, AGG [N x din], din <= 64. */
int gdi_mpnn_dense_fwd(int64_t N, const float *X, const float *AGG, int32_t din, const uint16_t *Ws,
                       const uint16_t *Wn, const float *b, float *H, void *stream);

/* Backward of one layer given dH = dL/dH [N x 64]: dPRE = dH * [H > 0] [N x 64],
 * dXs = dPRE Ws^T and T = dPRE Wn^T [N x din] (then dL/dX = dXs + A_mean^T T). */
int gdi_mpnn_dense_bwd(int64_t N, int32_t din, const uint16_t *Ws, const uint16_t *Wn, const float *H,
                       const float *dH, float *dPRE, float *dXs, float *T, void *stream);

/* out [din x dout] += A^T B (A [N x din], B [N x dout]); colsum [dout] += column sums of B if not
 * NULL.  Weight and bias gradients.  Accumulates with float atomics, so the summation order (and
 * the last bits of the result) may differ between runs. */
int gdi_mpnn_wgrad(int64_t N, const float *A, int32_t din, const float *B, int32_t dout, float *out,
                   float *colsum, void *stream);

/* z [N] = H wo + bo (wo BF16 [64], bo float [1]). */
int gdi_mpnn_out_fwd(int64_t N, const float *H, const uint16_t *wo, const float *bo, float *z, void *stream);

/* dH [N x 64] = dz wo^T. */
int gdi_mpnn_out_bwd(int64_t N, const uint16_t *wo, const float *dz, float *dH, void *stream);

/* Sign-invariant loss against labels y (int8 +-1, a balanced partition per graph):
 * per graph, loss_g = min(mean softplus(-y z), mean softplus(y z)) + lambda (mean tanh z)^2;
 * *loss += mean_g loss_g (caller zeroes it); stats [G x 4] = (L(+y), L(-y), mean tanh z, loss_g);
 * dz [N] = d(mean_g loss_g)/dz for the chosen sign of every graph. */
int gdi_mpnn_loss(int32_t G, const int64_t *graph_ptr, const float *z, const int8_t *y, float lambda,
                  float *stats, float *dz, float *loss, void *stream);

/* One Adam step on P float parameters (step = 1, 2, ...), refreshing their BF16 copies. */
int gdi_mpnn_adam(int64_t P, float *params, const float *grads, float *m, float *v, uint16_t *params_bf16,
                  float lr, float beta1, float beta2, float eps, int32_t step, void *stream);

/* BF16 copies (round to nearest even) of P float parameters. */
int gdi_mpnn_to_bf16(int64_t P, const float *params, uint16_t *params_bf16, void *stream);

/* Exactly balanced spins from logits: in every graph the floor(n/2) largest logits (ties: the
 * smaller vertex id first) get +1, the others -1 (an odd n leaves G = -1).  max_n <= 8192. */
int gdi_mpnn_round(int32_t G, const int64_t *graph_ptr, int32_t max_n, const float *z, int8_t *spins,
                   void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GDI_MPNN_H */
