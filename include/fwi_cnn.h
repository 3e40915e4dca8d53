/* fwi_cnn.h - layers of the learned start-model network (GB300, sm_103a).
 *
 * The paper's Limitations section names the starting model as FWI's weak
 * point (cycle skipping). This part of libfwi trains a small encoder-decoder
 * CNN, on shot gathers that the library's own forward modelling generates, to
 * predict a starting velocity model; plain smooth-start FWI stays the fallback
 * and the yardstick of its error. The network is not from the paper.
 *
 * Conventions of every call:
 *   - activations are FP32, channel-major [C][B][H][W] (channel, batch, rows,
 *     columns), so that a convolution over the whole batch is one GEMM;
 *   - convolutions are 3x3 cross-correlations with zero padding 1 and stride
 *     (sh, sw): Ho = (H - 1) / sh + 1, Wo = (W - 1) / sw + 1;
 *     y[o][b][i][j] = bias[o] + sum_{c,p,q} w[o][c][p][q] x[c][b][sh i + p - 1][sw j + q - 1];
 *   - weights [O][C][3][3] are kept in FP32 by the caller and passed to the
 *     GEMMs as a BF16 copy (fwi_cnn_to_bf16); the GEMMs multiply BF16 operands
 *     with FP32 accumulation on the tcgen05 tensor cores (this library's own
 *     kernel: TMA-staged operands, accumulator in tensor memory); im2col,
 *     col2im and every element-wise step are this library's kernels too;
 *   - every pointer is a device pointer on the handle's device, every call is
 *     asynchronous on cuda_stream and returns FWI_EINVAL for a NULL required
 *     pointer or a non-positive size, FWI_ECUDA for a CUDA failure
 *     (fwi_last_error() has the message);
 *   - the handle owns the layer calls' workspace (im2col matrices, BF16
 *     copies, GEMM partials); it grows to the largest layer seen (cudaMalloc,
 *     which synchronises the device), so calls on one handle must be issued
 *     in order on one stream;
 *   - the GEMMs' waits are bounded: a wait that gives up writes NaN into its
 *     output tile and sets the handle's status, which fwi_cnn_check reports;
 *   - nothing is accumulated across calls: outputs are overwritten.
 */
#ifndef FWI_CNN_H
#define FWI_CNN_H

#include <stdint.h>

#include "fwi.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fwi_cnn fwi_cnn; /* workspace and status word on one device */

fwi_status fwi_cnn_create(fwi_cnn **h, int device);
fwi_status fwi_cnn_destroy(fwi_cnn *h);

/* Waits for cuda_stream and returns FWI_ETIMEOUT (clearing it) if a GEMM of
 * this handle gave up a bounded wait since the last check, else FWI_OK. */
fwi_status fwi_cnn_check(fwi_cnn *h, void *cuda_stream);

/* How the convolution GEMMs of the forward pass and of the stride-1 data
 * gradient get their tap operand: on != 0 (the default) gathers it from the
 * activations into the GEMM's shared-memory stages (no im2col matrix in device
 * memory); 0 builds the im2col matrix first and has TMA stage it. Both give the
 * same BF16 operand and the same results bit for bit. FWI_EINVAL if h is NULL. */
fwi_status fwi_cnn_set_conv_gather(fwi_cnn *h, int32_t on);

/* The tensor-core GEMM itself: out[n][m] = act(sum_k A[m][k] B[n][k] + bias[n]).
 * A: M rows of K BF16 values, row stride lda; B: N rows of K BF16 values, row
 * stride ldb (lda, ldb multiples of 8 and >= K; A, B 16-byte aligned).
 * out: FP32, element (n, m) at out[n * ldo + m] (ldo >= M): the product is
 * written transposed. bias [N] or NULL; relu != 0 applies max(., 0).
 * splits > 1 cuts K into that many runs whose FP32 partials are summed in a
 * fixed order (bias and relu then must be off). */
fwi_status fwi_cnn_gemm_bt(fwi_cnn *h, const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb, int64_t M,
                           int32_t N, int64_t K, float *out, int64_t ldo, const float *bias, int32_t relu,
                           int32_t splits, void *cuda_stream);

/* y = act(conv(x, w) + bias), act = ReLU if relu != 0 else identity.
 * x [C][B][H][W]; w_bf16 [O][C][3][3]; bias [O]; y [O][B][Ho][Wo].
 * One GEMM over the batch: pixels x taps (im2col) times taps x channels, the
 * bias and ReLU applied as the accumulator is written. */
fwi_status fwi_cnn_conv_forward(fwi_cnn *h, const float *x, int32_t C, int32_t B, int32_t H, int32_t W,
                                const uint16_t *w_bf16, const float *bias, int32_t O, int32_t sh,
                                int32_t sw, int32_t relu, float *y, void *cuda_stream);

/* Gradients of a loss L through one convolution layer.
 * y: the layer's output from fwi_cnn_conv_forward (used for the ReLU mask when relu != 0).
 * dy: dL/dy [O][B][Ho][Wo]; overwritten with dL/d(pre-activation).
 * dx: dL/dx [C][B][H][W], or NULL (first layer); dw [O][C][3][3]; db [O].
 * The GEMM operands are the BF16-rounded pre-activation gradient, x and w. A
 * stride-1 layer's dx is one GEMM (the gradient convolved with the flipped
 * weights); a strided layer's goes through a tap matrix and a col2im gather. */
fwi_status fwi_cnn_conv_backward(fwi_cnn *h, const float *x, int32_t C, int32_t B, int32_t H, int32_t W,
                                 const uint16_t *w_bf16, int32_t O, int32_t sh, int32_t sw, int32_t relu,
                                 const float *y, float *dy, float *dx, float *dw, float *db, void *cuda_stream);

/* Nearest-neighbour 2x upsampling of the last two axes: x [C][B][H][W] -> y [C][B][2H][2W],
 * and its gradient dx [C][B][H][W] from dy [C][B][2H][2W] (sums of 2x2 blocks, in the order
 * (dy[2r][2s] + dy[2r][2s+1]) + (dy[2r+1][2s] + dy[2r+1][2s+1])). The 2H x 2W tensor (y, or dy) must be
 * 8-byte aligned (FWI_EINVAL otherwise). */
fwi_status fwi_cnn_upsample2(const float *x, int32_t C, int32_t B, int32_t H, int32_t W, float *y,
                             void *cuda_stream);
fwi_status fwi_cnn_upsample2_backward(const float *dy, int32_t C, int32_t B, int32_t H, int32_t W, float *dx,
                                      void *cuda_stream);

/* loss = 1/(2n) sum (p - t)^2 (FP64, one device double) and dp = (p - t) / n.
 * The FP64 sum runs over a fixed number of block partials held by the handle. */
fwi_status fwi_cnn_mse(fwi_cnn *h, const float *p, const float *t, int64_t n, double *loss, float *dp,
                       void *cuda_stream);

/* One bias-corrected Adam step (Kingma & Ba) on n parameters at step >= 1;
 * theta_bf16, if not NULL, receives the BF16 copy of the updated theta. */
fwi_status fwi_cnn_adam(float *theta, const float *g, float *m, float *v, int64_t n, int32_t step, float lr,
                        float beta1, float beta2, float eps, uint16_t *theta_bf16, void *cuda_stream);

/* Round-to-nearest-even BF16 copy of n FP32 values. */
fwi_status fwi_cnn_to_bf16(const float *x, uint16_t *y, int64_t n, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
