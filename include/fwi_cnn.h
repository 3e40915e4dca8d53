/* fwi_cnn.h - layers of the learned start-model network (GB300, sm_103a).
 *
 * The paper's Limitations section names the starting model as FWI's weak
 * point (cycle skipping). This part of libfwi trains a small encoder-decoder
 * CNN, on shot gathers that the library's own forward modelling generates, to
 * predict a starting velocity model; plain smooth-start FWI stays the fallback
 * and the judge of its error. The network is not from the paper.
 *
 * Conventions of every call:
 *   - activations are FP32, channel-major [C][B][H][W] (channel, batch, rows,
 *     columns), so that a convolution over the whole batch is one GEMM;
 *   - convolutions are 3x3 cross-correlations with zero padding 1 and stride
 *     (sh, sw): Ho = (H - 1) / sh + 1, Wo = (W - 1) / sw + 1;
 *     y[o][b][i][j] = bias[o] + sum_{c,p,q} w[o][c][p][q] x[c][b][sh i + p - 1][sw j + q - 1];
 *   - weights [O][C][3][3] are kept in FP32 by the caller and passed to the
 *     GEMMs as a BF16 copy (fwi_cnn_to_bf16); the GEMMs multiply BF16 operands
 *     with FP32 accumulation on the tensor cores (cuBLAS), im2col, col2im and
 *     every element-wise step are this library's kernels;
 *   - every pointer is a device pointer on the handle's device, every call is
 *     asynchronous on cuda_stream and returns FWI_EINVAL for a NULL required
 *     pointer or a non-positive size, FWI_ECUDA for a CUDA or cuBLAS failure
 *     (fwi_last_error() has the message);
 *   - nothing is accumulated across calls: outputs are overwritten.
 */
#ifndef FWI_CNN_H
#define FWI_CNN_H

#include <stdint.h>

#include "fwi.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fwi_cnn fwi_cnn; /* owns a cuBLAS handle on one device */

fwi_status fwi_cnn_create(fwi_cnn **h, int device);
fwi_status fwi_cnn_destroy(fwi_cnn *h);

/* y = act(conv(x, w) + bias), act = ReLU if relu != 0 else identity.
 * x [C][B][H][W]; w_bf16 [O][C][3][3]; bias [O]; y [O][B][Ho][Wo].
 * col: workspace of C*9 * B*Ho*Wo BF16 values (the im2col matrix). */
fwi_status fwi_cnn_conv_forward(fwi_cnn *h, const float *x, int32_t C, int32_t B, int32_t H, int32_t W,
                                const uint16_t *w_bf16, const float *bias, int32_t O, int32_t sh,
                                int32_t sw, int32_t relu, uint16_t *col, float *y, void *cuda_stream);

/* Gradients of a loss L through one convolution layer.
 * y: the layer's output from fwi_cnn_conv_forward (used for the ReLU mask when relu != 0).
 * dy: dL/dy [O][B][Ho][Wo]; overwritten with dL/d(pre-activation).
 * dx: dL/dx [C][B][H][W], or NULL (first layer); dw [O][C][3][3]; db [O].
 * Workspaces: col (C*9 * B*Ho*Wo BF16), dy_bf16 (O * B*Ho*Wo BF16),
 * dcol (C*9 * B*Ho*Wo FP32; unused if dx is NULL). */
fwi_status fwi_cnn_conv_backward(fwi_cnn *h, const float *x, int32_t C, int32_t B, int32_t H, int32_t W,
                                 const uint16_t *w_bf16, int32_t O, int32_t sh, int32_t sw, int32_t relu,
                                 const float *y, float *dy, uint16_t *col, uint16_t *dy_bf16, float *dcol,
                                 float *dx, float *dw, float *db, void *cuda_stream);

/* Nearest-neighbour 2x upsampling of the last two axes: x [C][B][H][W] -> y [C][B][2H][2W],
 * and its gradient dx [C][B][H][W] from dy [C][B][2H][2W] (sums of 2x2 blocks). */
fwi_status fwi_cnn_upsample2(const float *x, int32_t C, int32_t B, int32_t H, int32_t W, float *y,
                             void *cuda_stream);
fwi_status fwi_cnn_upsample2_backward(const float *dy, int32_t C, int32_t B, int32_t H, int32_t W, float *dx,
                                      void *cuda_stream);

/* loss = 1/(2n) sum (p - t)^2 (FP64, one device double) and dp = (p - t) / n. */
fwi_status fwi_cnn_mse(const float *p, const float *t, int64_t n, double *loss, float *dp, void *cuda_stream);

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
