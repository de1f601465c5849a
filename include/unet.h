/*
 * unet.h -- C ABI of the U-Net surrogate of the mean flow (Sec. 4, Table 2,
 * and the appendix on the baseline models of the paper: a 3-D encoder-decoder
 * with skip connections that maps the obstacle mask and Re to the
 * time-averaged velocity and pressure; the best of the paper's surrogates).
 *
 * Network, for fields laid out [batch][channel][z][y][x] (x fastest) at the
 * boundary:
 *   block(c_in -> c)  : y = ReLU(BN(conv3(x)))   conv3: 3x3x3, zero padding 1,
 *                       stride 1, no bias; BN: batch statistics over
 *                       (batch, z, y, x), biased variance, eps 1e-5, affine
 *   encoder stage e   : two blocks (c_{e-1} -> c_e -> c_e), the output kept as
 *                       the skip s_e, then 2x2x2 max-pooling (stride 2)
 *   bottleneck        : two blocks (c_last -> bottleneck -> bottleneck)
 *   decoder stage d   : trilinear up-sampling by 2 of the stage below
 *                       (cell-centred: output o samples input (o + 1/2)/2 - 1/2,
 *                       clamped to the grid), concatenated after s_d along the
 *                       channels, then two blocks (c_d + c_below -> c_d -> c_d)
 *   output            : y = sigmoid(W_out h + b_out)   (1x1x1 convolution)
 * Loss: masked mean square error sum m (y - t)^2 / (cout * sum m).
 *
 * Parameters are one flat FP32 vector, in this order: for every block in
 * forward order (enc0a, enc0b, enc1a, ..., mida, midb, dec{n-1}a, dec{n-1}b,
 * ..., dec0a, dec0b): w [c_out][c_in][3][3][3], gamma [c_out], beta [c_out];
 * then W_out [cout][c_0], b_out [cout].
 *
 * On the device the activations are BF16, channel-last ([batch][z][y][x][c])
 * with FP32 accumulation; the convolutions (forward, input gradient, weight
 * gradient) run as implicit GEMMs on the tcgen05 tensor cores with the
 * accumulators in tensor memory and the operand tiles loaded by tensor-map
 * copies (zero padding from the copies' out-of-range fill).
 *
 * Conventions as in lbm.h: every call returns lbm_status; x, t, m and y may be
 * host or device memory; work runs on the stream given at creation.  Every
 * device-side wait of the tensor-core kernels is bounded: unet_sync reports
 * one that gave up as LBM_ERR_TIMEOUT.
 */
#ifndef GB300_UNET_H
#define GB300_UNET_H

#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct unet_ctx unet_ctx;

typedef struct {
    int32_t nx, ny, nz;          /* grid; each a power of two divisible by 2^stages */
    int32_t cin, cout;           /* input channels (<= 32), outputs                 */
    int32_t stages;              /* encoder stages (1..4)                           */
    int32_t channels[4];         /* channels of the encoder stages (multiples of 32) */
    int32_t bottleneck;          /* bottleneck channels (multiple of 32)            */
    int32_t max_batch;           /* largest batch a call may pass                   */
    int32_t reserved[2];
    uint64_t seed;               /* initial parameters                              */
} unet_config;

/* The paper's configuration: 128x64x64 grid, 4 inputs (mask, log10 Re, cos
 * and sin of the angle of attack), encoder [32, 64, 128, 256], bottleneck
 * 512, 4 outputs (u, v, w, p), batch 8.  Initial parameters: He-normal
 * convolution weights (std sqrt(2 / (27 c_in))), gamma 1, beta 0, W_out
 * uniform within 1/sqrt(c_0), b_out 0. */
void unet_config_default(unet_config *c);

lbm_status unet_create(const unet_config *c, void *cuda_stream, unet_ctx **out);
lbm_status unet_destroy(unet_ctx *u);

/* Number of FP32 parameters (the flat vector above). */
int64_t unet_num_params(const unet_ctx *u);

lbm_status unet_set_params(unet_ctx *u, const float *src);
lbm_status unet_get_params(unet_ctx *u, float *dst);
/* Gradients of the last unet_loss_grad / unet_train_step (same layout). */
lbm_status unet_get_grads(unet_ctx *u, float *dst);

/* y [batch][cout][N] FP32 from x [batch][cin][N] FP32 (N = nx*ny*nz); the
 * batch normalisation uses the statistics of this batch (training mode, as
 * the network is defined); batch <= max_batch. */
lbm_status unet_forward(unet_ctx *u, const float *x, float *y, int32_t batch);

/* Forward and backward of the masked mean square error; m [batch][N] FP32
 * weights.  Stores the gradients; *loss receives the loss (may be NULL). */
lbm_status unet_loss_grad(unet_ctx *u, const float *x, const float *t, const float *m, int32_t batch,
                          double *loss);

/* One Adam step (beta1, beta2, eps; bias-corrected) with the stored
 * gradients at learning rate lr. */
lbm_status unet_adam_step(unet_ctx *u, float lr, float beta1, float beta2, float eps);

/* unet_loss_grad followed by unet_adam_step with beta1 0.9, beta2 0.999,
 * eps 1e-8. */
lbm_status unet_train_step(unet_ctx *u, const float *x, const float *t, const float *m, int32_t batch, float lr,
                           double *loss);

/* Wait for the stream; LBM_ERR_TIMEOUT if a bounded wait of a tensor-core
 * kernel gave up since the last call (its outputs are then not valid; the
 * status word is cleared). */
lbm_status unet_sync(unet_ctx *u);

const char *unet_last_error(const unet_ctx *u);

/* The network's convolution alone, for checking and reuse; device buffers,
 * channel-last FP32, converted to BF16 on entry (the products are exact,
 * the sums FP32).  Grids as above (powers of two), channels multiples of 32.
 *   unet_conv3_forward       y[b][p][o] = sum_{d,i} w[o][i][d] x[b][p + d - 1][i]
 *   unet_conv3_backward_data gx[b][p][i] = sum_{d,o} w[o][i][d] gy[b][p - d + 1][o]
 *   unet_conv3_backward_weights gw[o][i][d] = sum_{b,p} gy[b][p][o] x[b][p + d - 1][i]
 * x [batch][nz][ny][nx][cin], y and gy [batch][nz][ny][nx][cout], w and gw
 * [cout][cin][27] (d = (dz*3 + dy)*3 + dx), zero outside the grid.  The call
 * allocates its own temporaries and waits for the stream; status as
 * unet_sync. */
lbm_status unet_conv3_forward(const float *x, const float *w, float *y, int32_t batch, int32_t nx, int32_t ny,
                              int32_t nz, int32_t cin, int32_t cout, void *cuda_stream);
lbm_status unet_conv3_backward_data(const float *gy, const float *w, float *gx, int32_t batch, int32_t nx, int32_t ny,
                                    int32_t nz, int32_t cin, int32_t cout, void *cuda_stream);
lbm_status unet_conv3_backward_weights(const float *x, const float *gy, float *gw, int32_t batch, int32_t nx,
                                       int32_t ny, int32_t nz, int32_t cin, int32_t cout, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GB300_UNET_H */
