/*
 * fno.h -- C ABI of the Fourier Neural Operator surrogate of the mean flow
 * (Sec. 4 and the appendix on the baseline models of the paper: an FNO that
 * maps the obstacle mask and Re to the time-averaged velocity and pressure,
 * trained with a masked mean square error on the inner region of the
 * channel, Adam, cosine learning-rate schedule).
 *
 * Network (App. B: feed-forward lifting network, Fourier layers, SIREN
 * projection of Sitzmann et al. 2020), for fields laid out
 * [batch][channel][z][y][x] (x fastest):
 *   lift      v0 = P2 GELU(P1 x + bP1) + bP2           (cin -> lift_hidden -> width)
 *   layer l   v_{l+1} = act(K_l v_l + W_l v_l + b_l)   (GELU except after the last)
 *             K_l v = IDFT_r(R_l . DFT_r(v))           (retained modes only)
 *   project   y = Q2 sin(omega0 (Q1 v_L + bQ1)) + bQ2  (width -> hidden -> cout)
 * DFT_r keeps kx in [0,mx) U [-mx,0), ky in [0,my) U [-my,0), kz in [0,mz)
 * (z is the real-to-half-complex axis); the inverse is
 * y(x) = (1/N) Re[sum_k c_kz G(k) exp(+i theta_k . x)], c_0 = 1, c_kz = 2.
 * R_l holds one complex width x width matrix per retained mode.
 *
 * Parameters are one flat FP32 vector, in this order:
 *   R_0 .. R_{layers-1}, each [K][width_in][width_out][re, im] (K = mz*2my*2mx
 *   modes, k = (kz*2my + jy)*2mx + jx; first, so that every complex entry is
 *   8-byte aligned), P1_w [lift_hidden][cin], P1_b [lift_hidden],
 *   P2_w [width][lift_hidden], P2_b [width],
 *   per layer l: W_l_w [width][width], W_l_b [width],
 *   Q1_w [hidden][width], Q1_b [hidden], Q2_w [cout][hidden], Q2_b [cout].
 *
 * Conventions as in lbm.h: every call returns lbm_status; buffers may be
 * host or device memory; work runs on the stream given at creation.
 */
#ifndef GB300_FNO_H
#define GB300_FNO_H

#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fno_ctx fno_ctx;

typedef struct {
    int32_t nx, ny, nz;          /* grid (x streamwise)                            */
    int32_t cin, width, cout;    /* input channels, co-domain width, outputs        */
    int32_t mx, my, mz;          /* retained modes (see above), mz < nz/2          */
    int32_t layers, hidden;      /* Fourier layers, projection hidden width        */
    int32_t max_batch;           /* largest batch a call may pass                  */
    int32_t act_bf16;            /* 1: activations stored in BF16 (else FP32)      */
    int32_t tensor_cores;        /* 1: mode contraction on tensor cores in BF16
                                    with FP32 accumulation (needs width % 8 == 0) */
    int32_t lift_hidden;         /* hidden width of the lifting network (<= 32)    */
    float omega0;                /* SIREN frequency factor (> 0; default 30)       */
    int32_t umma;                /* 1: the forward x stage of BF16 rows (nx = 128,
                                    32 x modes) on tcgen05 tensor cores with TMEM
                                    accumulators and tensor-map loads           */
    int32_t reserved;
    uint64_t seed;               /* initial parameters                             */
} fno_config;

/* Defaults of the channel surrogate: 128x64x64 grid, 4 inputs (mask, log10
 * Re, cos and sin of the angle of attack), lift 4 -> 32 -> 32, width 32, modes
 * 16x8x8, 4 layers, SIREN projection 32 -> 128 -> 4 with omega0 = 30, 4
 * outputs (u, v, w, p), batch 8, BF16 activations, tensor cores.  Initial
 * parameters: uniform within 1/sqrt(fan_in), spectral weights within
 * 1/width^2, SIREN first layer within 1/fan_in and output layer within
 * sqrt(6/fan_in)/omega0 (Sitzmann et al. 2020). */
void fno_config_default(fno_config *c);

lbm_status fno_create(const fno_config *c, void *cuda_stream, fno_ctx **out);
lbm_status fno_destroy(fno_ctx *f);

/* Number of FP32 parameters (the flat vector above). */
int64_t fno_num_params(const fno_ctx *f);

lbm_status fno_set_params(fno_ctx *f, const float *src);
lbm_status fno_get_params(fno_ctx *f, float *dst);
/* Gradients of the last fno_loss_grad / fno_train_step (same layout). */
lbm_status fno_get_grads(fno_ctx *f, float *dst);

/* y [batch][cout][N] FP32 from x [batch][cin][N] FP32 (N = nx*ny*nz). */
lbm_status fno_forward(fno_ctx *f, const float *x, float *y, int32_t batch);

/* Forward and backward of the masked mean square error
 * sum_{b,c,cell} m (y - t)^2 / (cout * sum m); m [batch][N] FP32 weights.
 * Stores the gradients; *loss receives the loss (may be NULL). */
lbm_status fno_loss_grad(fno_ctx *f, const float *x, const float *t, const float *m, int32_t batch,
                         double *loss);

/* One Adam step (beta1, beta2, eps; bias-corrected; real and imaginary parts
 * of the spectral weights handled as separate reals) with the stored
 * gradients at learning rate lr. */
lbm_status fno_adam_step(fno_ctx *f, float lr, float beta1, float beta2, float eps);

/* fno_loss_grad followed by fno_adam_step with beta1 0.9, beta2 0.999, eps 1e-8. */
lbm_status fno_train_step(fno_ctx *f, const float *x, const float *t, const float *m, int32_t batch, float lr,
                          double *loss);

/* Checkpoint of the trained state: the network's shape (every fno_config
 * field that fixes the parameter layout), the Adam step count, and the FP32
 * parameters and both Adam moments, to a binary file ("GBFNOCK1" header).
 * fno_load accepts only a checkpoint of the same shape (LBM_ERR_IO
 * otherwise, the context unchanged) and waits for the stream. */
lbm_status fno_save(fno_ctx *f, const char *path);
lbm_status fno_load(fno_ctx *f, const char *path);

/* Wait for the context's stream and report device conditions: LBM_ERR_TIMEOUT
 * if a bounded wait of the tcgen05 x stage gave up (its output is then not
 * valid; the status word is cleared). */
lbm_status fno_sync(fno_ctx *f);

const char *fno_last_error(const fno_ctx *f);

#ifdef __cplusplus
}
#endif
#endif /* GB300_FNO_H */
