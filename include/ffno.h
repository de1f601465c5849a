/*
 * ffno.h -- C ABI of the factorised Fourier Neural Operator surrogate (the
 * FFNO of the paper's Table 2; its appendix on the baselines: "follows the
 * structure of Tran et al." with the FNO models' modes, channels, lift and
 * projection).
 *
 * Network, for fields laid out [batch][channel][z][y][x] (x fastest):
 *   lift      v0 = P2 GELU(P1 x + bP1) + bP2                 (cin -> lift_hidden -> width)
 *   layer l   u = sum over the axes d = z, y, x of IDFT_d(R_{l,d} . DFT_d(v_l))
 *             v_{l+1} = v_l + F2_l GELU(F1_l u + b1_l) + b2_l (width -> ff_hidden -> width)
 *   project   y = Q2 sin(omega0 (Q1 v_L + bQ1)) + bQ2         (width -> hidden -> cout)
 * DFT_d is the real discrete Fourier transform along axis d alone, the first
 * m_d wave numbers k in [0, m_d) kept: V(k) = sum_n v(n) exp(-2 pi i k n / L_d);
 * IDFT_d(W)(n) = (1/L_d) Re[sum_k c_k W(k) exp(+2 pi i k n / L_d)], c_0 = 1,
 * c_{L_d/2} = 1 (L_d even), otherwise 2.  R_{l,d} holds one complex
 * width x width matrix per wave number: W(b, o, ., k) = sum_i V(b, i, ., k) R(i, o, k).
 *
 * Parameters are one flat FP32 vector, in this order: P1_w [lift_hidden][cin],
 * P1_b, P2_w [width][lift_hidden], P2_b; per layer l: R_{l,z}, R_{l,y},
 * R_{l,x}, each [width_in][width_out][m_d][re, im], F1_w [ff_hidden][width],
 * F1_b, F2_w [width][ff_hidden], F2_b; then Q1_w [hidden][width], Q1_b,
 * Q2_w [cout][hidden], Q2_b.
 *
 * This first GPU path computes in FP32 with one thread per output element
 * (transforms as explicit sums against twiddle tables).  Conventions as in
 * lbm.h: every call returns lbm_status; x, t, m and y may be host or device
 * memory; work runs on the stream given at creation.
 */
#ifndef GB300_FFNO_H
#define GB300_FFNO_H

#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffno_ctx ffno_ctx;

typedef struct {
    int32_t nx, ny, nz;          /* grid (x streamwise)                                */
    int32_t cin, width, cout;    /* input channels, channel width, outputs             */
    int32_t mx, my, mz;          /* wave numbers kept along x, y, z (<= L/2 + 1)       */
    int32_t layers;              /* factorised Fourier layers                          */
    int32_t ff_hidden;           /* hidden width of each layer's feed-forward block    */
    int32_t hidden;              /* SIREN projection hidden width                      */
    int32_t lift_hidden;         /* hidden width of the lifting network                */
    int32_t max_batch;           /* largest batch a call may pass                      */
    float omega0;                /* SIREN frequency factor (> 0)                       */
    int32_t reserved;
    uint64_t seed;               /* initial parameters                                 */
} ffno_config;

/* Defaults of the channel surrogate: 128x64x64 grid, 4 inputs, width 32,
 * wave numbers 32, 16, 16 along x, y, z (the paper's 32 x 16 x 16 modes),
 * 4 layers, feed-forward width 32, lift 4 -> 32 -> 32, SIREN 32 -> 128 -> 4
 * with omega0 = 30, batch 8. */
void ffno_config_default(ffno_config *c);

lbm_status ffno_create(const ffno_config *c, void *cuda_stream, ffno_ctx **out);
lbm_status ffno_destroy(ffno_ctx *f);

/* Number of FP32 parameters (the flat vector above). */
int64_t ffno_num_params(const ffno_ctx *f);
lbm_status ffno_set_params(ffno_ctx *f, const float *src);
lbm_status ffno_get_params(ffno_ctx *f, float *dst);
/* Gradients of the last ffno_loss_grad (same layout). */
lbm_status ffno_get_grads(ffno_ctx *f, float *dst);

/* y [batch][cout][nz][ny][nx] from x [batch][cin][nz][ny][nx]. */
lbm_status ffno_forward(ffno_ctx *f, const float *x, float *y, int32_t batch);
/* Masked mean square error sum_{b,c,n} m(b,n) (y - t)^2 / (cout sum m) and its
 * gradients with respect to every parameter; m [batch][nz][ny][nx]. */
lbm_status ffno_loss_grad(ffno_ctx *f, const float *x, const float *t, const float *m, int32_t batch,
                          double *loss);
/* One bias-corrected Adam step on the gradients of the last ffno_loss_grad. */
lbm_status ffno_adam_step(ffno_ctx *f, float lr, float b1, float b2, float eps);

lbm_status ffno_sync(ffno_ctx *f);
const char *ffno_last_error(const ffno_ctx *f);

#ifdef __cplusplus
}
#endif

#endif
