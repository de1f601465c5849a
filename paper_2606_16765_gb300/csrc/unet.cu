// unet.cu -- the U-Net surrogate of include/unet.h: forward, hand-written
// backward and Adam, with the convolutions on the tcgen05 tensor cores
// (unet_gemm.cu) and the rest in the kernels below.
//
// Activations are BF16, channel-last [batch][z][y][x][c], so that a cell's
// channels are one contiguous run: the convolutions read them as GEMM rows
// and the element-wise kernels below move 8 channels (16 bytes) per access.
//   k_pack_input     x [B][cin][N] FP32 -> [B][N][32] BF16 (channels padded
//                    with zeros to the 32 the tensor cores take per row)
//   k_pack_w         FP32 weights [o][i][27] -> BF16 [27][o][i] (forward) and
//                    [27][i][o] with the taps reversed (input gradient)
//   k_bn_stats/final batch statistics: per-channel FP32 block partials of
//                    z and z^2, combined in FP64 into mean and 1/sigma, and the
//                    affine map a z + b of the normalisation
//   k_bn_apply       y = max(a z + b, 0), into the block's own buffer or the
//                    skip slot of the decoder's concatenation buffer
//   k_maxpool        2x2x2 maximum (the first maximum in (dz, dy, dx) order
//                    is the one the backward routes to)
//   k_up_concat      trilinear x2 up-sampling into the second channel slot of
//                    the concatenation buffer
//   k_out_fwd        1x1x1 output convolution + sigmoid, [B][cout][N] FP32
//   k_loss_*         masked mean square error, FP64 sums
//   k_out_bwd/wgrad  output layer gradients
//   k_bn_bwd_*       ReLU and batch-normalisation backward (two reductions,
//                    then the input gradient of the normalisation)
//   k_pool_bwd       max-pooling backward plus the skip connection's gradient
//   k_up_bwd         adjoint of the up-sampling
//   k_wg_convert     weight gradient [(tap, i)][o] -> the parameter layout
//   k_adam           Adam update of the flat FP32 parameter vector
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/unet.h"
#include "sm_count.h"
#include "unet_gemm.h"

namespace {

typedef __nv_bfloat16 bf16;
constexpr int TPB = 256;
constexpr double BN_EPS = 1e-5;
constexpr int CPAD = 32;                       // input channels as stored for the first convolution

int grid_for(int64_t n)
{
    const int64_t b = (n + TPB - 1) / TPB;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)gb300::sm_count() * 8));
}

__device__ __forceinline__ void ld8(const bf16 *p, float *v)
{
    const uint4 u = *reinterpret_cast<const uint4 *>(p);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 f = __bfloat1622float2(h[q]);
        v[2 * q] = f.x;
        v[2 * q + 1] = f.y;
    }
}

__device__ __forceinline__ void st8(bf16 *p, const float *v)
{
    uint4 u;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
    for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
    *reinterpret_cast<uint4 *>(p) = u;
}

// ---------------------------------------------------------------------------
// layout conversions
// ---------------------------------------------------------------------------
__global__ void k_pack_input(const float *__restrict__ x, int64_t N, int B, int cin, bf16 *__restrict__ x0)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)B * N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / N, p = i % N;
        float v[CPAD];
#pragma unroll
        for (int c = 0; c < CPAD; ++c) v[c] = c < cin ? x[(b * cin + c) * N + p] : 0.f;
#pragma unroll
        for (int q = 0; q < CPAD / 8; ++q) st8(x0 + i * CPAD + 8 * q, v + 8 * q);
    }
}

__global__ void k_f2bf(const float *__restrict__ s, bf16 *__restrict__ d, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = __float2bfloat16_rn(s[i]);
}

// w [o][i][27] FP32 -> wf [27][o][ip] (i < cin, zeros above) and, if given,
// wb [26 - d][ip][o] (the same values with the taps reversed, transposed).
__global__ void k_pack_w(const float *__restrict__ w, int cout, int cin, int ip, bf16 *__restrict__ wf,
                         bf16 *__restrict__ wb)
{
    const int64_t n = (int64_t)27 * cout * ip;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(k / ((int64_t)cout * ip));
        const int r = (int)(k % ((int64_t)cout * ip));
        const int o = r / ip, i = r % ip;
        const bf16 v = __float2bfloat16_rn(i < cin ? w[((int64_t)o * cin + i) * 27 + d] : 0.f);
        wf[k] = v;
        if (wb) wb[((int64_t)(26 - d) * ip + i) * cout + o] = v;
    }
}

// gwt [(d * ip + i)][o] -> gw [o][i][d]
__global__ void k_wg_convert(const float *__restrict__ gwt, int cin, int ip, int cout, float *__restrict__ gw)
{
    const int64_t n = (int64_t)cout * cin * 27;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(k % 27);
        const int64_t r = k / 27;
        const int i = (int)(r % cin), o = (int)(r / cin);
        gw[k] = gwt[((int64_t)d * ip + i) * cout + o];
    }
}

// ---------------------------------------------------------------------------
// batch normalisation + ReLU
// ---------------------------------------------------------------------------
// Per-block partial sums over cells of two per-channel quantities:
// mode 0: (z, z^2); mode 1: (gn, gn * xh) with gn = gy [a z + b > 0],
// xh = (z - mu) / sigma (coef = a, b, mu, 1/sigma).
template <int MODE>
__global__ void __launch_bounds__(TPB) k_bn_reduce(const bf16 *__restrict__ z, const bf16 *__restrict__ gy, int ldgy,
                                                   int64_t cells, int C, const float *__restrict__ coef,
                                                   float2 *__restrict__ part)
{
    __shared__ float red[2][TPB * 8];
    const int g8 = C / 8, rows = TPB / g8;
    const int g = threadIdx.x % g8, r = threadIdx.x / g8;
    float s[8], q[8], ca[8], cb[8], cm[8], cr[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        s[j] = q[j] = 0.f;
        if (MODE == 1) {
            ca[j] = coef[g * 8 + j];
            cb[j] = coef[C + g * 8 + j];
            cm[j] = coef[2 * C + g * 8 + j];
            cr[j] = coef[3 * C + g * 8 + j];
        }
    }
    if (r < rows) {
        for (int64_t cell = (int64_t)blockIdx.x * rows + r; cell < cells; cell += (int64_t)gridDim.x * rows) {
            float v[8];
            ld8(z + cell * C + g * 8, v);
            if (MODE == 0) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    s[j] += v[j];
                    q[j] += v[j] * v[j];
                }
            } else {
                float gv[8];
                ld8(gy + cell * ldgy + g * 8, gv);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float gn = (ca[j] * v[j] + cb[j] > 0.f) ? gv[j] : 0.f;
                    s[j] += gn;
                    q[j] += gn * ((v[j] - cm[j]) * cr[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            red[0][r * C + g * 8 + j] = s[j];
            red[1][r * C + g * 8 + j] = q[j];
        }
    }
    __syncthreads();
    for (int ch = threadIdx.x; ch < C; ch += blockDim.x) {
        float a = 0.f, b = 0.f;
        for (int rr = 0; rr < rows; ++rr) {
            a += red[0][rr * C + ch];
            b += red[1][rr * C + ch];
        }
        part[(int64_t)blockIdx.x * C + ch] = make_float2(a, b);
    }
}

int bn_blocks(int64_t cells, int C)
{
    const int rows = TPB / (C / 8);
    return (int)std::max<int64_t>(1, std::min<int64_t>((cells + rows - 1) / rows, (int64_t)gb300::sm_count() * 4));
}

// mean, 1/sigma (biased variance + eps) and a = gamma / sigma, b = beta - mu a
__global__ void k_bn_final(const float2 *__restrict__ part, int P, int C, double M, const float *__restrict__ gamma,
                           const float *__restrict__ beta, float *__restrict__ coef)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double S = 0.0, Q = 0.0;
    for (int p = 0; p < P; ++p) {
        const float2 v = part[(int64_t)p * C + c];
        S += v.x;
        Q += v.y;
    }
    const double mu = S / M;
    const double var = std::max(Q / M - mu * mu, 0.0);
    const double rs = 1.0 / std::sqrt(var + BN_EPS);
    const double a = (double)gamma[c] * rs;
    coef[c] = (float)a;
    coef[C + c] = (float)((double)beta[c] - mu * a);
    coef[2 * C + c] = (float)mu;
    coef[3 * C + c] = (float)rs;
}

__global__ void k_bn_apply(const bf16 *__restrict__ z, int64_t cells, int C, const float *__restrict__ coef,
                           bf16 *__restrict__ y, int ldy, int yoff)
{
    const int g8 = C / 8;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cells * g8; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = k / g8;
        const int g = (int)(k % g8);
        float v[8];
        ld8(z + cell * C + g * 8, v);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = fmaxf(coef[g * 8 + j] * v[j] + coef[C + g * 8 + j], 0.f);
        st8(y + cell * ldy + yoff + g * 8, v);
    }
}

// ggamma = sum gn xh, gbeta = sum gn; k3 = (gamma / sigma, mean gn, mean gn xh)
__global__ void k_bn_bwd_final(const float2 *__restrict__ part, int P, int C, double M, const float *__restrict__ coef,
                               const float *__restrict__ gamma, float *__restrict__ ggamma, float *__restrict__ gbeta,
                               float *__restrict__ k3)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double S1 = 0.0, S2 = 0.0;
    for (int p = 0; p < P; ++p) {
        const float2 v = part[(int64_t)p * C + c];
        S1 += v.x;
        S2 += v.y;
    }
    ggamma[c] = (float)S2;
    gbeta[c] = (float)S1;
    k3[c] = gamma[c] * coef[3 * C + c];
    k3[C + c] = (float)(S1 / M);
    k3[2 * C + c] = (float)(S2 / M);
}

// gz = gamma / sigma (gn - mean gn - xh mean(gn xh))
__global__ void k_bn_bwd_apply(const bf16 *__restrict__ z, const bf16 *__restrict__ gy, int ldgy, int64_t cells, int C,
                               const float *__restrict__ coef, const float *__restrict__ k3, bf16 *__restrict__ gz)
{
    const int g8 = C / 8;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cells * g8; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = k / g8;
        const int g = (int)(k % g8);
        float v[8], gv[8];
        ld8(z + cell * C + g * 8, v);
        ld8(gy + cell * ldgy + g * 8, gv);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = g * 8 + j;
            const float gn = (coef[c] * v[j] + coef[C + c] > 0.f) ? gv[j] : 0.f;
            const float xh = (v[j] - coef[2 * C + c]) * coef[3 * C + c];
            v[j] = k3[c] * (gn - k3[C + c] - xh * k3[2 * C + c]);
        }
        st8(gz + cell * C + g * 8, v);
    }
}

// ---------------------------------------------------------------------------
// pooling, up-sampling
// ---------------------------------------------------------------------------
__global__ void k_maxpool(const bf16 *__restrict__ y, int ldy, int X, int Y, int Z, int B, int C, bf16 *__restrict__ p)
{
    const int Xc = X / 2, Yc = Y / 2, Zc = Z / 2, g8 = C / 8;
    const int64_t n = (int64_t)B * Zc * Yc * Xc * g8;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(k % g8);
        int64_t r = k / g8;
        const int xc = (int)(r % Xc), yc = (int)((r / Xc) % Yc), zc = (int)((r / ((int64_t)Xc * Yc)) % Zc);
        const int64_t b = r / ((int64_t)Xc * Yc * Zc);
        float best[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) best[j] = -INFINITY;
        for (int q = 0; q < 8; ++q) {
            const int64_t f = ((b * Z + 2 * zc + (q >> 2)) * Y + 2 * yc + ((q >> 1) & 1)) * X + 2 * xc + (q & 1);
            float v[8];
            ld8(y + f * ldy + g * 8, v);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (v[j] > best[j]) best[j] = v[j];
        }
        st8(p + r * C + g * 8, best);
    }
}

// g[fine] = (fine is its window's first maximum of y ? gp[coarse] : 0) + gs[fine]
__global__ void k_pool_bwd(const bf16 *__restrict__ gp, const bf16 *__restrict__ y, int ldy,
                           const bf16 *__restrict__ gs, int ldgs, int X, int Y, int Z, int B, int C,
                           bf16 *__restrict__ g)
{
    const int Xc = X / 2, Yc = Y / 2, Zc = Z / 2, g8 = C / 8;
    const int64_t n = (int64_t)B * Zc * Yc * Xc * g8;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int gi = (int)(k % g8);
        const int64_t r = k / g8;
        const int xc = (int)(r % Xc), yc = (int)((r / Xc) % Yc), zc = (int)((r / ((int64_t)Xc * Yc)) % Zc);
        const int64_t b = r / ((int64_t)Xc * Yc * Zc);
        float best[8];
        int arg[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            best[j] = -INFINITY;
            arg[j] = 0;
        }
        int64_t fine[8];
        for (int q = 0; q < 8; ++q) {
            fine[q] = ((b * Z + 2 * zc + (q >> 2)) * Y + 2 * yc + ((q >> 1) & 1)) * X + 2 * xc + (q & 1);
            float v[8];
            ld8(y + fine[q] * ldy + gi * 8, v);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (v[j] > best[j]) {
                    best[j] = v[j];
                    arg[j] = q;
                }
        }
        float gv[8];
        ld8(gp + r * C + gi * 8, gv);
        for (int q = 0; q < 8; ++q) {
            float o[8];
            if (gs)
                ld8(gs + fine[q] * ldgs + gi * 8, o);
            else
#pragma unroll
                for (int j = 0; j < 8; ++j) o[j] = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (arg[j] == q) o[j] += gv[j];
            st8(g + fine[q] * C + gi * 8, o);
        }
    }
}

// Cell-centred linear up-sampling by 2 along an axis of n samples: output o
// sits at s = (o + 1/2)/2 - 1/2 in input coordinates, clamped to [0, n - 1].
__device__ __forceinline__ void up_coord(int o, int n, int &i0, int &i1, float &w)
{
    float s = (o + 0.5f) * 0.5f - 0.5f;
    s = fminf(fmaxf(s, 0.f), (float)(n - 1));
    i0 = (int)floorf(s);
    i1 = min(i0 + 1, n - 1);
    w = s - (float)i0;
}

// weight of input sample j in output sample o
__device__ __forceinline__ float up_weight(int o, int j, int n)
{
    int i0, i1;
    float w;
    up_coord(o, n, i0, i1, w);
    return (i0 == j ? 1.f - w : 0.f) + (i1 == j ? w : 0.f);
}

__global__ void k_up_concat(const bf16 *__restrict__ h, int Xc, int Yc, int Zc, int B, int cb, bf16 *__restrict__ cat,
                            int ldc, int off)
{
    const int X = 2 * Xc, Y = 2 * Yc, Z = 2 * Zc, g8 = cb / 8;
    const int64_t n = (int64_t)B * Z * Y * X * g8;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(k % g8);
        const int64_t r = k / g8;
        const int x = (int)(r % X), y = (int)((r / X) % Y), z = (int)((r / ((int64_t)X * Y)) % Z);
        const int64_t b = r / ((int64_t)X * Y * Z);
        int xi[2], yi[2], zi[2];
        float wx, wy, wz;
        up_coord(x, Xc, xi[0], xi[1], wx);
        up_coord(y, Yc, yi[0], yi[1], wy);
        up_coord(z, Zc, zi[0], zi[1], wz);
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int q = 0; q < 8; ++q) {
            const int a = q >> 2, bb = (q >> 1) & 1, cc = q & 1;
            const float wt = (a ? wz : 1.f - wz) * (bb ? wy : 1.f - wy) * (cc ? wx : 1.f - wx);
            if (wt == 0.f) continue;
            const int64_t src = ((b * Zc + zi[a]) * Yc + yi[bb]) * Xc + xi[cc];
            float v[8];
            ld8(h + src * cb + g * 8, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += wt * v[j];
        }
        st8(cat + r * ldc + off + g * 8, acc);
    }
}

__global__ void k_up_bwd(const bf16 *__restrict__ gc, int ldc, int off, int Xc, int Yc, int Zc, int B, int cb,
                         bf16 *__restrict__ gh)
{
    const int X = 2 * Xc, Y = 2 * Yc, Z = 2 * Zc, g8 = cb / 8;
    const int64_t n = (int64_t)B * Zc * Yc * Xc * g8;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(k % g8);
        const int64_t r = k / g8;
        const int xc = (int)(r % Xc), yc = (int)((r / Xc) % Yc), zc = (int)((r / ((int64_t)Xc * Yc)) % Zc);
        const int64_t b = r / ((int64_t)Xc * Yc * Zc);
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int oz = max(0, 2 * zc - 1); oz <= min(Z - 1, 2 * zc + 2); ++oz) {
            const float wz = up_weight(oz, zc, Zc);
            if (wz == 0.f) continue;
            for (int oy = max(0, 2 * yc - 1); oy <= min(Y - 1, 2 * yc + 2); ++oy) {
                const float wy = up_weight(oy, yc, Yc);
                if (wy == 0.f) continue;
                for (int ox = max(0, 2 * xc - 1); ox <= min(X - 1, 2 * xc + 2); ++ox) {
                    const float wx = up_weight(ox, xc, Xc);
                    if (wx == 0.f) continue;
                    const int64_t f = ((b * Z + oz) * Y + oy) * X + ox;
                    float v[8];
                    ld8(gc + f * ldc + off + g * 8, v);
                    const float wt = wz * wy * wx;
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[j] += wt * v[j];
                }
            }
        }
        st8(gh + r * cb + g * 8, acc);
    }
}

// ---------------------------------------------------------------------------
// output layer and loss
// ---------------------------------------------------------------------------
constexpr int MAXOUT = 8;

__global__ void k_out_fwd(const bf16 *__restrict__ h, int c0, const float *__restrict__ ow, const float *__restrict__ ob,
                          int cout, int64_t N, int B, float *__restrict__ y)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)B * N;
         i += (int64_t)gridDim.x * blockDim.x) {
        float acc[MAXOUT];
        for (int o = 0; o < cout; ++o) acc[o] = ob[o];
        for (int c = 0; c < c0; c += 8) {
            float v[8];
            ld8(h + i * c0 + c, v);
            for (int o = 0; o < cout; ++o)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[o] += ow[o * c0 + c + j] * v[j];
        }
        const int64_t b = i / N, p = i % N;
        for (int o = 0; o < cout; ++o) y[(b * cout + o) * N + p] = 1.f / (1.f + expf(-acc[o]));
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// per block: sum m (y - t)^2 over channels and sum m
__global__ void __launch_bounds__(TPB) k_loss_partial(const float *__restrict__ y, const float *__restrict__ t,
                                                      const float *__restrict__ m, int64_t N, int B, int cout,
                                                      double2 *__restrict__ part)
{
    __shared__ double sh[2][TPB / 32];
    double a = 0.0, s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)B * N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / N, p = i % N;
        const float mv = m[i];
        s += mv;
        float e = 0.f;
        for (int o = 0; o < cout; ++o) {
            const float d = y[(b * cout + o) * N + p] - t[(b * cout + o) * N + p];
            e += d * d;
        }
        a += (double)mv * e;
    }
    a = warp_sum(a);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = a;
        sh[1][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, S = 0.0;
        for (int w = 0; w < TPB / 32; ++w) {
            A += sh[0][w];
            S += sh[1][w];
        }
        part[blockIdx.x] = make_double2(A, S);
    }
}

__global__ void k_loss_final(const double2 *__restrict__ part, int P, int cout, double *__restrict__ res)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double A = 0.0, S = 0.0;
    for (int p = 0; p < P; ++p) {
        A += part[p].x;
        S += part[p].y;
    }
    res[0] = S > 0.0 ? A / (cout * S) : 0.0;
    res[1] = S;
}

// ga = dL/da of the output pre-activation, [cells][cout]; gh = W_out^T ga (BF16)
__global__ void k_out_bwd(const float *__restrict__ y, const float *__restrict__ t, const float *__restrict__ m,
                          const float *__restrict__ ow, const double *__restrict__ res, int64_t N, int B, int cout,
                          int c0, float *__restrict__ ga, bf16 *__restrict__ gh)
{
    const double S = res[1];
    const float scale = S > 0.0 ? (float)(2.0 / (cout * S)) : 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)B * N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / N, p = i % N;
        const float mv = m[i];
        float g[MAXOUT];
        for (int o = 0; o < cout; ++o) {
            const float yv = y[(b * cout + o) * N + p];
            g[o] = scale * mv * (yv - t[(b * cout + o) * N + p]) * yv * (1.f - yv);
            ga[i * cout + o] = g[o];
        }
        for (int c = 0; c < c0; c += 8) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float s = 0.f;
                for (int o = 0; o < cout; ++o) s += ow[o * c0 + c + j] * g[o];
                v[j] = s;
            }
            st8(gh + i * c0 + c, v);
        }
    }
}

// per block partial sums of ga[o] h[c] (o-major) and ga[o]
__global__ void __launch_bounds__(TPB) k_out_wgrad(const float *__restrict__ ga, const bf16 *__restrict__ h,
                                                   int64_t cells, int cout, int c0, float *__restrict__ part)
{
    const int nq = cout * c0 + cout;
    const int64_t per = (cells + gridDim.x - 1) / gridDim.x;
    const int64_t c_begin = (int64_t)blockIdx.x * per, c_end = std::min<int64_t>(cells, c_begin + per);
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        float acc = 0.f;
        if (q < cout * c0) {
            const int o = q / c0, c = q % c0;
            for (int64_t i = c_begin; i < c_end; ++i) acc += ga[i * cout + o] * __bfloat162float(h[i * c0 + c]);
        } else {
            const int o = q - cout * c0;
            for (int64_t i = c_begin; i < c_end; ++i) acc += ga[i * cout + o];
        }
        part[(int64_t)blockIdx.x * nq + q] = acc;
    }
}

__global__ void k_sum_parts(const float *__restrict__ part, int P, int n, float *__restrict__ out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double s = 0.0;
    for (int p = 0; p < P; ++p) s += part[(int64_t)p * n + q];
    out[q] = (float)s;
}

__global__ void k_adam(float *p, const float *g, float *m1, float *m2, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float gv = g[k];
        const float a = b1 * m1[k] + (1.f - b1) * gv;
        const float b = b2 * m2[k] + (1.f - b2) * gv * gv;
        m1[k] = a;
        m2[k] = b;
        p[k] -= lr * (a * c1) / (sqrtf(b * c2) + eps);
    }
}

bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

thread_local std::string g_unet_err;

struct Blk {
    int cin = 0, cout = 0, ip = 0, level = 0;      // ip: stored input channels (multiple of 32)
    int64_t ow = 0, og = 0, ob = 0;                 // parameter offsets
    bf16 *wf = nullptr, *wb = nullptr;              // packed weights (wb: null for the first block)
    const bf16 *x = nullptr;                        // input [cells][ip]
    bf16 *z = nullptr;                              // convolution output [cells][cout]
    bf16 *y = nullptr;                              // BN + ReLU output (row stride ldy, offset yoff)
    int ldy = 0, yoff = 0;
    float *coef = nullptr, *k3 = nullptr;           // [4][cout], [3][cout]
    bf16 *gz = nullptr, *gx = nullptr;              // gradients [cells][cout], [cells][ip]
    unet::ConvPlan fwd, bwd;
    unet::WgradPlan wg;
};

}  // namespace

struct unet_ctx {
    unet_config c{};
    cudaStream_t s = nullptr;
    int S = 0;
    int64_t N = 0, np = 0;
    std::vector<Blk> blk;                          // forward order
    int64_t oOw = 0, oOb = 0;
    float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
    int64_t adam_t = 0;
    std::vector<void *> allocs;
    bf16 *x0 = nullptr;
    float *xin = nullptr, *tin = nullptr, *min = nullptr, *y = nullptr, *ga = nullptr;
    bf16 *gh0 = nullptr;
    std::vector<bf16 *> cat, pool, gup, gyb;
    float *gwt = nullptr;
    float2 *part = nullptr;
    int part_max = 0;
    double2 *lpart = nullptr;
    double *res = nullptr;
    float *opart = nullptr;
    int *ustatus = nullptr;
    int planned_B = 0;
    std::string err;

    template <class T> T *alloc(size_t count)
    {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 16)) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        return static_cast<T *>(p);
    }
    int X(int l) const { return c.nx >> l; }
    int Y(int l) const { return c.ny >> l; }
    int Z(int l) const { return c.nz >> l; }
    int64_t cells(int l, int B) const { return (int64_t)B * X(l) * Y(l) * Z(l); }
    int below(int e) const { return e + 1 < S ? c.channels[e + 1] : c.bottleneck; }
};

#define UCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            u->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return LBM_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)

namespace {

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double unif01(uint64_t &s) { return ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

// Box-Muller normal deviate
double normal(uint64_t &s)
{
    const double a = unif01(s), b = unif01(s);
    return std::sqrt(-2.0 * std::log(a)) * std::cos(6.283185307179586 * b);
}

lbm_status pack_weights(unet_ctx *u)
{
    for (Blk &b : u->blk)
        k_pack_w<<<grid_for((int64_t)27 * b.cout * b.ip), TPB, 0, u->s>>>(u->params + b.ow, b.cout, b.cin, b.ip, b.wf,
                                                                          b.wb);
    UCK(cudaGetLastError());
    return LBM_OK;
}

lbm_status plan(unet_ctx *u, int B)
{
    if (u->planned_B == B) return LBM_OK;
    const int sms = gb300::sm_count();
    for (Blk &b : u->blk) {
        const int l = b.level;
        const char *e = nullptr;
        if (!unet::conv_plan(b.fwd, b.x, b.ip, b.ip, u->X(l), u->Y(l), u->Z(l), B, b.wf, b.cout, 27, b.cout, 0, sms, &e) ||
            (b.gx && !unet::conv_plan(b.bwd, b.gz, b.cout, b.cout, u->X(l), u->Y(l), u->Z(l), B, b.wb, b.ip, 27, b.ip, 0,
                                      sms, &e)) ||
            !unet::wgrad_plan(b.wg, b.x, b.ip, b.ip, b.gz, b.cout, b.cout, u->X(l), u->Y(l), u->Z(l), B, sms, &e)) {
            u->err = std::string("tensor-core plan failed: ") + (e ? e : "?");
            u->planned_B = 0;
            return LBM_ERR_ARG;
        }
    }
    u->planned_B = B;
    return LBM_OK;
}

void run_block(unet_ctx *u, Blk &b, int B)
{
    const int64_t n = u->cells(b.level, B);
    unet::conv_launch(b.fwd, b.z, false, u->ustatus, u->s);
    const int P = bn_blocks(n, b.cout);
    k_bn_reduce<0><<<P, TPB, 0, u->s>>>(b.z, nullptr, 0, n, b.cout, nullptr, u->part);
    k_bn_final<<<(b.cout + 127) / 128, 128, 0, u->s>>>(u->part, P, b.cout, (double)n, u->params + b.og,
                                                        u->params + b.ob, b.coef);
    k_bn_apply<<<grid_for(n * b.cout / 8), TPB, 0, u->s>>>(b.z, n, b.cout, b.coef, b.y, b.ldy, b.yoff);
}

lbm_status forward_impl(unet_ctx *u, int B)
{
    lbm_status st = plan(u, B);
    if (st != LBM_OK) return st;
    const unet_config &c = u->c;
    const int S = u->S;
    k_pack_input<<<grid_for(u->cells(0, B)), TPB, 0, u->s>>>(u->xin, u->N, B, c.cin, u->x0);
    int k = 0;
    for (int e = 0; e < S; ++e) {
        run_block(u, u->blk[k++], B);
        run_block(u, u->blk[k++], B);
        const int ce = c.channels[e];
        k_maxpool<<<grid_for(u->cells(e + 1, B) * ce / 8), TPB, 0, u->s>>>(u->cat[e], ce + u->below(e), u->X(e), u->Y(e),
                                                                           u->Z(e), B, ce, u->pool[e]);
    }
    run_block(u, u->blk[k++], B);
    run_block(u, u->blk[k++], B);
    for (int d = S - 1; d >= 0; --d) {
        const Blk &src = u->blk[k - 1];                 // the stage below: its second block's output
        const int cd = c.channels[d], cb = u->below(d);
        k_up_concat<<<grid_for(u->cells(d, B) * cb / 8), TPB, 0, u->s>>>(src.y, u->X(d + 1), u->Y(d + 1), u->Z(d + 1), B,
                                                                         cb, u->cat[d], cd + cb, cd);
        run_block(u, u->blk[k++], B);
        run_block(u, u->blk[k++], B);
    }
    const Blk &last = u->blk[k - 1];
    k_out_fwd<<<grid_for(u->cells(0, B)), TPB, 0, u->s>>>(last.y, c.channels[0], u->params + u->oOw, u->params + u->oOb,
                                                          c.cout, u->N, B, u->y);
    UCK(cudaGetLastError());
    return LBM_OK;
}

// gradients of one block from the gradient gy (row stride ldgy) of its output
void back_block(unet_ctx *u, Blk &b, const bf16 *gy, int ldgy, int B)
{
    const int64_t n = u->cells(b.level, B);
    const int P = bn_blocks(n, b.cout);
    k_bn_reduce<1><<<P, TPB, 0, u->s>>>(b.z, gy, ldgy, n, b.cout, b.coef, u->part);
    k_bn_bwd_final<<<(b.cout + 127) / 128, 128, 0, u->s>>>(u->part, P, b.cout, (double)n, b.coef, u->params + b.og,
                                                            u->grads + b.og, u->grads + b.ob, b.k3);
    k_bn_bwd_apply<<<grid_for(n * b.cout / 8), TPB, 0, u->s>>>(b.z, gy, ldgy, n, b.cout, b.coef, b.k3, b.gz);
    cudaMemsetAsync(u->gwt, 0, sizeof(float) * 27 * (size_t)b.ip * b.cout, u->s);
    unet::wgrad_launch(b.wg, u->gwt, u->ustatus, u->s);
    k_wg_convert<<<grid_for((int64_t)27 * b.cout * b.cin), TPB, 0, u->s>>>(u->gwt, b.cin, b.ip, b.cout,
                                                                           u->grads + b.ow);
    if (b.gx) unet::conv_launch(b.bwd, b.gx, false, u->ustatus, u->s);
}

lbm_status backward_impl(unet_ctx *u, int B)
{
    const unet_config &c = u->c;
    const int S = u->S, c0 = c.channels[0];
    const int64_t n0 = u->cells(0, B);
    const int nb = (int)u->blk.size();
    const Blk &last = u->blk[nb - 1];
    k_out_bwd<<<grid_for(n0), TPB, 0, u->s>>>(u->y, u->tin, u->min, u->params + u->oOw, u->res, u->N, B, c.cout, c0,
                                              u->ga, u->gh0);
    const int P = std::min<int>(gb300::sm_count() * 4, (int)std::max<int64_t>(1, n0 / 256));
    const int nq = c.cout * c0 + c.cout;
    k_out_wgrad<<<P, TPB, 0, u->s>>>(u->ga, last.y, n0, c.cout, c0, u->opart);
    k_sum_parts<<<(nq + 127) / 128, 128, 0, u->s>>>(u->opart, P, nq, u->grads + u->oOw);
    // decoder, the last stage first
    int k = nb - 1;
    const bf16 *gy = u->gh0;
    int ldgy = c0;
    for (int d = 0; d < S; ++d) {
        Blk &bb = u->blk[k--];
        back_block(u, bb, gy, ldgy, B);
        Blk &ba = u->blk[k--];
        back_block(u, ba, bb.gx, bb.ip, B);
        const int cd = c.channels[d], cb = u->below(d);
        k_up_bwd<<<grid_for(u->cells(d + 1, B) * cb / 8), TPB, 0, u->s>>>(ba.gx, cd + cb, cd, u->X(d + 1), u->Y(d + 1),
                                                                          u->Z(d + 1), B, cb, u->gup[d]);
        gy = u->gup[d];
        ldgy = cb;
    }
    // bottleneck
    Blk &mb = u->blk[k--];
    back_block(u, mb, gy, ldgy, B);
    Blk &ma = u->blk[k--];
    back_block(u, ma, mb.gx, mb.ip, B);
    const bf16 *gp = ma.gx;
    // encoder, the deepest stage first
    for (int e = S - 1; e >= 0; --e) {
        const int ce = c.channels[e], cb = u->below(e);
        const Blk &dec_a = u->blk[nb - 2 - 2 * e];     // dec{e}a: its input gradient holds the skip's
        k_pool_bwd<<<grid_for(u->cells(e + 1, B) * ce / 8), TPB, 0, u->s>>>(gp, u->cat[e], ce + cb, dec_a.gx, ce + cb,
                                                                            u->X(e), u->Y(e), u->Z(e), B, ce, u->gyb[e]);
        Blk &eb = u->blk[k--];
        back_block(u, eb, u->gyb[e], ce, B);
        Blk &ea = u->blk[k--];
        back_block(u, ea, eb.gx, eb.ip, B);
        gp = ea.gx;
    }
    UCK(cudaGetLastError());
    return LBM_OK;
}

lbm_status stage_input(unet_ctx *u, const float *src, float *dst, int64_t count)
{
    UCK(cudaMemcpyAsync(dst, src, count * sizeof(float), on_device(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        u->s));
    return LBM_OK;
}

}  // namespace

extern "C" void unet_config_default(unet_config *c)
{
    std::memset(c, 0, sizeof(*c));
    c->nx = 128; c->ny = 64; c->nz = 64;
    c->cin = 4; c->cout = 4;
    c->stages = 4;
    c->channels[0] = 32; c->channels[1] = 64; c->channels[2] = 128; c->channels[3] = 256;
    c->bottleneck = 512;
    c->max_batch = 8;
    c->seed = 1234;
}

extern "C" lbm_status unet_destroy(unet_ctx *u)
{
    if (!u) return LBM_ERR_ARG;
    if (u->s) cudaStreamSynchronize(u->s);
    for (void *p : u->allocs) cudaFree(p);
    delete u;
    return LBM_OK;
}

extern "C" lbm_status unet_create(const unet_config *cfg, void *stream, unet_ctx **out)
{
    if (!cfg || !out) return LBM_ERR_ARG;
    *out = nullptr;
    const unet_config c = *cfg;
    const int S = c.stages;
    auto bad = [](const char *m) {
        g_unet_err = m;
        return LBM_ERR_ARG;
    };
    if (S < 1 || S > 4) return bad("stages must be in [1, 4]");
    if (!pow2(c.nx) || !pow2(c.ny) || !pow2(c.nz) || (c.nx >> S) < 1 || (c.ny >> S) < 1 || (c.nz >> S) < 1)
        return bad("grid sides must be powers of two divisible by 2^stages");
    if (c.cin < 1 || c.cin > CPAD || c.cout < 1 || c.cout > MAXOUT) return bad("cin must be in [1, 32], cout in [1, 8]");
    for (int e = 0; e < S; ++e)
        if (c.channels[e] < 32 || c.channels[e] % 32) return bad("stage channels must be positive multiples of 32");
    if (c.bottleneck < 32 || c.bottleneck % 32 || c.bottleneck > 512) return bad("bottleneck must be a multiple of 32, <= 512");
    for (int e = 0; e < S; ++e)
        if (c.channels[e] > 512) return bad("stage channels must be <= 512");
    if (c.max_batch < 1) return bad("max_batch must be >= 1");
    if (!unet::gemm_set_attrs()) return bad("cannot configure the tensor-core kernels");

    unet_ctx *u = new unet_ctx;
    u->c = c;
    u->s = static_cast<cudaStream_t>(stream);
    u->S = S;
    u->N = (int64_t)c.nx * c.ny * c.nz;
    const int MB = c.max_batch;
    // blocks in forward order with their parameter offsets
    int64_t off = 0;
    auto add = [&](int cin, int cout, int level) {
        Blk b;
        b.cin = cin;
        b.cout = cout;
        b.ip = ((cin + 31) / 32) * 32;
        b.level = level;
        b.ow = off;
        off += (int64_t)cout * cin * 27;
        b.og = off;
        off += cout;
        b.ob = off;
        off += cout;
        u->blk.push_back(b);
    };
    int cprev = c.cin;
    for (int e = 0; e < S; ++e) {
        add(cprev, c.channels[e], e);
        add(c.channels[e], c.channels[e], e);
        cprev = c.channels[e];
    }
    add(cprev, c.bottleneck, S);
    add(c.bottleneck, c.bottleneck, S);
    for (int d = S - 1; d >= 0; --d) {
        add(c.channels[d] + u->below(d), c.channels[d], d);
        add(c.channels[d], c.channels[d], d);
    }
    u->oOw = off;
    off += (int64_t)c.cout * c.channels[0];
    u->oOb = off;
    off += c.cout;
    u->np = off;

    bool ok = (u->params = u->alloc<float>(u->np)) && (u->grads = u->alloc<float>(u->np)) &&
              (u->m1 = u->alloc<float>(u->np)) && (u->m2 = u->alloc<float>(u->np)) &&
              (u->ustatus = u->alloc<int>(1)) && (u->res = u->alloc<double>(2));
    const int64_t n0 = u->cells(0, MB);
    ok = ok && (u->x0 = u->alloc<bf16>(n0 * CPAD)) && (u->xin = u->alloc<float>(n0 * c.cin)) &&
         (u->tin = u->alloc<float>(n0 * c.cout)) && (u->min = u->alloc<float>(n0)) &&
         (u->y = u->alloc<float>(n0 * c.cout)) && (u->ga = u->alloc<float>(n0 * c.cout)) &&
         (u->gh0 = u->alloc<bf16>(n0 * c.channels[0]));
    u->cat.assign(S, nullptr);
    u->pool.assign(S, nullptr);
    u->gup.assign(S, nullptr);
    u->gyb.assign(S, nullptr);
    for (int e = 0; ok && e < S; ++e) {
        const int ce = c.channels[e], cb = u->below(e);
        ok = (u->cat[e] = u->alloc<bf16>(u->cells(e, MB) * (ce + cb))) &&
             (u->pool[e] = u->alloc<bf16>(u->cells(e + 1, MB) * ce)) &&
             (u->gup[e] = u->alloc<bf16>(u->cells(e + 1, MB) * cb)) && (u->gyb[e] = u->alloc<bf16>(u->cells(e, MB) * ce));
    }
    size_t gwt_max = 0;
    int cmax = 0;
    for (size_t i = 0; ok && i < u->blk.size(); ++i) {
        Blk &b = u->blk[i];
        const int64_t n = u->cells(b.level, MB);
        gwt_max = std::max(gwt_max, (size_t)27 * b.ip * b.cout);
        cmax = std::max(cmax, b.cout);
        ok = (b.wf = u->alloc<bf16>((size_t)27 * b.cout * b.ip)) && (b.z = u->alloc<bf16>(n * b.cout)) &&
             (b.coef = u->alloc<float>(4 * b.cout)) && (b.k3 = u->alloc<float>(3 * b.cout)) &&
             (b.gz = u->alloc<bf16>(n * b.cout));
        if (ok && i > 0) ok = (b.wb = u->alloc<bf16>((size_t)27 * b.cout * b.ip)) && (b.gx = u->alloc<bf16>(n * b.ip));
    }
    u->part_max = gb300::sm_count() * 4;
    const int nq = c.cout * c.channels[0] + c.cout;
    ok = ok && (u->gwt = u->alloc<float>(gwt_max)) && (u->part = u->alloc<float2>((size_t)u->part_max * cmax)) &&
         (u->lpart = u->alloc<double2>(u->part_max)) && (u->opart = u->alloc<float>((size_t)u->part_max * nq));
    if (!ok) {
        g_unet_err = "device allocation failed";
        unet_destroy(u);
        return LBM_ERR_OOM;
    }
    // wiring: inputs and outputs of every block
    {
        int k = 0;
        for (int e = 0; e < S; ++e) {
            const int ce = c.channels[e], cb = u->below(e);
            Blk &a = u->blk[k++];
            a.x = e == 0 ? u->x0 : u->pool[e - 1];
            a.y = u->alloc<bf16>(u->cells(e, MB) * ce);
            a.ldy = ce;
            Blk &b = u->blk[k++];
            b.x = a.y;
            b.y = u->cat[e];                          // the skip slot of the decoder's concatenation
            b.ldy = ce + cb;
            ok = ok && a.y;
        }
        Blk &ma = u->blk[k++];
        ma.x = u->pool[S - 1];
        ma.y = u->alloc<bf16>(u->cells(S, MB) * c.bottleneck);
        ma.ldy = c.bottleneck;
        Blk &mb = u->blk[k++];
        mb.x = ma.y;
        mb.y = u->alloc<bf16>(u->cells(S, MB) * c.bottleneck);
        mb.ldy = c.bottleneck;
        ok = ok && ma.y && mb.y;
        for (int d = S - 1; d >= 0; --d) {
            const int cd = c.channels[d];
            Blk &a = u->blk[k++];
            a.x = u->cat[d];
            a.y = u->alloc<bf16>(u->cells(d, MB) * cd);
            a.ldy = cd;
            Blk &b = u->blk[k++];
            b.x = a.y;
            b.y = u->alloc<bf16>(u->cells(d, MB) * cd);
            b.ldy = cd;
            ok = ok && a.y && b.y;
        }
    }
    if (!ok) {
        g_unet_err = "device allocation failed";
        unet_destroy(u);
        return LBM_ERR_OOM;
    }
    // initial parameters
    std::vector<float> h(u->np, 0.f);
    uint64_t st = c.seed;
    for (const Blk &b : u->blk) {
        const double sd = std::sqrt(2.0 / (27.0 * b.cin));
        for (int64_t i = 0; i < (int64_t)b.cout * b.cin * 27; ++i) h[b.ow + i] = (float)(sd * normal(st));
        for (int o = 0; o < b.cout; ++o) h[b.og + o] = 1.f;
    }
    const double lim = 1.0 / std::sqrt((double)c.channels[0]);
    for (int64_t i = 0; i < (int64_t)c.cout * c.channels[0]; ++i) h[u->oOw + i] = (float)(lim * (2.0 * unif01(st) - 1.0));
    if (cudaMemcpy(u->params, h.data(), u->np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(u->grads, 0, u->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(u->m1, 0, u->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(u->m2, 0, u->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(u->ustatus, 0, sizeof(int)) != cudaSuccess) {
        g_unet_err = "device initialisation failed";
        unet_destroy(u);
        return LBM_ERR_CUDA;
    }
    if (pack_weights(u) != LBM_OK || cudaStreamSynchronize(u->s) != cudaSuccess) {
        g_unet_err = u->err.empty() ? "weight packing failed" : u->err;
        unet_destroy(u);
        return LBM_ERR_CUDA;
    }
    *out = u;
    return LBM_OK;
}

extern "C" int64_t unet_num_params(const unet_ctx *u) { return u ? u->np : -1; }

extern "C" lbm_status unet_set_params(unet_ctx *u, const float *src)
{
    if (!u || !src) return LBM_ERR_ARG;
    UCK(cudaMemcpyAsync(u->params, src, u->np * sizeof(float), cudaMemcpyDefault, u->s));
    lbm_status st = pack_weights(u);
    if (st != LBM_OK) return st;
    UCK(cudaStreamSynchronize(u->s));
    return LBM_OK;
}

extern "C" lbm_status unet_get_params(unet_ctx *u, float *dst)
{
    if (!u || !dst) return LBM_ERR_ARG;
    UCK(cudaMemcpyAsync(dst, u->params, u->np * sizeof(float), cudaMemcpyDefault, u->s));
    UCK(cudaStreamSynchronize(u->s));
    return LBM_OK;
}

extern "C" lbm_status unet_get_grads(unet_ctx *u, float *dst)
{
    if (!u || !dst) return LBM_ERR_ARG;
    UCK(cudaMemcpyAsync(dst, u->grads, u->np * sizeof(float), cudaMemcpyDefault, u->s));
    UCK(cudaStreamSynchronize(u->s));
    return LBM_OK;
}

extern "C" lbm_status unet_forward(unet_ctx *u, const float *x, float *y, int32_t batch)
{
    if (!u || !x || !y || batch < 1 || batch > u->c.max_batch) {
        if (u) u->err = "batch must be in [1, max_batch]";
        return LBM_ERR_ARG;
    }
    const int B = batch;
    lbm_status st = stage_input(u, x, u->xin, (int64_t)B * u->c.cin * u->N);
    if (st == LBM_OK) st = forward_impl(u, B);
    if (st != LBM_OK) return st;
    UCK(cudaMemcpyAsync(y, u->y, (int64_t)B * u->c.cout * u->N * sizeof(float), cudaMemcpyDefault, u->s));
    if (!on_device(y)) UCK(cudaStreamSynchronize(u->s));
    return LBM_OK;
}

extern "C" lbm_status unet_loss_grad(unet_ctx *u, const float *x, const float *t, const float *m, int32_t batch,
                                     double *loss)
{
    if (!u || !x || !t || !m || batch < 1 || batch > u->c.max_batch) {
        if (u) u->err = "batch must be in [1, max_batch]";
        return LBM_ERR_ARG;
    }
    const unet_config &c = u->c;
    const int B = batch;
    lbm_status st = stage_input(u, x, u->xin, (int64_t)B * c.cin * u->N);
    if (st == LBM_OK) st = stage_input(u, t, u->tin, (int64_t)B * c.cout * u->N);
    if (st == LBM_OK) st = stage_input(u, m, u->min, (int64_t)B * u->N);
    if (st == LBM_OK) st = forward_impl(u, B);
    if (st != LBM_OK) return st;
    const int P = std::min<int>(u->part_max, grid_for(u->cells(0, B)));
    k_loss_partial<<<P, TPB, 0, u->s>>>(u->y, u->tin, u->min, u->N, B, c.cout, u->lpart);
    k_loss_final<<<1, 32, 0, u->s>>>(u->lpart, P, c.cout, u->res);
    st = backward_impl(u, B);
    if (st != LBM_OK) return st;
    if (loss) {
        double r[2];
        UCK(cudaMemcpyAsync(r, u->res, sizeof r, cudaMemcpyDeviceToHost, u->s));
        UCK(cudaStreamSynchronize(u->s));
        *loss = r[0];
    }
    return LBM_OK;
}

extern "C" lbm_status unet_adam_step(unet_ctx *u, float lr, float b1, float b2, float eps)
{
    if (!u) return LBM_ERR_ARG;
    u->adam_t++;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)u->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)u->adam_t)));
    k_adam<<<grid_for(u->np), TPB, 0, u->s>>>(u->params, u->grads, u->m1, u->m2, u->np, lr, b1, b2, eps, c1, c2);
    UCK(cudaGetLastError());
    return pack_weights(u);
}

extern "C" lbm_status unet_train_step(unet_ctx *u, const float *x, const float *t, const float *m, int32_t batch,
                                      float lr, double *loss)
{
    lbm_status st = unet_loss_grad(u, x, t, m, batch, loss);
    if (st != LBM_OK) return st;
    return unet_adam_step(u, lr, 0.9f, 0.999f, 1e-8f);
}

extern "C" lbm_status unet_sync(unet_ctx *u)
{
    if (!u) return LBM_ERR_ARG;
    UCK(cudaStreamSynchronize(u->s));
    int st = 0;
    UCK(cudaMemcpy(&st, u->ustatus, sizeof st, cudaMemcpyDeviceToHost));
    if (st != 0) {
        UCK(cudaMemset(u->ustatus, 0, sizeof(int)));
        u->err = "a bounded wait of a tensor-core kernel gave up (code " + std::to_string(st) + ")";
        return LBM_ERR_TIMEOUT;
    }
    return LBM_OK;
}

extern "C" const char *unet_last_error(const unet_ctx *u) { return u ? u->err.c_str() : g_unet_err.c_str(); }

// ---------------------------------------------------------------------------
// the convolution alone
// ---------------------------------------------------------------------------
namespace {

struct OpScratch {
    std::vector<void *> p;
    ~OpScratch()
    {
        for (void *q : p) cudaFree(q);
    }
    template <class T> T *get(size_t n)
    {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(n * sizeof(T), 16)) != cudaSuccess) return nullptr;
        p.push_back(q);
        return static_cast<T *>(q);
    }
};

lbm_status op_check(const void *a, const void *b, const void *c, int32_t B, int32_t nx, int32_t ny, int32_t nz,
                    int32_t cin, int32_t cout)
{
    if (!a || !b || !c || B < 1 || !pow2(nx) || !pow2(ny) || !pow2(nz) || cin < 32 || cin % 32 || cout < 32 ||
        cout % 32 || cin > 1024 || cout > 1024) {
        g_unet_err = "convolution: device buffers, power-of-two grid, channels multiples of 32 required";
        return LBM_ERR_ARG;
    }
    if (!on_device(a) || !on_device(b) || !on_device(c)) {
        g_unet_err = "convolution: buffers must be device memory";
        return LBM_ERR_ARG;
    }
    if (!unet::gemm_set_attrs()) {
        g_unet_err = "cannot configure the tensor-core kernels";
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

lbm_status op_finish(cudaStream_t s, int *status)
{
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        g_unet_err = std::string("convolution: ") + cudaGetErrorString(e);
        return LBM_ERR_CUDA;
    }
    int st = 0;
    if (cudaMemcpy(&st, status, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ERR_CUDA;
    if (st) {
        g_unet_err = "a bounded wait of a tensor-core kernel gave up (code " + std::to_string(st) + ")";
        return LBM_ERR_TIMEOUT;
    }
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status unet_conv3_forward(const float *x, const float *w, float *y, int32_t B, int32_t nx, int32_t ny,
                                         int32_t nz, int32_t cin, int32_t cout, void *stream)
{
    lbm_status st = op_check(x, w, y, B, nx, ny, nz, cin, cout);
    if (st != LBM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)B * nx * ny * nz;
    OpScratch sc;
    bf16 *xb = sc.get<bf16>(n * cin), *wf = sc.get<bf16>((size_t)27 * cin * cout);
    int *status = sc.get<int>(1);
    if (!xb || !wf || !status) return LBM_ERR_OOM;
    cudaMemsetAsync(status, 0, sizeof(int), s);
    k_f2bf<<<grid_for(n * cin), TPB, 0, s>>>(x, xb, n * cin);
    k_pack_w<<<grid_for((int64_t)27 * cout * cin), TPB, 0, s>>>(w, cout, cin, cin, wf, nullptr);
    unet::ConvPlan p;
    const char *e = nullptr;
    if (!unet::conv_plan(p, xb, cin, cin, nx, ny, nz, B, wf, cout, 27, cout, 0, gb300::sm_count(), &e)) {
        cudaStreamSynchronize(s);
        g_unet_err = e ? e : "plan failed";
        return LBM_ERR_ARG;
    }
    unet::conv_launch(p, y, true, status, s);
    return op_finish(s, status);
}

extern "C" lbm_status unet_conv3_backward_data(const float *gy, const float *w, float *gx, int32_t B, int32_t nx,
                                               int32_t ny, int32_t nz, int32_t cin, int32_t cout, void *stream)
{
    lbm_status st = op_check(gy, w, gx, B, nx, ny, nz, cin, cout);
    if (st != LBM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)B * nx * ny * nz;
    OpScratch sc;
    bf16 *gb = sc.get<bf16>(n * cout), *wf = sc.get<bf16>((size_t)27 * cin * cout),
         *wb = sc.get<bf16>((size_t)27 * cin * cout);
    int *status = sc.get<int>(1);
    if (!gb || !wf || !wb || !status) return LBM_ERR_OOM;
    cudaMemsetAsync(status, 0, sizeof(int), s);
    k_f2bf<<<grid_for(n * cout), TPB, 0, s>>>(gy, gb, n * cout);
    k_pack_w<<<grid_for((int64_t)27 * cout * cin), TPB, 0, s>>>(w, cout, cin, cin, wf, wb);
    unet::ConvPlan p;
    const char *e = nullptr;
    if (!unet::conv_plan(p, gb, cout, cout, nx, ny, nz, B, wb, cin, 27, cin, 0, gb300::sm_count(), &e)) {
        cudaStreamSynchronize(s);
        g_unet_err = e ? e : "plan failed";
        return LBM_ERR_ARG;
    }
    unet::conv_launch(p, gx, true, status, s);
    return op_finish(s, status);
}

extern "C" lbm_status unet_conv3_backward_weights(const float *x, const float *gy, float *gw, int32_t B, int32_t nx,
                                                  int32_t ny, int32_t nz, int32_t cin, int32_t cout, void *stream)
{
    lbm_status st = op_check(x, gy, gw, B, nx, ny, nz, cin, cout);
    if (st != LBM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)B * nx * ny * nz;
    OpScratch sc;
    bf16 *xb = sc.get<bf16>(n * cin), *gb = sc.get<bf16>(n * cout);
    float *gwt = sc.get<float>((size_t)27 * cin * cout);
    int *status = sc.get<int>(1);
    if (!xb || !gb || !gwt || !status) return LBM_ERR_OOM;
    cudaMemsetAsync(status, 0, sizeof(int), s);
    cudaMemsetAsync(gwt, 0, sizeof(float) * 27 * (size_t)cin * cout, s);
    k_f2bf<<<grid_for(n * cin), TPB, 0, s>>>(x, xb, n * cin);
    k_f2bf<<<grid_for(n * cout), TPB, 0, s>>>(gy, gb, n * cout);
    unet::WgradPlan p;
    const char *e = nullptr;
    if (!unet::wgrad_plan(p, xb, cin, cin, gb, cout, cout, nx, ny, nz, B, gb300::sm_count(), &e)) {
        cudaStreamSynchronize(s);
        g_unet_err = e ? e : "plan failed";
        return LBM_ERR_ARG;
    }
    unet::wgrad_launch(p, gwt, status, s);
    k_wg_convert<<<grid_for((int64_t)27 * cout * cin), TPB, 0, s>>>(gwt, cin, cin, cout, gw);
    return op_finish(s, status);
}
