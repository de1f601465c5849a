// fno.cu -- kernels and host orchestration of the Fourier Neural Operator
// surrogate declared in include/fno.h (paper Sec. 4 and the appendix on the
// baseline models: FNO of Li et al. 2021 mapping mask and Re to the mean
// field).
//
// Network (App. B): feed-forward lift P2 GELU(P1 x), Fourier layers, SIREN
// projection Q2 sin(omega0 (Q1 v + b)) (Sitzmann et al. 2020).
//
// Kernels:
//   k_pw_fwd_*   pointwise layers (lift, W path, projection) with fused bias,
//                spectral-branch add and activation (GELU, or the SIREN sine,
//                whose kept value is cos(omega0 z) for the backward)
//   k_proj_fused inference projection Q2 sin(omega0 (Q1 v + b1)) without
//                storing the hidden activations
//   k_pw_bwd_*   input gradients of pointwise layers with the fused
//                activation derivative
//   k_outer      weight/bias gradients sum_{b,cell} gout x (k_outer_async:
//                cp.async double-buffered tiles)
//   k_dft*       truncated DFT in three separable stages (x, y, z) and the
//                inverse (z, y, x), FP32 with twiddle tables in shared memory;
//                the real x stages fold samples x and nx - x
//   k_contract_tc  per-mode complex channel mixing on tensor cores
//                (mma.sync m16n8k16 BF16 operands, FP32 accumulation); complex
//                numbers enter as real 2x2 blocks, the batch is the n8 axis
//   k_contract_f32 the same contraction in FP32 (reference and small widths)
//   k_grad_R     spectral weight gradients sum_b gG conj(V)
//   k_mse_*      masked mean square error and its gradient (deterministic)
//   k_adam       Adam update of the flat parameter vector
#include <cmath>
#include <type_traits>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/fno.h"
#include "sm_count.h"
#include "fno_umma.h"

namespace {

constexpr int TPB = 256;

// ---------------------------------------------------------------------------
// activation storage
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ldf(const float *p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float *p, float v) { *p = v; }
__device__ __forceinline__ void stf(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// Activations of the pointwise layers.  The forward keeps, per element, what
// the backward needs: the pre-activation z for GELU, cos(omega0 z) for the
// SIREN sine (so that the backward needs no transcendental and does not
// amplify the storage rounding of z by omega0).  FP32 activations take the
// accurate sincosf, BF16 activations the hardware __sincosf, whose phase
// error (about |omega0 z| x 2^-23) is far below BF16's rounding.
enum { ACT_NONE = 0, ACT_GELU = 1, ACT_SIREN = 2 };

template <bool FAST>
__device__ __forceinline__ float act_fwd(int act, float w0, float z, float &keep)
{
    if (act == ACT_SIREN) {
        float sn, cs;
        if (FAST) __sincosf(w0 * z, &sn, &cs);
        else sincosf(w0 * z, &sn, &cs);
        keep = cs;
        return sn;
    }
    keep = z;
    return act == ACT_GELU ? gelu(z) : z;
}

__device__ __forceinline__ float act_grad(int act, float w0, float kept)
{
    return act == ACT_SIREN ? w0 * kept : gelu_grad(kept);
}

template <class T> struct IsBF16 { static constexpr bool value = false; };
template <> struct IsBF16<__nv_bfloat16> { static constexpr bool value = true; };

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a conj(b)

int grid_for(int64_t n, int block = TPB) { return (int)std::min<int64_t>((n + block - 1) / block, gb300::sm_count() * 16); }

// ---------------------------------------------------------------------------
// pointwise layers
// ---------------------------------------------------------------------------
// y = act(W x + b + extra) for ci <= 32 (inputs cached in registers).
template <class TI, class TO>
__global__ void __launch_bounds__(TPB) k_pw_fwd_in(const TI *x, int ci, int co, const float *W, const float *bias,
                                                   const float *extra, TO *pre, TO *y, int act, float w0, int64_t N,
                                                   int B)
{
    extern __shared__ float sm[];
    float *sw = sm, *sb = sm + co * ci;
    for (int k = threadIdx.x; k < co * ci; k += blockDim.x) sw[k] = W[k];
    for (int k = threadIdx.x; k < co; k += blockDim.x) sb[k] = bias[k];
    __syncthreads();
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / N, n = idx - b * N;
        float xv[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) xv[i] = i < ci ? ldf(x + (b * ci + i) * N + n) : 0.f;
        for (int o = 0; o < co; ++o) {
            float acc = sb[o];
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (i < ci) acc += sw[o * ci + i] * xv[i];
            const int64_t off = (b * co + o) * N + n;
            if (extra) acc += extra[off];
            float keep;
            const float out = act_fwd<IsBF16<TO>::value>(act, w0, acc, keep);
            if (pre) stf(pre + off, keep);
            stf(y + off, out);
        }
    }
}

// y = W x + b for co <= 8 (outputs accumulated in registers, inputs streamed).
template <class TI>
__global__ void __launch_bounds__(TPB) k_pw_fwd_out(const TI *x, int ci, int co, const float *W, const float *bias,
                                                    float *y, int64_t N, int B)
{
    extern __shared__ float sm[];
    float *sw = sm, *sb = sm + co * ci;
    for (int k = threadIdx.x; k < co * ci; k += blockDim.x) sw[k] = W[k];
    for (int k = threadIdx.x; k < co; k += blockDim.x) sb[k] = bias[k];
    __syncthreads();
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / N, n = idx - b * N;
        float acc[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o] = o < co ? sb[o] : 0.f;
        for (int i = 0; i < ci; ++i) {
            const float xv = ldf(x + (b * ci + i) * N + n);
#pragma unroll
            for (int o = 0; o < 8; ++o)
                if (o < co) acc[o] += sw[o * ci + i] * xv;
        }
#pragma unroll
        for (int o = 0; o < 8; ++o)
            if (o < co) y[(b * co + o) * N + n] = acc[o];
    }
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p)
{
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Copies `total` floats (a multiple of 4) into shared memory from a
// contiguous source of which the first `cnt` are valid (zeros after), with
// eight 4-element loads in flight per thread.
template <class TI>
__device__ __forceinline__ void stage4(float *dst, const TI *src, int cnt, int total)
{
    const int step = 4 * blockDim.x;
    for (int k0 = 4 * threadIdx.x; k0 < total; k0 += 8 * step) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u * step;
            v[u] = k < cnt ? ld4(src + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u * step;
            if (k < total) *reinterpret_cast<float4 *>(dst + k) = v[u];
        }
    }
}

// Two adjacent cells per thread (N even): loads and stores of pairs, each
// weight read from shared memory serves both cells.
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ float2 ld2(const __nv_bfloat16 *p)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
}
__device__ __forceinline__ void st2(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }
__device__ __forceinline__ void st2(__nv_bfloat16 *p, float a, float b)
{
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}

// y = act(W x + b + extra) for CI inputs (a multiple of 4) held in registers.
template <class TI, class TO, int CI>
__global__ void __launch_bounds__(TPB) k_pw_fwd_in2(const TI *x, int co, const float *W, const float *bias,
                                                    const float *extra, TO *pre, TO *y, int act, float w0, int64_t N,
                                                    int B)
{
    extern __shared__ float4 smv[];
    float *sw = reinterpret_cast<float *>(smv), *sb = sw + co * CI;
    for (int k = threadIdx.x; k < co * CI; k += blockDim.x) sw[k] = W[k];
    for (int k = threadIdx.x; k < co; k += blockDim.x) sb[k] = bias[k];
    __syncthreads();
    const int64_t half = N / 2;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * half;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / half, n = 2 * (idx - b * half);
        float2 xv[CI];
#pragma unroll
        for (int i = 0; i < CI; ++i) xv[i] = ld2(x + (b * CI + i) * N + n);
        for (int o0 = 0; o0 < co; o0 += 8) {                 // co % 8 == 0
            float2 e[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) e[u] = extra ? ld2(extra + (b * co + o0 + u) * N + n) : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int o = o0 + u;
                float a0 = sb[o] + e[u].x, a1 = sb[o] + e[u].y;
                const float4 *w4 = reinterpret_cast<const float4 *>(sw + o * CI);
#pragma unroll
                for (int q = 0; q < CI / 4; ++q) {
                    const float4 w = w4[q];
                    a0 += w.x * xv[4 * q].x + w.y * xv[4 * q + 1].x + w.z * xv[4 * q + 2].x + w.w * xv[4 * q + 3].x;
                    a1 += w.x * xv[4 * q].y + w.y * xv[4 * q + 1].y + w.z * xv[4 * q + 2].y + w.w * xv[4 * q + 3].y;
                }
                const int64_t off = (b * co + o) * N + n;
                float k0, k1;
                const float y0 = act_fwd<IsBF16<TO>::value>(act, w0, a0, k0);
                const float y1 = act_fwd<IsBF16<TO>::value>(act, w0, a1, k1);
                if (pre) st2(pre + off, k0, k1);
                st2(y + off, y0, y1);
            }
        }
    }
}

// Inference lift in one pass: v0 = P2 GELU(P1 x + b1) + b2 from the FP32
// input [B][4][N] to the BF16 layer input [B][32][N], two adjacent cells per
// thread, the 32 hidden units in registers.  The input and the hidden units
// are rounded to BF16 where the training path stores them, so that both
// paths evaluate the same network.  Shared memory: P1 [32][4], b1, P2
// [32][32], b2.
constexpr int LIFT_CI = 4, LIFT_H = 32, LIFT_CO = 32;
__global__ void __launch_bounds__(TPB, 2) k_lift_fused(const float *x, const float *P1, const float *b1, const float *P2,
                                                    const float *b2, __nv_bfloat16 *y, int64_t N, int B)
{
    __shared__ float4 s1[LIFT_H];                 // P1 rows
    __shared__ float4 s2[LIFT_CO * LIFT_H / 4];   // P2 rows
    __shared__ float sb1[LIFT_H], sb2[LIFT_CO];
    for (int k = threadIdx.x; k < LIFT_H; k += blockDim.x) {
        s1[k] = make_float4(P1[4 * k], P1[4 * k + 1], P1[4 * k + 2], P1[4 * k + 3]);
        sb1[k] = b1[k];
    }
    for (int k = threadIdx.x; k < LIFT_CO * LIFT_H; k += blockDim.x) reinterpret_cast<float *>(s2)[k] = P2[k];
    for (int k = threadIdx.x; k < LIFT_CO; k += blockDim.x) sb2[k] = b2[k];
    __syncthreads();
    const int64_t half = N / 2;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * half;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / half, n = 2 * (idx - b * half);
        float2 xv[LIFT_CI];
#pragma unroll
        for (int i = 0; i < LIFT_CI; ++i) {
            const float2 v = ld2(x + (b * LIFT_CI + i) * N + n);
            xv[i] = make_float2(__bfloat162float(__float2bfloat16_rn(v.x)), __bfloat162float(__float2bfloat16_rn(v.y)));
        }
        float2 h[LIFT_H];
#pragma unroll
        for (int o = 0; o < LIFT_H; ++o) {
            const float4 w = s1[o];
            float a0 = sb1[o] + 0.f, a1 = sb1[o] + 0.f;
            a0 += w.x * xv[0].x + w.y * xv[1].x + w.z * xv[2].x + w.w * xv[3].x;
            a1 += w.x * xv[0].y + w.y * xv[1].y + w.z * xv[2].y + w.w * xv[3].y;
            h[o] = make_float2(__bfloat162float(__float2bfloat16_rn(gelu(a0))),
                               __bfloat162float(__float2bfloat16_rn(gelu(a1))));
        }
#pragma unroll 1
        for (int o = 0; o < LIFT_CO; ++o) {
            float a0 = sb2[o] + 0.f, a1 = sb2[o] + 0.f;
            const float4 *w4 = s2 + o * (LIFT_H / 4);
#pragma unroll
            for (int q = 0; q < LIFT_H / 4; ++q) {
                const float4 w = w4[q];
                a0 += w.x * h[4 * q].x + w.y * h[4 * q + 1].x + w.z * h[4 * q + 2].x + w.w * h[4 * q + 3].x;
                a1 += w.x * h[4 * q].y + w.y * h[4 * q + 1].y + w.z * h[4 * q + 2].y + w.w * h[4 * q + 3].y;
            }
            st2(y + (b * LIFT_CO + o) * N + n, a0, a1);
        }
    }
}

// Inference projection y = Q2 sin(omega0 (Q1 v + b1)) + b2 in one pass (the hidden
// activations are never stored): CI inputs and co <= 8 outputs in registers,
// the H hidden units streamed, two adjacent cells per thread.  Shared
// memory: Q1 [H][CI], b1 [H], Q2 transposed to [H][8] (zero padded).
template <class TI, int CI>
__global__ void __launch_bounds__(TPB) k_proj_fused(const TI *v, int H, int co, const float *W1, const float *b1,
                                                    const float *W2, const float *b2, float w0, float *y, int64_t N,
                                                    int B)
{
    extern __shared__ float4 smv[];
    float *s1 = reinterpret_cast<float *>(smv);
    float *sb1 = s1 + H * CI;
    float *s2 = sb1 + ((H + 3) & ~3);
    for (int k = threadIdx.x; k < H * CI; k += blockDim.x) s1[k] = W1[k];
    for (int k = threadIdx.x; k < H; k += blockDim.x) sb1[k] = b1[k];
    for (int k = threadIdx.x; k < H * 8; k += blockDim.x) {
        const int hh = k / 8, o = k % 8;
        s2[k] = o < co ? W2[o * H + hh] : 0.f;
    }
    __syncthreads();
    const int64_t half = N / 2;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * half;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / half, n = 2 * (idx - b * half);
        float2 xv[CI];
#pragma unroll
        for (int i = 0; i < CI; ++i) xv[i] = ld2(v + (b * CI + i) * N + n);
        float2 acc[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o] = o < co ? make_float2(b2[o], b2[o]) : make_float2(0.f, 0.f);
        for (int hh = 0; hh < H; ++hh) {
            float a0 = sb1[hh], a1 = a0;
            const float4 *w4 = reinterpret_cast<const float4 *>(s1 + hh * CI);
#pragma unroll
            for (int q = 0; q < CI / 4; ++q) {
                const float4 w = w4[q];
                a0 += w.x * xv[4 * q].x + w.y * xv[4 * q + 1].x + w.z * xv[4 * q + 2].x + w.w * xv[4 * q + 3].x;
                a1 += w.x * xv[4 * q].y + w.y * xv[4 * q + 1].y + w.z * xv[4 * q + 2].y + w.w * xv[4 * q + 3].y;
            }
            float k0, k1;
            const float g0 = act_fwd<IsBF16<TI>::value>(ACT_SIREN, w0, a0, k0);
            const float g1 = act_fwd<IsBF16<TI>::value>(ACT_SIREN, w0, a1, k1);
            const float4 wa = reinterpret_cast<const float4 *>(s2)[2 * hh];
            const float4 wb = reinterpret_cast<const float4 *>(s2)[2 * hh + 1];
            const float w2[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                acc[o].x += w2[o] * g0;
                acc[o].y += w2[o] * g1;
            }
        }
#pragma unroll
        for (int o = 0; o < 8; ++o)
            if (o < co) st2(y + (b * co + o) * N + n, acc[o].x, acc[o].y);
    }
}

// y = W x + b (FP32 out) for co <= 8 outputs and any number of inputs; the
// weights are transposed in shared memory to [ci][8].
template <class TI>
__global__ void __launch_bounds__(TPB) k_pw_fwd_out2(const TI *x, int ci, int co, const float *W, const float *bias,
                                                     float *y, int64_t N, int B)
{
    extern __shared__ float4 smv[];
    float *swt = reinterpret_cast<float *>(smv);
    for (int k = threadIdx.x; k < ci * 8; k += blockDim.x) {
        const int i = k / 8, o = k % 8;
        swt[k] = o < co ? W[o * ci + i] : 0.f;
    }
    __syncthreads();
    const int64_t half = N / 2;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * half;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / half, n = 2 * (idx - b * half);
        float2 acc[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o] = o < co ? make_float2(bias[o], bias[o]) : make_float2(0.f, 0.f);
        for (int i0 = 0; i0 < ci; i0 += 8) {                 // ci % 8 == 0
            float2 xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) xv[u] = ld2(x + (b * ci + i0 + u) * N + n);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 wa = reinterpret_cast<const float4 *>(swt)[2 * (i0 + u)];
                const float4 wb = reinterpret_cast<const float4 *>(swt)[2 * (i0 + u) + 1];
                const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    acc[o].x += w[o] * xv[u].x;
                    acc[o].y += w[o] * xv[u].y;
                }
            }
        }
#pragma unroll
        for (int o = 0; o < 8; ++o)
            if (o < co) st2(y + (b * co + o) * N + n, acc[o].x, acc[o].y);
    }
}

// gx = (W^T g) * (pre_in ? act'(pre_in) : 1) for CI inputs (a multiple of 4);
// pre_in holds what the forward kept (see act_fwd).
template <class TP, int CI>
__global__ void __launch_bounds__(TPB) k_pw_bwd_in2(const float *g, int co, const float *W, const TP *pre_in,
                                                    int act, float w0, float *gx, int64_t N, int B)
{
    extern __shared__ float4 smv[];
    float *sw = reinterpret_cast<float *>(smv);
    for (int k = threadIdx.x; k < co * CI; k += blockDim.x) sw[k] = W[k];
    __syncthreads();
    const int64_t half = N / 2;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * half;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / half, n = 2 * (idx - b * half);
        float2 acc[CI];
#pragma unroll
        for (int i = 0; i < CI; ++i) acc[i] = make_float2(0.f, 0.f);
        for (int o0 = 0; o0 < co; o0 += 8) {                 // co % 8 == 0
            float2 gq[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) gq[u] = ld2(g + (b * co + o0 + u) * N + n);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float2 gv = gq[u];
                const float4 *w4 = reinterpret_cast<const float4 *>(sw + (o0 + u) * CI);
#pragma unroll
                for (int q = 0; q < CI / 4; ++q) {
                    const float4 w = w4[q];
                    acc[4 * q].x += w.x * gv.x;     acc[4 * q].y += w.x * gv.y;
                    acc[4 * q + 1].x += w.y * gv.x; acc[4 * q + 1].y += w.y * gv.y;
                    acc[4 * q + 2].x += w.z * gv.x; acc[4 * q + 2].y += w.z * gv.y;
                    acc[4 * q + 3].x += w.w * gv.x; acc[4 * q + 3].y += w.w * gv.y;
                }
            }
        }
        if (pre_in) {
#pragma unroll
            for (int i = 0; i < CI; ++i) {
                const float2 p = ld2(pre_in + (b * CI + i) * N + n);
                acc[i].x *= act_grad(act, w0, p.x);
                acc[i].y *= act_grad(act, w0, p.y);
            }
        }
#pragma unroll
        for (int i = 0; i < CI; ++i) st2(gx + (b * CI + i) * N + n, acc[i].x, acc[i].y);
    }
}

// Same for co <= 8 gradient rows and any number of inputs ([ci][8] weights).
template <class TP>
__global__ void __launch_bounds__(TPB) k_pw_bwd_out2(const float *g, int co, int ci, const float *W, const TP *pre_in,
                                                     int act, float w0, float *gx, int64_t N, int B)
{
    extern __shared__ float4 smv[];
    float *swt = reinterpret_cast<float *>(smv);
    for (int k = threadIdx.x; k < ci * 8; k += blockDim.x) {
        const int i = k / 8, o = k % 8;
        swt[k] = o < co ? W[o * ci + i] : 0.f;
    }
    __syncthreads();
    const int64_t half = N / 2;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * half;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / half, n = 2 * (idx - b * half);
        float2 gv[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) gv[o] = o < co ? ld2(g + (b * co + o) * N + n) : make_float2(0.f, 0.f);
        for (int i0 = 0; i0 < ci; i0 += 8) {                 // ci % 8 == 0
            float2 p[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) p[u] = pre_in ? ld2(pre_in + (b * ci + i0 + u) * N + n) : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u;
                const float4 wa = reinterpret_cast<const float4 *>(swt)[2 * i];
                const float4 wb = reinterpret_cast<const float4 *>(swt)[2 * i + 1];
                const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    a.x += w[o] * gv[o].x;
                    a.y += w[o] * gv[o].y;
                }
                if (pre_in) {
                    a.x *= act_grad(act, w0, p[u].x);
                    a.y *= act_grad(act, w0, p[u].y);
                }
                st2(gx + (b * ci + i) * N + n, a.x, a.y);
            }
        }
    }
}

// gx = (W^T g) * (pre_in ? act'(pre_in) : 1), ci <= 32 (gx accumulated in registers).
template <class TP>
__global__ void __launch_bounds__(TPB) k_pw_bwd_in(const float *g, int co, int ci, const float *W, const TP *pre_in,
                                                   int act, float w0, float *gx, int64_t N, int B)
{
    extern __shared__ float sm[];
    for (int k = threadIdx.x; k < co * ci; k += blockDim.x) sm[k] = W[k];
    __syncthreads();
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / N, n = idx - b * N;
        float acc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = 0.f;
        for (int o = 0; o < co; ++o) {
            const float gv = g[(b * co + o) * N + n];
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (i < ci) acc[i] += sm[o * ci + i] * gv;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (i < ci) {
                const int64_t off = (b * ci + i) * N + n;
                gx[off] = pre_in ? acc[i] * act_grad(act, w0, ldf(pre_in + off)) : acc[i];
            }
    }
}

// Same for co <= 8 and any ci (g cached in registers, inputs streamed).
template <class TP>
__global__ void __launch_bounds__(TPB) k_pw_bwd_out(const float *g, int co, int ci, const float *W, const TP *pre_in,
                                                    int act, float w0, float *gx, int64_t N, int B)
{
    extern __shared__ float sm[];
    for (int k = threadIdx.x; k < co * ci; k += blockDim.x) sm[k] = W[k];
    __syncthreads();
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / N, n = idx - b * N;
        float gv[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) gv[o] = o < co ? g[(b * co + o) * N + n] : 0.f;
        for (int i = 0; i < ci; ++i) {
            float acc = 0.f;
#pragma unroll
            for (int o = 0; o < 8; ++o)
                if (o < co) acc += sm[o * ci + i] * gv[o];
            const int64_t off = (b * ci + i) * N + n;
            gx[off] = pre_in ? acc * act_grad(act, w0, ldf(pre_in + off)) : acc;
        }
    }
}

// gW[o][i] += sum_{b,cell} g[b][o][cell] x[b][i][cell], gb[o] += sum g.  A
// block reduces a chunk of cells: tiles of OUTER_TILE cells are staged in
// shared memory as rows [channel][cell]; a thread owns four outputs o0..o0+3
// and four inputs i0 + 8u (u < 4) and walks a range of the tile four cells at
// a time (float4).  The eight lanes of a quarter warp share o0 (broadcast
// reads) and take consecutive i0 (rows 68 floats apart: distinct banks).
// When there are fewer than TPB such units, `groups` threads split the cells
// of a tile.  Partial sums are added atomically at the end.
constexpr int OUTER_TILE = 64;
constexpr int OUTER_LD = OUTER_TILE + 4;
constexpr int OUTER_CHUNK = 8192;

template <class TX, int UPT>
__global__ void __launch_bounds__(TPB) k_outer(const float *g, int co, const TX *x, int ci, float *gW, float *gb,
                                               int64_t N, int B, int groups)
{
    extern __shared__ float4 smv[];
    const int cop = (co + 3) & ~3, cip = ((ci + 31) / 32) * 32;
    const int nog = cop / 4, units = nog * (cip / 32) * 8;
    const int qpg = (OUTER_TILE / 4) / groups;
    float *sg = reinterpret_cast<float *>(smv);              // [cop][OUTER_LD]
    float *sx = sg + (size_t)cop * OUTER_LD;                 // [cip][OUTER_LD]
    float acc[UPT][16], bacc[UPT][4];
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[u][k] = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) bacc[u][k] = 0.f;
    }
    const int64_t total = (int64_t)B * N;
    const int64_t c0 = (int64_t)blockIdx.x * OUTER_CHUNK;
    const int64_t c1 = c0 + OUTER_CHUNK < total ? c0 + OUTER_CHUNK : total;
    const int jst = threadIdx.x % OUTER_TILE, chst = threadIdx.x / OUTER_TILE;
    const bool vec = N % OUTER_TILE == 0;                   // whole tiles inside one batch element
    constexpr int QPR = OUTER_TILE / 4;                     // float4 per staged row
    for (int64_t t0 = c0; t0 < c1; t0 += OUTER_TILE) {
        __syncthreads();
        if (vec) {
            const int64_t b = t0 / N, n0 = t0 - b * N;
            const int tot = (cop + cip) * QPR;
            for (int k0 = threadIdx.x; k0 < tot; k0 += 8 * TPB) {
                float4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {               // eight loads in flight before any store
                    const int k = k0 + u * TPB, ch = k / QPR, q = k % QPR;
                    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (k < tot) {
                        if (ch < co) v[u] = ld4(g + (b * co + ch) * N + n0 + 4 * q);
                        else if (ch >= cop && ch - cop < ci) v[u] = ld4(x + (b * ci + (ch - cop)) * N + n0 + 4 * q);
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = k0 + u * TPB;
                    if (k < tot) *reinterpret_cast<float4 *>(sg + (k / QPR) * OUTER_LD + 4 * (k % QPR)) = v[u];
                }
            }
        } else {
            const int64_t cell = t0 + jst;
            const bool cv = cell < c1;
            const int64_t b = cv ? cell / N : 0, n = cell - b * N;
            for (int ch = chst; ch < cop + cip; ch += TPB / OUTER_TILE) {
                float v = 0.f;
                if (cv) {
                    if (ch < co) v = g[(b * co + ch) * N + n];
                    else if (ch >= cop && ch - cop < ci) v = ldf(x + (b * ci + (ch - cop)) * N + n);
                }
                sg[ch * OUTER_LD + jst] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
            const int t = threadIdx.x + u * TPB;
            if (t >= units * groups) break;
            const int unit = t % units, grp = t / units;
            const int l8 = unit & 7, rest = unit >> 3;
            const int o0 = (rest % nog) * 4, i0 = (rest / nog) * 32 + l8;
            const bool bias = l8 == 0 && rest < nog;
            for (int q = grp * qpg; q < (grp + 1) * qpg; ++q) {
                float4 gv[4], xv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) gv[a] = *reinterpret_cast<const float4 *>(sg + (o0 + a) * OUTER_LD + 4 * q);
#pragma unroll
                for (int c = 0; c < 4; ++c) xv[c] = *reinterpret_cast<const float4 *>(sx + (i0 + 8 * c) * OUTER_LD + 4 * q);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        acc[u][4 * a + c] += gv[a].x * xv[c].x + gv[a].y * xv[c].y + gv[a].z * xv[c].z + gv[a].w * xv[c].w;
                if (bias) {
#pragma unroll
                    for (int a = 0; a < 4; ++a) bacc[u][a] += gv[a].x + gv[a].y + gv[a].z + gv[a].w;
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
        const int t = threadIdx.x + u * TPB;
        if (t >= units * groups) break;
        const int unit = t % units;
        const int l8 = unit & 7, rest = unit >> 3;
        const int o0 = (rest % nog) * 4, i0 = (rest / nog) * 32 + l8;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            if (o0 + a >= co) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (i0 + 8 * c < ci) atomicAdd(&gW[(o0 + a) * ci + i0 + 8 * c], acc[u][4 * a + c]);
            if (l8 == 0 && rest < nog) atomicAdd(&gb[o0 + a], bacc[u][a]);
        }
    }
}

// The same reduction when tiles never straddle a batch element (N a multiple
// of OUTER_TILE): tiles are copied into shared memory by cp.async, two
// buffers deep, so the copy of tile t+1 runs while tile t is reduced.  The
// inputs stay in their storage type in shared memory (BF16 rows 72 elements
// apart: 8-byte reads of eight consecutive rows hit distinct banks).
template <class TX> struct OuterX;
template <> struct OuterX<float> {
    static constexpr int LD = OUTER_TILE + 4;
    static __device__ __forceinline__ float4 ld(const float *p) { return *reinterpret_cast<const float4 *>(p); }
};
template <> struct OuterX<__nv_bfloat16> {
    static constexpr int LD = OUTER_TILE + 8;
    static __device__ __forceinline__ float4 ld(const __nv_bfloat16 *p) { return ld4(p); }
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NG> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NG) : "memory"); }

template <class TX>
__host__ __device__ constexpr size_t outer_buf_bytes(int cop, int cip)
{
    return sizeof(float) * (size_t)cop * OUTER_LD + sizeof(TX) * (size_t)cip * OuterX<TX>::LD;
}

template <class TX, int UPT>
__global__ void __launch_bounds__(TPB) k_outer_async(const float *g, int co, const TX *x, int ci, float *gW, float *gb,
                                                     int64_t N, int B, int groups)
{
    using XR = OuterX<TX>;
    extern __shared__ float4 smv[];
    const int cop = (co + 3) & ~3, cip = ((ci + 31) / 32) * 32;
    const int nog = cop / 4, units = nog * (cip / 32) * 8;
    const int qpg = (OUTER_TILE / 4) / groups;
    const size_t buf = outer_buf_bytes<TX>(cop, cip);
    char *base = reinterpret_cast<char *>(smv);
    for (size_t k = threadIdx.x; k < 2 * buf / 16; k += TPB) smv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();                                        // padding rows stay zero
    float acc[UPT][16], bacc[UPT][4];
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[u][k] = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) bacc[u][k] = 0.f;
    }
    const int64_t total = (int64_t)B * N;
    const int64_t c0 = (int64_t)blockIdx.x * OUTER_CHUNK;
    const int64_t c1 = c0 + OUTER_CHUNK < total ? c0 + OUTER_CHUNK : total;
    const int ntile = (int)((c1 - c0) / OUTER_TILE);
    constexpr int GCH = OUTER_TILE / 4;                     // 16-byte pieces of a gradient row
    constexpr int PER = 16 / (int)sizeof(TX);               // input elements per 16 bytes
    constexpr int XCH = OUTER_TILE / PER;
    auto issue = [&](int t, int bsel) {
        const int64_t t0 = c0 + (int64_t)t * OUTER_TILE;
        const int64_t bb = t0 / N, n0 = t0 - bb * N;
        float *sg = reinterpret_cast<float *>(base + bsel * buf);
        TX *sx = reinterpret_cast<TX *>(base + bsel * buf + sizeof(float) * (size_t)cop * OUTER_LD);
        const int ng = co * GCH, nt = ng + ci * XCH;
        for (int k = threadIdx.x; k < nt; k += TPB) {
            if (k < ng) {
                const int ch = k / GCH, q = k % GCH;
                cp_async16(sg + ch * OUTER_LD + 4 * q, g + (bb * co + ch) * N + n0 + 4 * q);
            } else {
                const int kk = k - ng, ch = kk / XCH, q = kk % XCH;
                cp_async16(sx + ch * XR::LD + PER * q, x + (bb * ci + ch) * N + n0 + PER * q);
            }
        }
        cp_async_commit();
    };
    if (ntile > 0) issue(0, 0);
    for (int t = 0; t < ntile; ++t) {
        if (t + 1 < ntile) {
            issue(t + 1, (t + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *sg = reinterpret_cast<const float *>(base + (t & 1) * buf);
        const TX *sx = reinterpret_cast<const TX *>(base + (t & 1) * buf + sizeof(float) * (size_t)cop * OUTER_LD);
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
            const int tt = threadIdx.x + u * TPB;
            if (tt >= units * groups) break;
            const int unit = tt % units, grp = tt / units;
            const int l8 = unit & 7, rest = unit >> 3;
            const int o0 = (rest % nog) * 4, i0 = (rest / nog) * 32 + l8;
            const bool bias = l8 == 0 && rest < nog;
            for (int q = grp * qpg; q < (grp + 1) * qpg; ++q) {
                float4 gv[4], xv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) gv[a] = *reinterpret_cast<const float4 *>(sg + (o0 + a) * OUTER_LD + 4 * q);
#pragma unroll
                for (int c = 0; c < 4; ++c) xv[c] = XR::ld(sx + (i0 + 8 * c) * XR::LD + 4 * q);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        acc[u][4 * a + c] += gv[a].x * xv[c].x + gv[a].y * xv[c].y + gv[a].z * xv[c].z + gv[a].w * xv[c].w;
                if (bias) {
#pragma unroll
                    for (int a = 0; a < 4; ++a) bacc[u][a] += gv[a].x + gv[a].y + gv[a].z + gv[a].w;
                }
            }
        }
        __syncthreads();                                    // the buffer is refilled two tiles on
    }
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
        const int tt = threadIdx.x + u * TPB;
        if (tt >= units * groups) break;
        const int unit = tt % units;
        const int l8 = unit & 7, rest = unit >> 3;
        const int o0 = (rest % nog) * 4, i0 = (rest / nog) * 32 + l8;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            if (o0 + a >= co) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (i0 + 8 * c < ci) atomicAdd(&gW[(o0 + a) * ci + i0 + 8 * c], acc[u][4 * a + c]);
            if (l8 == 0 && rest < nog) atomicAdd(&gb[o0 + a], bacc[u][a]);
        }
    }
}

int outer_units(int co, int ci) { return ((co + 3) / 4) * ((ci + 31) / 32) * 8; }
size_t smem_outer(int co, int ci)
{
    const int cop = (co + 3) & ~3, cip = ((ci + 31) / 32) * 32;
    return std::max(sizeof(float) * (size_t)(cop + cip) * OUTER_LD,
                    2 * std::max(outer_buf_bytes<float>(cop, cip), outer_buf_bytes<__nv_bfloat16>(cop, cip)));
}

// ---------------------------------------------------------------------------
// truncated DFT: forward stages x -> y -> z, inverse stages z -> y -> x.
// Twiddles: twx[x][jx] = exp(-i 2 pi kx x / nx), twy[y][jy], twz[z][kz].
// Spectral tensors are mode-major: S[k][b*C + c], k = (kz*Ky + jy)*Kx + jx.
// ---------------------------------------------------------------------------
struct Dims {
    int nx, ny, nz, Kx, Ky, Kz;
    int64_t BC;
};

constexpr int DFT_RT = 8;                            // rows per warp in the x stages
constexpr int DFT_ROWS = DFT_RT * (TPB / 32);        // rows per block pass in the x stages

// rows [R][nx] (real) -> A [R][Kx] (complex), folded: exp(-i t (nx - x)) is
// the conjugate of exp(-i t x), so with S_p = v[p] + v[nx - p] and
// D_p = v[p] - v[nx - p] (p = 1 .. (nx-1)/2), S_0 = v[0], D_0 = 0 and, for
// even nx, S_{nx/2} = v[nx/2], D_{nx/2} = 0:
//     A_j = sum_{p <= nx/2} S_p cos_pj + i sum_p D_p sin_pj,
// half the multiply-adds of the plain sum.  A block stages DFT_ROWS rows of
// (S, D) in shared memory (np_ = nx/2 + 1 entries, padded to a multiple of
// 4); lane j of a warp owns mode j (chunks of 32) for the warp's DFT_RT rows,
// reading S and D four entries at a time (float4 broadcast) against the
// twiddles tw[p][j] (consecutive in j: conflict-free).
template <class TI>
__global__ void __launch_bounds__(TPB) k_dftx_fwd(const TI *x, float2 *A, const float2 *twx, Dims d, int64_t R)
{
    extern __shared__ float4 smv[];
    const int h = d.nx / 2, np_ = h + 1, npp = (np_ + 3) & ~3, nq = npp / 4;
    const int nxp = (d.nx + 3) & ~3;
    float2 *tw = reinterpret_cast<float2 *>(smv);                           // [npp][Kx]
    float *sd = reinterpret_cast<float *>(tw + (size_t)npp * d.Kx);        // [DFT_ROWS][2][npp]
    float *raw = sd + (size_t)DFT_ROWS * 2 * npp;                          // [DFT_ROWS][nxp]
    for (int k = threadIdx.x; k < npp * d.Kx; k += blockDim.x)
        tw[k] = k < np_ * d.Kx ? twx[k] : make_float2(0.f, 0.f);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t r0 = (int64_t)blockIdx.x * DFT_ROWS; r0 < R; r0 += (int64_t)gridDim.x * DFT_ROWS) {
        const int nr = (int)(R - r0 < DFT_ROWS ? R - r0 : DFT_ROWS);
        __syncthreads();
        if (nxp == d.nx) {                                  // rows are one contiguous run
            stage4(raw, x + r0 * d.nx, nr * d.nx, DFT_ROWS * nxp);
        } else {
            for (int k = threadIdx.x; k < DFT_ROWS * nxp; k += blockDim.x) {
                const int lr = k / nxp, xx = k - lr * nxp;
                raw[k] = (lr < nr && xx < d.nx) ? ldf(x + (r0 + lr) * d.nx + xx) : 0.f;
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < DFT_ROWS * npp; k += blockDim.x) {
            const int lr = k / npp, pp = k - lr * npp;
            float sv = 0.f, dv = 0.f;
            if (pp < np_) {
                const float *row = raw + (size_t)lr * nxp;
                const float a = row[pp];
                if (pp > 0 && pp < d.nx - pp) {
                    const float b = row[d.nx - pp];
                    sv = a + b;
                    dv = a - b;
                } else {
                    sv = a;                              // p = 0, or the middle sample of an even row
                }
            }
            sd[(2 * lr) * npp + pp] = sv;
            sd[(2 * lr + 1) * npp + pp] = dv;
        }
        __syncthreads();
        const float4 *rw = reinterpret_cast<const float4 *>(sd) + (size_t)warp * DFT_RT * 2 * nq;
        for (int j0 = 0; j0 < d.Kx; j0 += 32) {
            const int j = j0 + lane;
            const int jj = j < d.Kx ? j : d.Kx - 1;
            float2 acc[DFT_RT];
#pragma unroll
            for (int r = 0; r < DFT_RT; ++r) acc[r] = make_float2(0.f, 0.f);
            for (int q = 0; q < nq; ++q) {
                const float2 t0 = tw[(4 * q) * d.Kx + jj], t1 = tw[(4 * q + 1) * d.Kx + jj];
                const float2 t2 = tw[(4 * q + 2) * d.Kx + jj], t3 = tw[(4 * q + 3) * d.Kx + jj];
#pragma unroll
                for (int r = 0; r < DFT_RT; ++r) {
                    const float4 sv = rw[(2 * r) * nq + q], dv = rw[(2 * r + 1) * nq + q];
                    acc[r].x += sv.x * t0.x + sv.y * t1.x + sv.z * t2.x + sv.w * t3.x;
                    acc[r].y += dv.x * t0.y + dv.y * t1.y + dv.z * t2.y + dv.w * t3.y;
                }
            }
            if (j < d.Kx) {
#pragma unroll
                for (int r = 0; r < DFT_RT; ++r)
                    if (warp * DFT_RT + r < nr) A[(r0 + warp * DFT_RT + r) * d.Kx + j] = acc[r];
            }
        }
    }
}

// The same forward x stage on tensor cores, for rows of nx = 128 samples
// and Kx = 32 modes: A[R][32] = rows[R][128] T[128][64] with
// T[x][2j] = Re twx[x][j], T[x][2j + 1] = Im twx[x][j], as mma.sync
// m16n8k16 products (BF16 operands, FP32 accumulation); the transform is a
// dense contraction, and as such this stage is bound by its 0.5 KB of HBM
// traffic per row rather than by FP32 multiply-adds.  Each twiddle enters
// as a BF16 pair hi + lo (hi = bf16(t), lo = bf16(t - hi)).  BF16 samples
// are exact: two products per tile (hi, lo table); FP32 samples are split
// the same way: three products (hi hi, hi lo, lo hi).  Either keeps about
// 2^-16 relative error.  A warp takes 16 rows per pass.  Lane (g, c)
// (g = lane / 4, c = lane % 4) loads the 32 consecutive samples
// x in [32c, 32c + 32) of rows g and g + 8 with 16-byte loads, and the
// contraction index is permuted to match: in k-step s, fragment column
// 2c + {0, 1} is sample 32c + 4s + {0, 1} and column 2c + 8 + {0, 1} is
// sample 32c + 4s + {2, 3}.  The table is stored in that order, fragment by
// fragment, so a lane reads its two B registers with one 8-byte load.
constexpr int TCX_NX = 128, TCX_KX = 32;

__device__ __forceinline__ uint32_t pack_bf16_pair(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// acc (m16n8 FP32 fragment) += A (m16k16 BF16: a0..a3) B (k16n8 BF16: b.x, b.y)
__device__ __forceinline__ void mma_bf16(float *acc, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint2 b)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                 : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b.x), "r"(b.y));
}

template <class TI>
__global__ void __launch_bounds__(TPB) k_dftx_fwd_tc(const TI *x, float2 *A, const float2 *twx, int64_t R)
{
    __shared__ uint2 bt[2][8 * 8 * 32];     // [hi, lo][(k-step * 8 + n-tile) * 32 + lane]
    for (int idx = threadIdx.x; idx < 8 * 8 * 32; idx += blockDim.x) {
        const int st = idx >> 8, nt = (idx >> 5) & 7, l = idx & 31;
        const int n = 8 * nt + (l >> 2), c = l & 3;
        const int j = n >> 1, im = n & 1;
        __nv_bfloat16 h[4], o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int xs = 32 * c + 4 * st + e;
            const float2 t = twx[xs * TCX_KX + j];
            const float v = im ? t.y : t.x;
            h[e] = __float2bfloat16_rn(v);
            o[e] = __float2bfloat16_rn(v - __bfloat162float(h[e]));
        }
        bt[0][idx] = make_uint2(pack_bf16_pair(h[0], h[1]), pack_bf16_pair(h[2], h[3]));
        bt[1][idx] = make_uint2(pack_bf16_pair(o[0], o[1]), pack_bf16_pair(o[2], o[3]));
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const int64_t tiles = (R + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * (TPB / 32) + warp; tile < tiles; tile += (int64_t)gridDim.x * (TPB / 32)) {
        const int64_t ra = tile * 16 + g, rb = ra + 8;
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
        if (std::is_same<TI, __nv_bfloat16>::value) {
            uint4 va[4], vb[4];
            const uint4 *pa = reinterpret_cast<const uint4 *>(x + ra * TCX_NX + 32 * c);
            const uint4 *pb = reinterpret_cast<const uint4 *>(x + rb * TCX_NX + 32 * c);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                va[q] = ra < R ? pa[q] : make_uint4(0u, 0u, 0u, 0u);
                vb[q] = rb < R ? pb[q] : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int st = 0; st < 8; ++st) {
                const uint4 &ua = va[st >> 1], &ub = vb[st >> 1];
                const uint32_t a0 = (st & 1) ? ua.z : ua.x, a2 = (st & 1) ? ua.w : ua.y;
                const uint32_t a1 = (st & 1) ? ub.z : ub.x, a3 = (st & 1) ? ub.w : ub.y;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        const uint2 b = bt[part][(st * 8 + nt) * 32 + lane];
                        mma_bf16(acc[nt], a0, a1, a2, a3, b);
                    }
                }
            }
        } else {
            const float4 *pa = reinterpret_cast<const float4 *>(x + ra * TCX_NX + 32 * c);
            const float4 *pb = reinterpret_cast<const float4 *>(x + rb * TCX_NX + 32 * c);
#pragma unroll
            for (int st = 0; st < 8; ++st) {
                // samples 32c + 4st + {0..3} of rows ra and rb
                const float4 fa = ra < R ? pa[st] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 fb = rb < R ? pb[st] : make_float4(0.f, 0.f, 0.f, 0.f);
                __nv_bfloat16 ah[8], al[8];
                split_bf16(fa.x, ah[0], al[0]); split_bf16(fa.y, ah[1], al[1]);
                split_bf16(fa.z, ah[2], al[2]); split_bf16(fa.w, ah[3], al[3]);
                split_bf16(fb.x, ah[4], al[4]); split_bf16(fb.y, ah[5], al[5]);
                split_bf16(fb.z, ah[6], al[6]); split_bf16(fb.w, ah[7], al[7]);
                const uint32_t h0 = pack_bf16_pair(ah[0], ah[1]), h2 = pack_bf16_pair(ah[2], ah[3]);
                const uint32_t h1 = pack_bf16_pair(ah[4], ah[5]), h3 = pack_bf16_pair(ah[6], ah[7]);
                const uint32_t l0 = pack_bf16_pair(al[0], al[1]), l2 = pack_bf16_pair(al[2], al[3]);
                const uint32_t l1 = pack_bf16_pair(al[4], al[5]), l3 = pack_bf16_pair(al[6], al[7]);
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const uint2 bh = bt[0][(st * 8 + nt) * 32 + lane], bl = bt[1][(st * 8 + nt) * 32 + lane];
                    mma_bf16(acc[nt], h0, h1, h2, h3, bh);
                    mma_bf16(acc[nt], h0, h1, h2, h3, bl);
                    mma_bf16(acc[nt], l0, l1, l2, l3, bh);
                }
            }
        }
        // D: (row g, columns 2c, 2c + 1) and (row g + 8, same columns) of
        // n-tile nt: the real and imaginary part of mode 4 nt + c
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (ra < R) A[ra * TCX_KX + 4 * nt + c] = make_float2(acc[nt][0], acc[nt][1]);
            if (rb < R) A[rb * TCX_KX + 4 * nt + c] = make_float2(acc[nt][2], acc[nt][3]);
        }
    }
}

// A [S][ny][Kx] -> B [S][Ky][Kx] = sum_y A exp(-i 2 pi ky y / ny), S = BC*nz
// slabs.  A block stages SB slabs per pass; a warp takes one slab and eight
// consecutive jy, a lane one jx; twiddles tw[y][jy] (jy padded to kyp, a
// multiple of 8) are read as float4 broadcasts.
__global__ void __launch_bounds__(TPB) k_dfty_fwd(const float2 *A, float2 *Bt, const float2 *twy, Dims d, int64_t S,
                                                  int SB)
{
    extern __shared__ float4 smv[];
    const int kyp = (d.Ky + 7) & ~7, cps = kyp / 8;
    const int slab_n = d.ny * d.Kx;
    float2 *tw = reinterpret_cast<float2 *>(smv);                           // [ny][kyp]
    float2 *slab = tw + (size_t)d.ny * kyp;                                 // [SB][ny][Kx]
    for (int k = threadIdx.x; k < d.ny * kyp; k += blockDim.x) {
        const int y = k / kyp, jy = k - y * kyp;
        tw[k] = jy < d.Ky ? twy[y * d.Ky + jy] : make_float2(0.f, 0.f);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t s0 = (int64_t)blockIdx.x * SB; s0 < S; s0 += (int64_t)gridDim.x * SB) {
        const int ns = (int)(S - s0 < SB ? S - s0 : SB);
        __syncthreads();
        stage4(reinterpret_cast<float *>(slab), reinterpret_cast<const float *>(A + s0 * slab_n), 2 * ns * slab_n,
               2 * SB * slab_n);
        __syncthreads();
        for (int task = warp; task < ns * cps; task += TPB / 32) {
            const int sb = task / cps, jc = task - sb * cps;
            const float2 *sl = slab + (size_t)sb * slab_n;
            for (int jx0 = 0; jx0 < d.Kx; jx0 += 32) {
                const int jx = jx0 + lane;
                const int jj = jx < d.Kx ? jx : d.Kx - 1;
                float2 acc[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
                for (int y = 0; y < d.ny; ++y) {
                    const float2 v = sl[y * d.Kx + jj];
                    const float4 *t4 = reinterpret_cast<const float4 *>(tw + y * kyp + jc * 8);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 t = t4[u];
                        acc[2 * u].x += v.x * t.x - v.y * t.y;
                        acc[2 * u].y += v.x * t.y + v.y * t.x;
                        acc[2 * u + 1].x += v.x * t.z - v.y * t.w;
                        acc[2 * u + 1].y += v.x * t.w + v.y * t.z;
                    }
                }
                if (jx < d.Kx) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int jy = jc * 8 + q;
                        if (jy < d.Ky) Bt[((s0 + sb) * d.Ky + jy) * d.Kx + jx] = acc[q];
                    }
                }
            }
        }
    }
}

// z stages: a block of ZW warps takes one channel row bc and 32 consecutive
// (ky, kx) modes (a lane each, so that the rows of a plane are read and
// written coalesced); the nz planes are split among the warps, which raises
// the parallelism of these short stages fourfold over one thread per mode.
constexpr int ZW = 4;

int dftz_blocks(const Dims &d)
{
    const int64_t items = d.BC * ((d.Ky * d.Kx + 31) / 32);
    return (int)std::min<int64_t>(items, (int64_t)gb300::sm_count() * 16);
}

// B [BC][nz][Ky][Kx] -> S[k][bc] with factor scale[kz]: each warp sums its
// planes, the partial sums are added in warp order.
__global__ void __launch_bounds__(ZW * 32) k_dftz_fwd(const float2 *Bt, float2 *Sp, const float2 *twz, const float *scale,
                                                      Dims d)
{
    __shared__ float2 part[ZW][16][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int P2 = d.Ky * d.Kx, pchunks = (P2 + 31) / 32;
    const int z0 = w * d.nz / ZW, z1 = (w + 1) * d.nz / ZW;
    for (int64_t item = blockIdx.x; item < d.BC * pchunks; item += gridDim.x) {
        const int64_t bc = item / pchunks;
        const int pbase = (int)(item % pchunks) * 32;
        const int p = pbase + lane;
        float2 acc[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = make_float2(0.f, 0.f);
        if (p < P2) {
            for (int z = z0; z < z1; ++z) {
                const float2 v = Bt[(bc * d.nz + z) * P2 + p];
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < d.Kz) {
                        const float2 t = cmul(v, twz[z * d.Kz + k]);
                        acc[k].x += t.x;
                        acc[k].y += t.y;
                    }
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < d.Kz) part[w][k][lane] = acc[k];
        __syncthreads();
        for (int e = threadIdx.x; e < d.Kz * 32; e += ZW * 32) {
            const int k = e >> 5, l = e & 31;
            if (pbase + l < P2) {
                float2 s = part[0][k][l];
#pragma unroll
                for (int ww = 1; ww < ZW; ++ww) {
                    s.x += part[ww][k][l].x;
                    s.y += part[ww][k][l].y;
                }
                Sp[((int64_t)k * P2 + pbase + l) * d.BC + bc] = make_float2(s.x * scale[k], s.y * scale[k]);
            }
        }
        __syncthreads();
    }
}

// S[k][bc] (times scale[kz]) -> H [BC][nz][Ky][Kx] = sum_kz G exp(+i 2 pi kz z / nz);
// each warp writes its own planes.
__global__ void __launch_bounds__(ZW * 32) k_dftz_inv(const float2 *Sp, float2 *Ht, const float2 *twz, const float *scale,
                                                      Dims d)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int P2 = d.Ky * d.Kx, pchunks = (P2 + 31) / 32;
    const int z0 = w * d.nz / ZW, z1 = (w + 1) * d.nz / ZW;
    for (int64_t item = blockIdx.x; item < d.BC * pchunks; item += gridDim.x) {
        const int64_t bc = item / pchunks;
        const int p = (int)(item % pchunks) * 32 + lane;
        if (p >= P2) continue;
        float2 G[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            G[k] = make_float2(0.f, 0.f);
            if (k < d.Kz) {
                const float2 v = Sp[((int64_t)k * P2 + p) * d.BC + bc];
                G[k] = make_float2(v.x * scale[k], v.y * scale[k]);
            }
        }
        for (int z = z0; z < z1; ++z) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < d.Kz) {
                    const float2 t = cmulc(G[k], twz[z * d.Kz + k]);
                    acc.x += t.x;
                    acc.y += t.y;
                }
            Ht[(bc * d.nz + z) * P2 + p] = acc;
        }
    }
}

// H [S][Ky][Kx] -> I [S][ny][Kx] = sum_jy H exp(+i 2 pi ky y / ny).  A warp
// takes one slab and eight consecutive y, a lane one jx; the twiddles are
// transposed into twT[jy][y] (y padded to nyp) so that eight y are two
// float4 broadcasts.
__global__ void __launch_bounds__(TPB) k_dfty_inv(const float2 *Ht, float2 *It, const float2 *twy, Dims d, int64_t S,
                                                  int SB)
{
    extern __shared__ float4 smv[];
    const int nyp = (d.ny + 7) & ~7, cps = nyp / 8;
    const int slab_n = d.Ky * d.Kx;
    float2 *tw = reinterpret_cast<float2 *>(smv);                           // [Ky][nyp]
    float2 *slab = tw + (size_t)d.Ky * nyp;                                 // [SB][Ky][Kx]
    for (int k = threadIdx.x; k < d.Ky * nyp; k += blockDim.x) {
        const int jy = k / nyp, y = k - jy * nyp;
        tw[k] = y < d.ny ? twy[y * d.Ky + jy] : make_float2(0.f, 0.f);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t s0 = (int64_t)blockIdx.x * SB; s0 < S; s0 += (int64_t)gridDim.x * SB) {
        const int ns = (int)(S - s0 < SB ? S - s0 : SB);
        __syncthreads();
        stage4(reinterpret_cast<float *>(slab), reinterpret_cast<const float *>(Ht + s0 * slab_n), 2 * ns * slab_n,
               2 * SB * slab_n);
        __syncthreads();
        for (int task = warp; task < ns * cps; task += TPB / 32) {
            const int sb = task / cps, yc = task - sb * cps;
            const float2 *sl = slab + (size_t)sb * slab_n;
            for (int jx0 = 0; jx0 < d.Kx; jx0 += 32) {
                const int jx = jx0 + lane;
                const int jj = jx < d.Kx ? jx : d.Kx - 1;
                float2 acc[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
                for (int jy = 0; jy < d.Ky; ++jy) {
                    const float2 v = sl[jy * d.Kx + jj];
                    const float4 *t4 = reinterpret_cast<const float4 *>(tw + jy * nyp + yc * 8);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {               // v conj(t)
                        const float4 t = t4[u];
                        acc[2 * u].x += v.x * t.x + v.y * t.y;
                        acc[2 * u].y += v.y * t.x - v.x * t.y;
                        acc[2 * u + 1].x += v.x * t.z + v.y * t.w;
                        acc[2 * u + 1].y += v.y * t.z - v.x * t.w;
                    }
                }
                if (jx < d.Kx) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int y = yc * 8 + q;
                        if (y < d.ny) It[((s0 + sb) * d.ny + y) * d.Kx + jx] = acc[q];
                    }
                }
            }
        }
    }
}

// I [R][Kx] -> out [R][nx] = Re sum_jx I exp(+i 2 pi kx x / nx); mode 0: store,
// mode 1: add to out; then, if pre is given, multiply by gelu'(pre).
// Folded: with (c, s) the twiddle of sample p, a_p = sum_j Re(I_j) c_pj and
// b_p = sum_j Im(I_j) s_pj give out[p] = a_p + b_p and out[nx - p] =
// a_p - b_p (p = 1 .. (nx-1)/2), out[0] = a_0; the middle sample of an even
// row, out[nx/2] = sum_j Re(I_j) (-1)^k_j, is a warp reduction.  The
// twiddles are transposed into twT[j][p] (p padded to a multiple of 64) so
// that lane l reads p = l + 32u (u < 2) conflict-free; a warp takes DFT_RT
// rows and reads their coefficients two modes at a time (float4 broadcast).
template <class TP>
__global__ void __launch_bounds__(TPB) k_dftx_inv(const float2 *It, float *out, const float2 *twx, Dims d, int64_t R,
                                                  int accumulate, const TP *pre)
{
    extern __shared__ float4 smv[];
    const int ns = (d.nx + 1) / 2, ldp = (ns + 63) & ~63, kh = d.Kx / 2;
    const bool mid = (d.nx & 1) == 0;
    float2 *tw = reinterpret_cast<float2 *>(smv);                           // [Kx][ldp]
    float4 *rows = reinterpret_cast<float4 *>(tw + (size_t)d.Kx * ldp);    // [DFT_ROWS][Kx/2]
    for (int k = threadIdx.x; k < d.Kx * ldp; k += blockDim.x) {
        const int j = k / ldp, pp = k - j * ldp;
        tw[k] = pp < ns ? twx[pp * d.Kx + j] : make_float2(0.f, 0.f);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t r0 = (int64_t)blockIdx.x * DFT_ROWS; r0 < R; r0 += (int64_t)gridDim.x * DFT_ROWS) {
        const int nr = (int)(R - r0 < DFT_ROWS ? R - r0 : DFT_ROWS);
        __syncthreads();
        stage4(reinterpret_cast<float *>(rows), reinterpret_cast<const float *>(It + r0 * d.Kx), 2 * nr * d.Kx,
               2 * DFT_ROWS * d.Kx);
        __syncthreads();
        const float4 *rw = rows + (size_t)warp * DFT_RT * kh;
        for (int pc = 0; pc < ns; pc += 64) {
            float a[DFT_RT][2], b[DFT_RT][2];
#pragma unroll
            for (int r = 0; r < DFT_RT; ++r)
#pragma unroll
                for (int u = 0; u < 2; ++u) a[r][u] = b[r][u] = 0.f;
            for (int jp = 0; jp < kh; ++jp) {
                float2 ta[2], tb[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    ta[u] = tw[(2 * jp) * ldp + pc + lane + 32 * u];
                    tb[u] = tw[(2 * jp + 1) * ldp + pc + lane + 32 * u];
                }
#pragma unroll
                for (int r = 0; r < DFT_RT; ++r) {
                    const float4 v = rw[r * kh + jp];               // modes 2jp, 2jp+1 of row r
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        a[r][u] += v.x * ta[u].x + v.z * tb[u].x;
                        b[r][u] += v.y * ta[u].y + v.w * tb[u].y;
                    }
                }
            }
            // epilogue four rows at a time: all loads of a group before its stores
#pragma unroll
            for (int r4 = 0; r4 < DFT_RT; r4 += 4) {
                float prev[4][2][2], pv[4][2][2];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int pp = pc + lane + 32 * u;
                        const bool ok = warp * DFT_RT + r4 + r < nr && pp < ns;
                        const int64_t base = (r0 + warp * DFT_RT + r4 + r) * d.nx;
                        const int64_t o1 = base + pp, o2 = base + (d.nx - pp);
                        const bool ok2 = ok && pp > 0;
                        prev[r][u][0] = ok && accumulate ? out[o1] : 0.f;
                        prev[r][u][1] = ok2 && accumulate ? out[o2] : 0.f;
                        pv[r][u][0] = ok && pre ? ldf(pre + o1) : 0.f;
                        pv[r][u][1] = ok2 && pre ? ldf(pre + o2) : 0.f;
                    }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int pp = pc + lane + 32 * u;
                        if (warp * DFT_RT + r4 + r >= nr || pp >= ns) continue;
                        const int64_t base = (r0 + warp * DFT_RT + r4 + r) * d.nx;
                        float v1 = a[r4 + r][u] + b[r4 + r][u] + prev[r][u][0];
                        if (pre) v1 *= gelu_grad(pv[r][u][0]);
                        out[base + pp] = v1;
                        if (pp > 0) {
                            float v2 = a[r4 + r][u] - b[r4 + r][u] + prev[r][u][1];
                            if (pre) v2 *= gelu_grad(pv[r][u][1]);
                            out[base + d.nx - pp] = v2;
                        }
                    }
            }
        }
        if (mid) {                                           // out[nx/2] = sum_j Re(I_j) c_(nx/2) j
            const int hmid = d.nx / 2;
            const float2 *rows2 = reinterpret_cast<const float2 *>(rows);
            for (int r = 0; r < DFT_RT; ++r) {
                const int row = warp * DFT_RT + r;
                float sum = 0.f;
                for (int j = lane; j < d.Kx; j += 32) sum += rows2[(size_t)row * d.Kx + j].x * twx[hmid * d.Kx + j].x;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
                if (lane == 0 && row < nr) {
                    const int64_t off = (r0 + row) * d.nx + hmid;
                    float v = accumulate ? out[off] + sum : sum;
                    if (pre) v *= gelu_grad(ldf(pre + off));
                    out[off] = v;
                }
            }
        }
    }
}

// The same inverse x stage on tensor cores for nx = 128 and Kx = 32:
// out[R][128] (+)= I[R][64] T[64][128], I read as 64 reals per row (the
// real and imaginary part of each mode in turn) and T[2j][x] = Re twx[x][j],
// T[2j + 1][x] = Im twx[x][j] (Im twx = -sin, so the sum is the real part
// of sum_j I_j exp(+i 2 pi k_j x / nx)).  Both operands enter as BF16
// pairs hi + lo, and three products per tile (hi hi, hi lo, lo hi) keep
// about 2^-16 relative error.  A warp takes 16 rows per pass.  Lane (g, c)
// loads the 16 consecutive reals [16c, 16c + 16) of rows g and g + 8 with
// 16-byte loads; in k-step s, fragment column 2c + {0, 1} is real
// 16c + 4s + {0, 1} and column 2c + 8 + {0, 1} is real 16c + 4s + {2, 3},
// and the table is stored in that order, fragment by fragment.  The
// epilogue adds the previous output (accumulate) and multiplies by
// gelu'(pre) when pre is given, as the plain kernel does.

template <class TP>
__global__ void __launch_bounds__(TPB) k_dftx_inv_tc(const float2 *It, float *out, const float2 *twx, int64_t R,
                                                     int accumulate, const TP *pre)
{
    __shared__ uint2 bt[2][4 * 16 * 32];    // [hi, lo][(k-step * 16 + n-tile) * 32 + lane]
    for (int idx = threadIdx.x; idx < 4 * 16 * 32; idx += blockDim.x) {
        const int st = idx >> 9, nt = (idx >> 5) & 15, l = idx & 31;
        const int xs = 8 * nt + (l >> 2), c = l & 3;
        __nv_bfloat16 h[4], o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = 16 * c + 4 * st + e;          // real index: mode k / 2, part k % 2
            const float2 t = twx[xs * TCX_KX + (k >> 1)];
            split_bf16((k & 1) ? t.y : t.x, h[e], o[e]);
        }
        bt[0][idx] = make_uint2(pack_bf16_pair(h[0], h[1]), pack_bf16_pair(h[2], h[3]));
        bt[1][idx] = make_uint2(pack_bf16_pair(o[0], o[1]), pack_bf16_pair(o[2], o[3]));
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const int64_t tiles = (R + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * (TPB / 32) + warp; tile < tiles; tile += (int64_t)gridDim.x * (TPB / 32)) {
        const int64_t ra = tile * 16 + g, rb = ra + 8;
        float4 va[4], vb[4];
        const float4 *pa = reinterpret_cast<const float4 *>(It + ra * TCX_KX) + 4 * c;
        const float4 *pb = reinterpret_cast<const float4 *>(It + rb * TCX_KX) + 4 * c;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            va[q] = ra < R ? pa[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            vb[q] = rb < R ? pb[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
        for (int st = 0; st < 4; ++st) {
            // reals 16c + 4st + {0..3} of rows ra (va[st]) and rb (vb[st])
            __nv_bfloat16 ah[8], al[8];
            split_bf16(va[st].x, ah[0], al[0]); split_bf16(va[st].y, ah[1], al[1]);
            split_bf16(va[st].z, ah[2], al[2]); split_bf16(va[st].w, ah[3], al[3]);
            split_bf16(vb[st].x, ah[4], al[4]); split_bf16(vb[st].y, ah[5], al[5]);
            split_bf16(vb[st].z, ah[6], al[6]); split_bf16(vb[st].w, ah[7], al[7]);
            const uint32_t h0 = pack_bf16_pair(ah[0], ah[1]), h2 = pack_bf16_pair(ah[2], ah[3]);
            const uint32_t h1 = pack_bf16_pair(ah[4], ah[5]), h3 = pack_bf16_pair(ah[6], ah[7]);
            const uint32_t l0 = pack_bf16_pair(al[0], al[1]), l2 = pack_bf16_pair(al[2], al[3]);
            const uint32_t l1 = pack_bf16_pair(al[4], al[5]), l3 = pack_bf16_pair(al[6], al[7]);
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                const uint2 bh = bt[0][(st * 16 + nt) * 32 + lane];
                const uint2 bl = bt[1][(st * 16 + nt) * 32 + lane];
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                    : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
                    : "r"(h0), "r"(h1), "r"(h2), "r"(h3), "r"(bh.x), "r"(bh.y));
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                    : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
                    : "r"(h0), "r"(h1), "r"(h2), "r"(h3), "r"(bl.x), "r"(bl.y));
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                    : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
                    : "r"(l0), "r"(l1), "r"(l2), "r"(l3), "r"(bh.x), "r"(bh.y));
            }
        }
        // D of n-tile nt: samples x = 8 nt + 2c + {0, 1} of rows g and g + 8
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const int xs = 8 * nt + 2 * c;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t r = h ? rb : ra;
                if (r >= R) continue;
                float2 v = make_float2(acc[nt][2 * h], acc[nt][2 * h + 1]);
                float2 *dst = reinterpret_cast<float2 *>(out + r * TCX_NX + xs);
                if (accumulate) {
                    const float2 p0 = *dst;
                    v.x += p0.x;
                    v.y += p0.y;
                }
                if (pre) {
                    v.x *= gelu_grad(ldf(pre + r * TCX_NX + xs));
                    v.y *= gelu_grad(ldf(pre + r * TCX_NX + xs + 1));
                }
                *dst = v;
            }
        }
    }
}

// Weight and bias gradients gW[o][i] += sum over cells of g[b][o][cell]
// x[b][i][cell] and gb[o] += sum g, on tensor cores, for BF16 inputs with
// ci = 32 and co a multiple of 32: D = A B with the cells as the contraction
// index, A = g (FP32, entering as BF16 hi + lo pairs, two products per
// tile), B = x (BF16, exact); a fifth n-tile whose first column is 1 gives
// the bias gradient.  Grid x: chunks of OUTER_CHUNK cells; grid y: groups of
// 32 output rows (two m-tiles).  A warp takes every eighth 16-cell k-step of
// its block's chunk (a k-step never straddles samples: N % 16 == 0); the
// block adds its warps' fragments in shared memory, then adds the block's
// sums to gW and gb atomically, as the SIMT reduction does.
__global__ void __launch_bounds__(TPB) k_outer_tc(const float *g, int co, const __nv_bfloat16 *x, float *gW, float *gb,
                                                  int64_t N, int B)
{
    __shared__ float red[32][33];
    for (int k = threadIdx.x; k < 32 * 33; k += blockDim.x) (&red[0][0])[k] = 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
    const int o0 = blockIdx.y * 32;
    float acc[2][5][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 5; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
    const uint32_t onev = gq == 0 ? 0x3F803F80u : 0u;                 // bf16 (1, 1) in column 0
    const uint2 bones = make_uint2(onev, onev);
    const int64_t total = (int64_t)B * N;
    const int64_t c0 = (int64_t)blockIdx.x * OUTER_CHUNK;
    const int64_t c1 = c0 + OUTER_CHUNK < total ? c0 + OUTER_CHUNK : total;
    for (int64_t k0 = c0 + 16 * warp; k0 < c1; k0 += 16 * (TPB / 32)) {
        const int64_t bb = k0 / N, n0 = k0 - bb * N;
        const float *gp = g + (bb * co + o0) * N + n0 + 2 * t;
        const __nv_bfloat16 *xp = x + (bb * 32 + gq) * N + n0 + 2 * t;
        uint2 bx[4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const __nv_bfloat16 *q = xp + (int64_t)(8 * nt) * N;
            bx[nt] = make_uint2(*reinterpret_cast<const uint32_t *>(q), *reinterpret_cast<const uint32_t *>(q + 8));
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const float *r0 = gp + (int64_t)(16 * mt + gq) * N, *r1 = r0 + 8 * N;
            const float2 p00 = *reinterpret_cast<const float2 *>(r0), p10 = *reinterpret_cast<const float2 *>(r1);
            const float2 p01 = *reinterpret_cast<const float2 *>(r0 + 8), p11 = *reinterpret_cast<const float2 *>(r1 + 8);
            __nv_bfloat16 h[8], l[8];
            split_bf16(p00.x, h[0], l[0]); split_bf16(p00.y, h[1], l[1]);
            split_bf16(p10.x, h[2], l[2]); split_bf16(p10.y, h[3], l[3]);
            split_bf16(p01.x, h[4], l[4]); split_bf16(p01.y, h[5], l[5]);
            split_bf16(p11.x, h[6], l[6]); split_bf16(p11.y, h[7], l[7]);
            const uint32_t a0 = pack_bf16_pair(h[0], h[1]), a1 = pack_bf16_pair(h[2], h[3]);
            const uint32_t a2 = pack_bf16_pair(h[4], h[5]), a3 = pack_bf16_pair(h[6], h[7]);
            const uint32_t c0l = pack_bf16_pair(l[0], l[1]), c1l = pack_bf16_pair(l[2], l[3]);
            const uint32_t c2l = pack_bf16_pair(l[4], l[5]), c3l = pack_bf16_pair(l[6], l[7]);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                mma_bf16(acc[mt][nt], a0, a1, a2, a3, bx[nt]);
                mma_bf16(acc[mt][nt], c0l, c1l, c2l, c3l, bx[nt]);
            }
            mma_bf16(acc[mt][4], a0, a1, a2, a3, bones);
            mma_bf16(acc[mt][4], c0l, c1l, c2l, c3l, bones);
        }
    }
    // fragment (mt, nt): e = 0, 1: row 16 mt + gq, column 8 nt + 2t + e;
    // e = 2, 3: row 16 mt + gq + 8; the bias sits in column 0 of n-tile 4
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                atomicAdd(&red[16 * mt + gq + 8 * (e >> 1)][8 * nt + 2 * t + (e & 1)], acc[mt][nt][e]);
        if (t == 0) {
            atomicAdd(&red[16 * mt + gq][32], acc[mt][4][0]);
            atomicAdd(&red[16 * mt + gq + 8][32], acc[mt][4][2]);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 32 * 32; k += blockDim.x) atomicAdd(&gW[(int64_t)(o0 + k / 32) * 32 + k % 32], red[k / 32][k % 32]);
    for (int k = threadIdx.x; k < 32; k += blockDim.x) atomicAdd(&gb[o0 + k], red[k][32]);
}

// Complex DFT along the rows of a slab on tensor cores, for the y stages of
// the transforms in the BF16-activation configuration:
//   Y[s][i][jx] = sum_j W(i, j) X[s][j][jx],   W(i, j) = tw[j * Ky + i]        (forward: i = ky, j = y)
//                                                W(i, j) = conj(tw[i * Ky + j])  (inverse: i = y, j = ky)
// as the real product [Re Y; Im Y] = [[Wr, -Wi], [Wi, Wr]] [Re X; Im X]
// with m16n8k16 BF16 operands and FP32 accumulation.  An m-tile is eight
// outputs i: rows g take the real part of output 8 mt + g, rows g + 8 its
// imaginary part.  A k-step is eight inputs j, the contraction index
// running (j, re), (j, im) so that a lane's B register pair is one float2
// X[s][j][jx] (j = 8 ks + t and 8 ks + t + 4, jx = 8 nt + g).  Both operands
// enter as BF16 hi + lo pairs (three products per tile, about 2^-16 relative
// error, as in the x stages).  One warp per slab; the twiddle fragments of
// every (m-tile, k-step) are built once per block in shared memory.
template <int NT>
__global__ void __launch_bounds__(TPB) k_cdft_tc(const float2 *X, float2 *Y, const float2 *tw, int Ky, int inv,
                                                 int I, int J, int64_t S)
{
    extern __shared__ uint4 af[];                        // [hi, lo][MT * KS * 32]
    constexpr int KX = NT * 8;
    const int MT = I / 8, KS = J / 8, nf = MT * KS * 32;
    for (int idx = threadIdx.x; idx < nf; idx += blockDim.x) {
        const int mt = idx / (KS * 32), ks = (idx / 32) % KS, l = idx & 31, g = l >> 2, t = l & 3;
        const int i = 8 * mt + g;
        float2 w[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 8 * ks + t + 4 * h;
            const float2 v = inv ? tw[i * Ky + j] : tw[j * Ky + i];
            w[h] = inv ? make_float2(v.x, -v.y) : v;
        }
        // a0 = (Wr, -Wi), a1 = (Wi, Wr) of j = 8 ks + t; a2, a3 the same of j + 4
        const float e[8] = {w[0].x, -w[0].y, w[0].y, w[0].x, w[1].x, -w[1].y, w[1].y, w[1].x};
        __nv_bfloat16 hh[8], ll[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) split_bf16(e[q], hh[q], ll[q]);
        af[idx] = make_uint4(pack_bf16_pair(hh[0], hh[1]), pack_bf16_pair(hh[2], hh[3]), pack_bf16_pair(hh[4], hh[5]),
                             pack_bf16_pair(hh[6], hh[7]));
        af[nf + idx] = make_uint4(pack_bf16_pair(ll[0], ll[1]), pack_bf16_pair(ll[2], ll[3]),
                                  pack_bf16_pair(ll[4], ll[5]), pack_bf16_pair(ll[6], ll[7]));
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int64_t s = (int64_t)blockIdx.x * (TPB / 32) + warp; s < S; s += (int64_t)gridDim.x * (TPB / 32)) {
        const float2 *xs = X + s * J * KX;
        float2 *ys = Y + s * I * KX;
        for (int mt = 0; mt < MT; ++mt) {
            float acc[NT][4];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
            for (int ks = 0; ks < KS; ++ks) {
                const uint4 ah = af[(mt * KS + ks) * 32 + lane], al = af[nf + (mt * KS + ks) * 32 + lane];
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const float2 x0 = xs[(8 * ks + t) * KX + 8 * nt + g];
                    const float2 x1 = xs[(8 * ks + t + 4) * KX + 8 * nt + g];
                    __nv_bfloat16 h0, l0, h1, l1, h2, l2, h3, l3;
                    split_bf16(x0.x, h0, l0); split_bf16(x0.y, h1, l1);
                    split_bf16(x1.x, h2, l2); split_bf16(x1.y, h3, l3);
                    const uint2 bh = make_uint2(pack_bf16_pair(h0, h1), pack_bf16_pair(h2, h3));
                    const uint2 bl = make_uint2(pack_bf16_pair(l0, l1), pack_bf16_pair(l2, l3));
                    mma_bf16(acc[nt], ah.x, ah.y, ah.z, ah.w, bh);
                    mma_bf16(acc[nt], ah.x, ah.y, ah.z, ah.w, bl);
                    mma_bf16(acc[nt], al.x, al.y, al.z, al.w, bh);
                }
            }
            // d0, d1: Re of output 8 mt + g at jx = 8 nt + 2t, +1; d2, d3: Im
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
                *reinterpret_cast<float4 *>(ys + (int64_t)(8 * mt + g) * KX + 8 * nt + 2 * t) =
                    make_float4(acc[nt][0], acc[nt][2], acc[nt][1], acc[nt][3]);
        }
    }
}

// Fourier-layer output in one pass, for BF16 activations, nx = 128, 32
// retained x modes and width 32.  For a line (b, z, y) of 128 cells a warp
// computes, for all 32 output channels o,
//   pre[o][x] = sum_j It[(b, o, z, y)][j] T[j][x]  +  sum_c W[o][c] v[c][x]  +  bias[o]
//   out[o][x] = act(pre[o][x])
// i.e. the inverse x stage of the spectral branch (the contraction of
// k_dftx_inv_tc: It rows and the twiddle table as BF16 hi + lo pairs, three
// products per tile) and the pointwise path (W as hi + lo pairs against the
// exact BF16 inputs, two products per tile) accumulated in the same m16n8
// fragments, so that the spectral branch never goes through memory.  The
// inputs v of the line (32 channels x 128 cells, 8 KB) are staged in shared
// memory with 16-byte loads and read back as B fragments by
// ldmatrix.trans; rows are 256 bytes and their 16-byte chunks are XOR-
// swizzled by (row % 8) so that those reads hit distinct banks.  Outputs go
// through a 16-row staging tile, written row by row with 16-byte stores.
// A warp takes the 16 output channels of one m-tile at a time (64 FP32
// accumulators).
constexpr int FUSE_WARPS = 4;
constexpr int FUSE_C = 32;
constexpr size_t FUSE_SMEM = sizeof(uint2) * 2 * 4 * 16 * 32     // twiddle fragments, hi and lo
                           + sizeof(uint4) * 2 * 2 * 2 * 32      // W fragments [hi/lo][mt][ks][lane]
                           + sizeof(float) * FUSE_C              // bias
                           + (size_t)FUSE_WARPS * (FUSE_C * TCX_NX * 2 + 16 * TCX_NX * 2);   // v and out tiles

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// byte offset of element (row, x) in a 256-byte-row tile with swizzled chunks
__device__ __forceinline__ int swz(int row, int x) { return row * 256 + ((((x >> 3) ^ (row & 7)) & 15) << 4) + (x & 7) * 2; }

__global__ void __launch_bounds__(FUSE_WARPS * 32, 2) k_layer_tc(const float2 *It, const __nv_bfloat16 *v,
                                                               const float *W, const float *bias, const float2 *twx,
                                                               __nv_bfloat16 *pre, __nv_bfloat16 *out, int act,
                                                               int64_t lines_per_sample, int64_t N, int B)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    uint2 *bt = reinterpret_cast<uint2 *>(fsm);                          // [2][4 * 16 * 32]
    uint4 *wa = reinterpret_cast<uint4 *>(fsm + sizeof(uint2) * 2 * 4 * 16 * 32);   // [2][2][2][32]
    float *sb = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(wa) + sizeof(uint4) * 2 * 2 * 2 * 32);
    unsigned char *tiles = reinterpret_cast<unsigned char *>(sb + FUSE_C);
    constexpr int BT = 4 * 16 * 32;
    for (int idx = threadIdx.x; idx < BT; idx += blockDim.x) {
        const int st = idx >> 9, nt = (idx >> 5) & 15, l = idx & 31;
        const int xs = 8 * nt + (l >> 2), c = l & 3;
        __nv_bfloat16 h[4], o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = 16 * c + 4 * st + e;
            const float2 t = twx[xs * TCX_KX + (k >> 1)];
            split_bf16((k & 1) ? t.y : t.x, h[e], o[e]);
        }
        bt[idx] = make_uint2(pack_bf16_pair(h[0], h[1]), pack_bf16_pair(h[2], h[3]));
        bt[BT + idx] = make_uint2(pack_bf16_pair(o[0], o[1]), pack_bf16_pair(o[2], o[3]));
    }
    for (int idx = threadIdx.x; idx < 2 * 2 * 32; idx += blockDim.x) {
        const int mt = idx >> 6, ks = (idx >> 5) & 1, l = idx & 31, g = l >> 2, c = l & 3;
        const int r0 = 16 * mt + g, r1 = r0 + 8;
        const int k0 = 16 * ks + 2 * c, k2 = k0 + 8;
        const float w[8] = {W[r0 * FUSE_C + k0], W[r0 * FUSE_C + k0 + 1], W[r1 * FUSE_C + k0], W[r1 * FUSE_C + k0 + 1],
                            W[r0 * FUSE_C + k2], W[r0 * FUSE_C + k2 + 1], W[r1 * FUSE_C + k2], W[r1 * FUSE_C + k2 + 1]};
        __nv_bfloat16 h[8], o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) split_bf16(w[e], h[e], o[e]);
        wa[idx] = make_uint4(pack_bf16_pair(h[0], h[1]), pack_bf16_pair(h[2], h[3]), pack_bf16_pair(h[4], h[5]),
                             pack_bf16_pair(h[6], h[7]));
        wa[2 * 2 * 32 + idx] = make_uint4(pack_bf16_pair(o[0], o[1]), pack_bf16_pair(o[2], o[3]),
                                          pack_bf16_pair(o[4], o[5]), pack_bf16_pair(o[6], o[7]));
    }
    for (int k = threadIdx.x; k < FUSE_C; k += blockDim.x) sb[k] = bias[k];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    unsigned char *vt = tiles + (size_t)warp * (FUSE_C * TCX_NX * 2 + 16 * TCX_NX * 2);
    unsigned char *ot = vt + FUSE_C * TCX_NX * 2;
    const int64_t lines = (int64_t)B * lines_per_sample;
    for (int64_t line = (int64_t)blockIdx.x * FUSE_WARPS + warp; line < lines; line += (int64_t)gridDim.x * FUSE_WARPS) {
        const int64_t b = line / lines_per_sample, zy = line - b * lines_per_sample;
        const int64_t off = zy * TCX_NX;                        // cell of x = 0 within a channel plane
        // stage v[b][0..31][line][0..127] (16 bytes per lane and step)
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int row = 2 * i + (lane >> 4), ch = lane & 15;
            const uint4 q = *reinterpret_cast<const uint4 *>(v + ((b * FUSE_C + row) * N + off) + ch * 8);
            *reinterpret_cast<uint4 *>(vt + swz(row, ch * 8)) = q;
        }
        __syncwarp();
#pragma unroll 1
        for (int mt = 0; mt < 2; ++mt) {
            float acc[16][4];
#pragma unroll
            for (int nt = 0; nt < 16; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
            // pointwise path: W (hi + lo) times the exact BF16 inputs
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint4 ah = wa[(mt * 2 + ks) * 32 + lane], al = wa[2 * 2 * 32 + (mt * 2 + ks) * 32 + lane];
                const int row = 16 * ks + (lane & 7) + 8 * ((lane >> 3) & 1);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4_trans(smem_u32(vt + swz(row, 8 * (2 * j + (lane >> 4)))), b0, b1, b2, b3);
                    mma_bf16(acc[2 * j], ah.x, ah.y, ah.z, ah.w, make_uint2(b0, b1));
                    mma_bf16(acc[2 * j], al.x, al.y, al.z, al.w, make_uint2(b0, b1));
                    mma_bf16(acc[2 * j + 1], ah.x, ah.y, ah.z, ah.w, make_uint2(b2, b3));
                    mma_bf16(acc[2 * j + 1], al.x, al.y, al.z, al.w, make_uint2(b2, b3));
                }
            }
            // spectral branch: inverse x transform of the rows of channels
            // 16 mt + g and 16 mt + g + 8
            const int64_t ra = (b * FUSE_C + 16 * mt + g) * lines_per_sample + zy;
            const int64_t rb = ra + 8 * lines_per_sample;
            const float4 *pa = reinterpret_cast<const float4 *>(It + ra * TCX_KX) + 4 * c;
            const float4 *pb = reinterpret_cast<const float4 *>(It + rb * TCX_KX) + 4 * c;
            float4 va[4], vb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                va[q] = pa[q];
                vb[q] = pb[q];
            }
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                __nv_bfloat16 ah[8], al[8];
                split_bf16(va[st].x, ah[0], al[0]); split_bf16(va[st].y, ah[1], al[1]);
                split_bf16(va[st].z, ah[2], al[2]); split_bf16(va[st].w, ah[3], al[3]);
                split_bf16(vb[st].x, ah[4], al[4]); split_bf16(vb[st].y, ah[5], al[5]);
                split_bf16(vb[st].z, ah[6], al[6]); split_bf16(vb[st].w, ah[7], al[7]);
                const uint32_t h0 = pack_bf16_pair(ah[0], ah[1]), h2 = pack_bf16_pair(ah[2], ah[3]);
                const uint32_t h1 = pack_bf16_pair(ah[4], ah[5]), h3 = pack_bf16_pair(ah[6], ah[7]);
                const uint32_t l0 = pack_bf16_pair(al[0], al[1]), l2 = pack_bf16_pair(al[2], al[3]);
                const uint32_t l1 = pack_bf16_pair(al[4], al[5]), l3 = pack_bf16_pair(al[6], al[7]);
#pragma unroll
                for (int nt = 0; nt < 16; ++nt) {
                    const uint2 bh = bt[(st * 16 + nt) * 32 + lane];
                    const uint2 bl = bt[BT + (st * 16 + nt) * 32 + lane];
                    mma_bf16(acc[nt], h0, h1, h2, h3, bh);
                    mma_bf16(acc[nt], h0, h1, h2, h3, bl);
                    mma_bf16(acc[nt], l0, l1, l2, l3, bh);
                }
            }
            // epilogue: element e of n-tile nt is output 16 mt + g + 8 (e >> 1)
            // (local row g + 8 (e >> 1)) at x = 8 nt + 2c + (e & 1)
#pragma unroll
            for (int nt = 0; nt < 16; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = g + 8 * h;
                    const float bb = sb[16 * mt + r];
                    acc[nt][2 * h] += bb;
                    acc[nt][2 * h + 1] += bb;
                    float k0, k1;
                    const float y0 = act_fwd<true>(act, 0.f, acc[nt][2 * h], k0);
                    const float y1 = act_fwd<true>(act, 0.f, acc[nt][2 * h + 1], k1);
                    *reinterpret_cast<__nv_bfloat162 *>(ot + swz(r, 8 * nt + 2 * c)) = __floats2bfloat162_rn(y0, y1);
                }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int row = 2 * i + (lane >> 4), ch = lane & 15;
                *reinterpret_cast<uint4 *>(out + ((b * FUSE_C + 16 * mt + row) * N + off) + ch * 8) =
                    *reinterpret_cast<const uint4 *>(ot + swz(row, ch * 8));
            }
            __syncwarp();
            if (pre) {
#pragma unroll
                for (int nt = 0; nt < 16; ++nt)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        *reinterpret_cast<__nv_bfloat162 *>(ot + swz(g + 8 * h, 8 * nt + 2 * c)) =
                            __floats2bfloat162_rn(acc[nt][2 * h], acc[nt][2 * h + 1]);
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int row = 2 * i + (lane >> 4), ch = lane & 15;
                    *reinterpret_cast<uint4 *>(pre + ((b * FUSE_C + 16 * mt + row) * N + off) + ch * 8) =
                        *reinterpret_cast<const uint4 *>(ot + swz(row, ch * 8));
                }
                __syncwarp();
            }
        }
        __syncwarp();
    }
}

// Inference projection y = Q2 sin(omega0 (Q1 v + b1)) + b2 on tensor cores, for
// BF16 activations with 32 channels, 128 hidden units and co <= 8 outputs:
// a warp takes 16 cells of one sample per pass.  First product: cells x
// channels (BF16, exact) times Q1^T (BF16 hi + lo pairs, two products per
// tile), 16 x 128 FP32 accumulators; bias and the sine on the accumulators,
// which then serve directly as the A fragments of the second product (two
// adjacent n8 tiles of the first are one k16 step of the second), split into
// hi + lo; second product against Q2^T (hi + lo; three products per step),
// 16 x 8 outputs.  The hidden activations never leave registers.  The
// channels of a cell are planes N apart, so each lane gathers its sixteen
// BF16 inputs with 2-byte loads (a warp instruction covers 8 consecutive
// cells of 4 channels).
constexpr int PTC_CI = 32, PTC_H = 128;

__global__ void __launch_bounds__(TPB, 2) k_proj_tc(const __nv_bfloat16 *v, int co, const float *W1, const float *b1,
                                                 const float *W2, const float *b2, float w0, float *y, int64_t N,
                                                 int B)
{
    __shared__ uint2 q1[2][2 * 16 * 32];    // [hi, lo][(k-step * 16 + n-tile) * 32 + lane]
    __shared__ uint2 q2[2][8 * 32];         // [hi, lo][k-step * 32 + lane]
    __shared__ float sb1[PTC_H], sb2[8];
    for (int idx = threadIdx.x; idx < 2 * 16 * 32; idx += blockDim.x) {
        const int st = idx >> 9, nt = (idx >> 5) & 15, l = idx & 31;
        const int hh = 8 * nt + (l >> 2), c = l & 3;
        const int ks[4] = {16 * st + 2 * c, 16 * st + 2 * c + 1, 16 * st + 2 * c + 8, 16 * st + 2 * c + 9};
        __nv_bfloat16 h[4], o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_bf16(W1[hh * PTC_CI + ks[e]], h[e], o[e]);
        q1[0][idx] = make_uint2(pack_bf16_pair(h[0], h[1]), pack_bf16_pair(h[2], h[3]));
        q1[1][idx] = make_uint2(pack_bf16_pair(o[0], o[1]), pack_bf16_pair(o[2], o[3]));
    }
    for (int idx = threadIdx.x; idx < 8 * 32; idx += blockDim.x) {
        const int st = idx >> 5, l = idx & 31;
        const int oo = l >> 2, c = l & 3;
        const int ks[4] = {16 * st + 2 * c, 16 * st + 2 * c + 1, 16 * st + 2 * c + 8, 16 * st + 2 * c + 9};
        __nv_bfloat16 h[4], o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_bf16(oo < co ? W2[oo * PTC_H + ks[e]] : 0.f, h[e], o[e]);
        q2[0][idx] = make_uint2(pack_bf16_pair(h[0], h[1]), pack_bf16_pair(h[2], h[3]));
        q2[1][idx] = make_uint2(pack_bf16_pair(o[0], o[1]), pack_bf16_pair(o[2], o[3]));
    }
    for (int k = threadIdx.x; k < PTC_H; k += blockDim.x) sb1[k] = b1[k];
    if (threadIdx.x < 8) sb2[threadIdx.x] = threadIdx.x < co ? b2[threadIdx.x] : 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const int64_t tpb = N / 16, tiles = (int64_t)B * tpb;
    const unsigned short *vs = reinterpret_cast<const unsigned short *>(v);
    for (int64_t tile = (int64_t)blockIdx.x * (TPB / 32) + warp; tile < tiles; tile += (int64_t)gridDim.x * (TPB / 32)) {
        const int64_t b = tile / tpb, n0 = (tile - b * tpb) * 16;
        const unsigned short *base = vs + b * PTC_CI * N + n0 + g;
        // A of the first product: (cell g | g + 8, channel pairs 2c, 2c + 1 and 2c + 8, 2c + 9 of each k-step)
        uint32_t a[2][4];
#pragma unroll
        for (int st = 0; st < 2; ++st) {
            const int ch = 16 * st + 2 * c;
            const unsigned short *p0 = base + (int64_t)ch * N, *p1 = p0 + N, *p8 = p0 + 8 * N, *p9 = p0 + 9 * N;
            a[st][0] = (uint32_t)p0[0] | ((uint32_t)p1[0] << 16);
            a[st][1] = (uint32_t)p0[8] | ((uint32_t)p1[8] << 16);
            a[st][2] = (uint32_t)p8[0] | ((uint32_t)p9[0] << 16);
            a[st][3] = (uint32_t)p8[8] | ((uint32_t)p9[8] << 16);
        }
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
        for (int st = 0; st < 2; ++st)
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                mma_bf16(acc[nt], a[st][0], a[st][1], a[st][2], a[st][3], q1[0][(st * 16 + nt) * 32 + lane]);
                mma_bf16(acc[nt], a[st][0], a[st][1], a[st][2], a[st][3], q1[1][(st * 16 + nt) * 32 + lane]);
            }
        // hidden units 8 nt + 2c + {0, 1} of cells g and g + 8
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const float c0 = sb1[8 * nt + 2 * c], c1 = sb1[8 * nt + 2 * c + 1];
            acc[nt][0] = __sinf(w0 * (acc[nt][0] + c0));
            acc[nt][1] = __sinf(w0 * (acc[nt][1] + c1));
            acc[nt][2] = __sinf(w0 * (acc[nt][2] + c0));
            acc[nt][3] = __sinf(w0 * (acc[nt][3] + c1));
        }
        float out[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int s2 = 0; s2 < 8; ++s2) {
            const float *lo_t = acc[2 * s2], *hi_t = acc[2 * s2 + 1];
            __nv_bfloat16 h[8], o[8];
            split_bf16(lo_t[0], h[0], o[0]); split_bf16(lo_t[1], h[1], o[1]);
            split_bf16(lo_t[2], h[2], o[2]); split_bf16(lo_t[3], h[3], o[3]);
            split_bf16(hi_t[0], h[4], o[4]); split_bf16(hi_t[1], h[5], o[5]);
            split_bf16(hi_t[2], h[6], o[6]); split_bf16(hi_t[3], h[7], o[7]);
            // a0: (cell g, k 2c, 2c+1), a1: (cell g+8, same), a2: (cell g, k 2c+8, +9), a3: (cell g+8, same)
            const uint32_t h0 = pack_bf16_pair(h[0], h[1]), h1 = pack_bf16_pair(h[2], h[3]);
            const uint32_t h2 = pack_bf16_pair(h[4], h[5]), h3 = pack_bf16_pair(h[6], h[7]);
            const uint32_t l0 = pack_bf16_pair(o[0], o[1]), l1 = pack_bf16_pair(o[2], o[3]);
            const uint32_t l2 = pack_bf16_pair(o[4], o[5]), l3 = pack_bf16_pair(o[6], o[7]);
            const uint2 bh = q2[0][s2 * 32 + lane], bl = q2[1][s2 * 32 + lane];
            mma_bf16(out, h0, h1, h2, h3, bh);
            mma_bf16(out, h0, h1, h2, h3, bl);
            mma_bf16(out, l0, l1, l2, l3, bh);
        }
        // outputs 2c, 2c + 1 of cells g (out[0], out[1]) and g + 8 (out[2], out[3])
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int o = 2 * c + (e & 1);
            const int64_t n = n0 + g + (e >> 1) * 8;
            if (o < co) y[(b * co + o) * N + n] = out[e] + sb2[o];
        }
    }
}

// Pointwise layer y = act(W x + b + extra) on tensor cores for BF16
// activations with 32 inputs and CO outputs (used for CO = 128): a warp takes 16
// cells of one sample per pass; cells x inputs (BF16, exact, gathered as in
// k_proj_tc) times W^T (BF16 hi + lo pairs, two products per tile), FP32
// accumulators, then bias, the extra (spectral) term, the stored
// pre-activation and the activation per element.
template <int CO>
__global__ void __launch_bounds__(TPB) k_pw_tc(const __nv_bfloat16 *x, const float *W, const float *bias,
                                               const float *extra, __nv_bfloat16 *pre, __nv_bfloat16 *y, int act,
                                               float w0, int64_t N, int B)
{
    constexpr int NT = CO / 8;
    __shared__ uint2 q[2][2 * NT * 32];     // [hi, lo][(k-step * NT + n-tile) * 32 + lane]
    __shared__ float sb[CO];
    for (int idx = threadIdx.x; idx < 2 * NT * 32; idx += blockDim.x) {
        const int st = idx / (NT * 32), nt = (idx / 32) % NT, l = idx & 31;
        const int o = 8 * nt + (l >> 2), c = l & 3;
        const int ks[4] = {16 * st + 2 * c, 16 * st + 2 * c + 1, 16 * st + 2 * c + 8, 16 * st + 2 * c + 9};
        __nv_bfloat16 h[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_bf16(W[o * PTC_CI + ks[e]], h[e], lo[e]);
        q[0][idx] = make_uint2(pack_bf16_pair(h[0], h[1]), pack_bf16_pair(h[2], h[3]));
        q[1][idx] = make_uint2(pack_bf16_pair(lo[0], lo[1]), pack_bf16_pair(lo[2], lo[3]));
    }
    for (int k = threadIdx.x; k < CO; k += blockDim.x) sb[k] = bias[k];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const int64_t tpb = N / 16, tiles = (int64_t)B * tpb;
    const unsigned short *xs = reinterpret_cast<const unsigned short *>(x);
    for (int64_t tile = (int64_t)blockIdx.x * (TPB / 32) + warp; tile < tiles; tile += (int64_t)gridDim.x * (TPB / 32)) {
        const int64_t b = tile / tpb, n0 = (tile - b * tpb) * 16;
        const unsigned short *base = xs + b * PTC_CI * N + n0 + g;
        uint32_t a[2][4];
#pragma unroll
        for (int st = 0; st < 2; ++st) {
            const unsigned short *p0 = base + (int64_t)(16 * st + 2 * c) * N, *p1 = p0 + N, *p8 = p0 + 8 * N,
                                 *p9 = p0 + 9 * N;
            a[st][0] = (uint32_t)p0[0] | ((uint32_t)p1[0] << 16);
            a[st][1] = (uint32_t)p0[8] | ((uint32_t)p1[8] << 16);
            a[st][2] = (uint32_t)p8[0] | ((uint32_t)p9[0] << 16);
            a[st][3] = (uint32_t)p8[8] | ((uint32_t)p9[8] << 16);
        }
        float acc[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
        for (int st = 0; st < 2; ++st)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                mma_bf16(acc[nt], a[st][0], a[st][1], a[st][2], a[st][3], q[0][(st * NT + nt) * 32 + lane]);
                mma_bf16(acc[nt], a[st][0], a[st][1], a[st][2], a[st][3], q[1][(st * NT + nt) * 32 + lane]);
            }
        // element e of n-tile nt: output 8 nt + 2c + (e & 1) of cell g + 8 (e >> 1)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int o = 8 * nt + 2 * c + (e & 1);
                const int64_t off = (b * CO + o) * N + n0 + g + 8 * (e >> 1);
                float v = acc[nt][e] + sb[o];
                if (extra) v += extra[off];
                float keep;
                const float out = act_fwd<true>(act, w0, v, keep);
                if (pre) pre[off] = __float2bfloat16_rn(keep);
                y[off] = __float2bfloat16_rn(out);
            }
    }
}

// ---------------------------------------------------------------------------
// mode contraction.  Forward: G[k][b][o] = sum_i V[k][b][i] R[k][i][o];
// adjoint: gV[k][b][i] = sum_o gG[k][b][o] conj(R[k][i][o]).
// ---------------------------------------------------------------------------
// Real form of one mode's matrix (rows: outputs re then im; cols: inputs re
// then im).
template <bool ADJ>
__device__ __forceinline__ float real_form(const float2 *Rk, int C, int r, int j)
{
    const int ro = r % C, jo = j % C;
    const bool rim = r >= C, jim = j >= C;
    if (!ADJ) {                 // out o = ro, in i = jo: R[i][o]
        const float2 w = Rk[jo * C + ro];
        return !rim ? (!jim ? w.x : -w.y) : (!jim ? w.y : w.x);
    } else {                    // out i = ro, in o = jo: conj(R[i][o])
        const float2 w = Rk[ro * C + jo];
        return !rim ? (!jim ? w.x : w.y) : (!jim ? -w.y : w.x);
    }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// One warp per mode, batch in groups of 8 (the n8 dimension); rows and
// columns of the real form are 2C (C % 8 == 0, so tiles of 16 divide them).
template <bool ADJ>
__global__ void __launch_bounds__(TPB) k_contract_tc(const float2 *Vin, const float2 *R, float2 *Gout, int C, int B,
                                                     int64_t K)
{
    const int lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int M = 2 * C;
    for (int64_t k = warp; k < K; k += nwarps) {
        const float2 *Rk = R + k * C * C;
        for (int b0 = 0; b0 < B; b0 += 8) {
            const int bcol = b0 + gid;                  // batch column this lane feeds in B fragments
            const float2 *Vk = Vin + (k * B) * C;
            for (int mt = 0; mt < M / 16; ++mt) {
                float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
                const int r0 = mt * 16 + gid, r1 = r0 + 8;
                for (int kt = 0; kt < M / 16; ++kt) {
                    const int j0 = kt * 16 + tig * 2;
                    const uint32_t a0 = pack_bf16(real_form<ADJ>(Rk, C, r0, j0), real_form<ADJ>(Rk, C, r0, j0 + 1));
                    const uint32_t a1 = pack_bf16(real_form<ADJ>(Rk, C, r1, j0), real_form<ADJ>(Rk, C, r1, j0 + 1));
                    const uint32_t a2 = pack_bf16(real_form<ADJ>(Rk, C, r0, j0 + 8), real_form<ADJ>(Rk, C, r0, j0 + 9));
                    const uint32_t a3 = pack_bf16(real_form<ADJ>(Rk, C, r1, j0 + 8), real_form<ADJ>(Rk, C, r1, j0 + 9));
                    float bv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = j0 + (q & 1) + (q >> 1) * 8;
                        float v = 0.f;
                        if (bcol < B) {
                            const float2 z = Vk[(int64_t)bcol * C + (j % C)];
                            v = j < C ? z.x : z.y;
                        }
                        bv[q] = v;
                    }
                    const uint32_t b0r = pack_bf16(bv[0], bv[1]);
                    const uint32_t b1r = pack_bf16(bv[2], bv[3]);
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
                        : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0r), "r"(b1r));
                }
                // D: (row gid, cols 2tig, 2tig+1), (row gid + 8, same cols)
                const float dv[4] = {c0, c1, c2, c3};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = (q < 2) ? r0 : r1;
                    const int b = b0 + tig * 2 + (q & 1);
                    if (b < B) {
                        float *dst = reinterpret_cast<float *>(Gout + (k * B + b) * C + (r % C));
                        dst[r >= C ? 1 : 0] = dv[q];
                    }
                }
            }
        }
    }
}

template <bool ADJ>
__global__ void __launch_bounds__(TPB) k_contract_f32(const float2 *Vin, const float2 *R, float2 *Gout, int C, int B,
                                                      int64_t K)
{
    const int64_t total = K * B * C;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / ((int64_t)B * C);
        const int b = (int)((t / C) % B), o = (int)(t % C);
        const float2 *Rk = R + k * C * C;
        const float2 *Vk = Vin + (k * B + b) * C;
        float2 acc = make_float2(0.f, 0.f);
        for (int i = 0; i < C; ++i) {
            const float2 v = !ADJ ? cmul(Vk[i], Rk[i * C + o]) : cmulc(Vk[i], Rk[o * C + i]);
            acc.x += v.x;
            acc.y += v.y;
        }
        Gout[t] = acc;
    }
}

// gR[k][i][o] = sum_b gG[k][b][o] conj(V[k][b][i])
__global__ void __launch_bounds__(TPB) k_grad_R(const float2 *gG, const float2 *V, float2 *gR, int C, int B, int64_t K)
{
    const int64_t total = K * C * C;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / ((int64_t)C * C);
        const int i = (int)((t / C) % C), o = (int)(t % C);
        float2 acc = make_float2(0.f, 0.f);
        for (int b = 0; b < B; ++b) {
            const float2 v = cmulc(gG[(k * B + b) * C + o], V[(k * B + b) * C + i]);
            acc.x += v.x;
            acc.y += v.y;
        }
        gR[t] = acc;
    }
}

// ---------------------------------------------------------------------------
// loss, conversion, Adam
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TPB) k_mse_partial(const float *y, const float *t, const float *m, int C, int64_t N,
                                                     int B, double *part)
{
    __shared__ double s0[TPB], s1[TPB];
    double a = 0, w = 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / N, n = idx - b * N;
        const float mv = m[idx];
        w += mv;
        for (int c = 0; c < C; ++c) {
            const double d = (double)y[(b * C + c) * N + n] - (double)t[(b * C + c) * N + n];
            a += mv * d * d;
        }
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = w;
    __syncthreads();
    for (int h = TPB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) { s0[threadIdx.x] += s0[threadIdx.x + h]; s1[threadIdx.x] += s1[threadIdx.x + h]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = s0[0]; part[2 * blockIdx.x + 1] = s1[0]; }
}

__global__ void k_mse_final(const double *part, int nb, int C, double *res)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0, w = 0;
        for (int k = 0; k < nb; ++k) { a += part[2 * k]; w += part[2 * k + 1]; }
        res[0] = w > 0 ? a / (C * w) : 0.0;             // loss
        res[1] = w > 0 ? 2.0 / (C * w) : 0.0;           // gradient factor
    }
}

__global__ void __launch_bounds__(TPB) k_mse_grad(const float *y, const float *t, const float *m, int C, int64_t N, int B,
                                                  const double *res, float *gy)
{
    const float f = (float)res[1];
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)B * C * N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / ((int64_t)C * N), n = idx % N;
        gy[idx] = f * (y[idx] - t[idx]) * m[b * N + n];
    }
}

template <class T>
__global__ void k_convert(const float *src, T *dst, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        stf(dst + k, src[k]);
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

// shared memory of the transform stages (independent of the batch)
size_t smem_dftx_fwd(const Dims &d)
{
    const size_t npp = ((size_t)d.nx / 2 + 1 + 3) & ~(size_t)3, nxp = ((size_t)d.nx + 3) & ~(size_t)3;
    return sizeof(float2) * npp * d.Kx + sizeof(float) * DFT_ROWS * (2 * npp + nxp);
}
size_t smem_dftx_inv(const Dims &d)
{
    const size_t ldp = (((size_t)d.nx + 1) / 2 + 63) & ~(size_t)63;
    return sizeof(float2) * ((size_t)d.Kx * ldp + (size_t)DFT_ROWS * d.Kx);
}
int dfty_fwd_slabs(const Dims &d) { return std::max(1, (TPB / 32) / ((d.Ky + 7) / 8)); }
int dfty_inv_slabs(const Dims &d) { return std::max(1, (TPB / 32) / ((d.ny + 7) / 8)); }
size_t smem_dfty_fwd(const Dims &d)
{
    const size_t kyp = (d.Ky + 7) & ~7;
    return sizeof(float2) * ((size_t)d.ny * kyp + (size_t)dfty_fwd_slabs(d) * d.ny * d.Kx);
}
size_t smem_dfty_inv(const Dims &d)
{
    const size_t nyp = (d.ny + 7) & ~7;
    return sizeof(float2) * ((size_t)d.Ky * nyp + (size_t)dfty_inv_slabs(d) * d.Ky * d.Kx);
}

bool set_smem_limits(size_t bytes)
{
    const int b = (int)bytes;
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    return cudaFuncSetAttribute(k_dftx_fwd<float>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_dftx_fwd<__nv_bfloat16>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_dftx_inv<float>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_dftx_inv<__nv_bfloat16>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_dfty_fwd, a, b) == cudaSuccess && cudaFuncSetAttribute(k_dfty_inv, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_outer<float, 1>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_outer<float, 2>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_outer<__nv_bfloat16, 1>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_outer<__nv_bfloat16, 2>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_outer_async<float, 1>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_outer_async<float, 2>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_outer_async<__nv_bfloat16, 1>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_outer_async<__nv_bfloat16, 2>, a, b) == cudaSuccess &&
           cudaFuncSetAttribute(k_layer_tc, a, (int)FUSE_SMEM) == cudaSuccess;
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

thread_local std::string g_fno_err;

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct fno_ctx {
    fno_config c{};
    cudaStream_t s = nullptr;
    int64_t N = 0, K = 0, np = 0;
    int Kx = 0, Ky = 0, Kz = 0;
    // parameter offsets in the flat vector
    int64_t oP1_w = 0, oP1_b = 0, oP2_w = 0, oP2_b = 0, oQ1_w = 0, oQ1_b = 0, oQ2_w = 0, oQ2_b = 0;
    std::vector<int64_t> oR, oW_w, oW_b;
    float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
    int64_t adam_t = 0;
    // device buffers
    std::vector<void *> allocs;
    void *xa = nullptr;                       // converted input (act type)
    std::vector<void *> v, pre;               // activations
    void *apre = nullptr, *a = nullptr;       // lift hidden layer: pre-activation, GELU output
    void *hcos = nullptr, *h = nullptr;       // SIREN hidden layer: cos(omega0 z), sin(omega0 z)
    float *y = nullptr, *spec = nullptr, *gy = nullptr, *ghpre = nullptr, *gA = nullptr, *gB = nullptr;
    float *xin = nullptr, *tin = nullptr, *min = nullptr;
    float2 *stA = nullptr, *stB = nullptr;    // DFT stage temporaries
    std::vector<float2 *> Vh;                 // per-layer spectra of the layer inputs
    float2 *G = nullptr, *gG = nullptr, *gVh = nullptr;
    float2 *twx = nullptr, *twy = nullptr, *twz = nullptr;
    float *scale_one = nullptr, *scale_inv = nullptr;
    double *part = nullptr, *res = nullptr;
    int nparts = 0;
    // tcgen05 forward x stage: one tensor map per layer input buffer, status word
    std::vector<std::vector<unsigned char>> vmaps;
    int *ustatus = nullptr;
    std::string err;
    int last_batch = 0;

    size_t es() const { return c.act_bf16 ? 2 : 4; }
    template <class T> T *alloc(size_t count)
    {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 16)) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        return static_cast<T *>(p);
    }
};

#define FCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            f->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return LBM_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)

extern "C" void fno_config_default(fno_config *c)
{
    std::memset(c, 0, sizeof(*c));
    c->nx = 128; c->ny = 64; c->nz = 64;
    c->cin = 4; c->width = 32; c->cout = 4;
    c->mx = 16; c->my = 8; c->mz = 8;
    c->layers = 4; c->hidden = 128;
    c->max_batch = 8;
    c->act_bf16 = 1;
    c->tensor_cores = 1;
    c->lift_hidden = 32;
    c->omega0 = 30.f;
    c->seed = 0;
}

// SplitMix64 (Steele, Lea & Flood 2014) for the initial parameters.
static uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double unif(uint64_t &s) { return 2.0 * ((splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) - 1.0; }

extern "C" lbm_status fno_destroy(fno_ctx *f)
{
    if (!f) return LBM_ERR_ARG;
    if (f->s) cudaStreamSynchronize(f->s);
    for (void *p : f->allocs) cudaFree(p);
    delete f;
    return LBM_OK;
}

extern "C" lbm_status fno_create(const fno_config *cfg, void *stream, fno_ctx **out)
{
    if (!out || !cfg) return LBM_ERR_ARG;
    *out = nullptr;
    const fno_config &c = *cfg;
    auto bad = [](const char *m) { g_fno_err = m; return LBM_ERR_ARG; };
    if (c.nx < 2 || c.ny < 2 || c.nz < 2 || c.cin < 1 || c.width < 1 || c.cout < 1 || c.layers < 1 || c.hidden < 1 ||
        c.max_batch < 1)
        return bad("non-positive size");
    if (c.cin > 32 || c.width > 32 || c.cout > 8) return bad("cin and width must be <= 32, cout <= 8");
    if (c.lift_hidden < 1 || c.lift_hidden > 32) return bad("lift_hidden must be in [1, 32]");
    if (!(c.omega0 > 0.f) || !std::isfinite(c.omega0)) return bad("omega0 must be a positive finite number");
    if (c.mx < 1 || c.my < 1 || c.mz < 1 || 2 * c.mx > c.nx || 2 * c.my > c.ny || c.mz >= c.nz / 2 + 1 || c.mz > 16)
        return bad("modes must satisfy 2mx <= nx, 2my <= ny, mz <= nz/2, mz <= 16");
    if (c.tensor_cores && c.width % 8 != 0) return bad("tensor-core contraction needs width % 8 == 0");
    if (2 * c.mx > 256) return bad("2mx must be <= 256");
    const Dims d0{c.nx, c.ny, c.nz, 2 * c.mx, 2 * c.my, c.mz, 1};
    const size_t sm_max = 160 * 1024;
    if (smem_dftx_fwd(d0) > sm_max || smem_dftx_inv(d0) > sm_max || smem_dfty_fwd(d0) > sm_max ||
        smem_dfty_inv(d0) > sm_max)
        return bad("grid x modes too large for the shared-memory twiddle tables");
    if (outer_units(c.hidden, c.width) > 2 * TPB || outer_units(c.cout, c.hidden) > 2 * TPB ||
        outer_units(c.width, c.width) > 2 * TPB || outer_units(c.width, c.lift_hidden) > 2 * TPB ||
        outer_units(c.lift_hidden, c.cin) > 2 * TPB)
        return bad("layer too wide for the gradient reduction");
    if (smem_outer(c.hidden, c.width) > sm_max || smem_outer(c.cout, c.hidden) > sm_max)
        return bad("layer too wide for the gradient reduction tiles");
    if (!set_smem_limits(sm_max)) return bad("cannot raise the shared-memory limit of the FNO kernels");
    fno_ctx *f = new fno_ctx();
    f->c = c;
    f->s = static_cast<cudaStream_t>(stream);
    f->N = (int64_t)c.nx * c.ny * c.nz;
    f->Kx = 2 * c.mx; f->Ky = 2 * c.my; f->Kz = c.mz;
    f->K = (int64_t)f->Kx * f->Ky * f->Kz;
    const int W = c.width, H = c.hidden, LH = c.lift_hidden;
    // spectral weights first: every R_l starts at an even float index, so
    // its complex entries are 8-byte aligned
    int64_t o = 0;
    for (int l = 0; l < c.layers; ++l) { f->oR.push_back(o); o += 2 * f->K * W * W; }
    f->oP1_w = o; o += (int64_t)LH * c.cin;
    f->oP1_b = o; o += LH;
    f->oP2_w = o; o += (int64_t)W * LH;
    f->oP2_b = o; o += W;
    for (int l = 0; l < c.layers; ++l) {
        f->oW_w.push_back(o); o += (int64_t)W * W;
        f->oW_b.push_back(o); o += W;
    }
    f->oQ1_w = o; o += (int64_t)H * W;
    f->oQ1_b = o; o += H;
    f->oQ2_w = o; o += (int64_t)c.cout * H;
    f->oQ2_b = o; o += c.cout;
    f->np = o;
    const int64_t B = c.max_batch, N = f->N, es = f->es();
    bool ok = true;
    auto chk = [&](void *p) { ok = ok && p != nullptr; };
    chk(f->params = f->alloc<float>(o));
    chk(f->grads = f->alloc<float>(o));
    chk(f->m1 = f->alloc<float>(o));
    chk(f->m2 = f->alloc<float>(o));
    chk(f->xa = f->alloc<char>(B * c.cin * N * es));
    for (int l = 0; l <= c.layers; ++l) { void *p = f->alloc<char>(B * W * N * es); chk(p); f->v.push_back(p); }
    for (int l = 0; l < c.layers; ++l) { void *p = f->alloc<char>(B * W * N * es); chk(p); f->pre.push_back(p); }
    chk(f->apre = f->alloc<char>(B * LH * N * es));
    chk(f->a = f->alloc<char>(B * LH * N * es));
    chk(f->hcos = f->alloc<char>(B * H * N * es));
    chk(f->h = f->alloc<char>(B * H * N * es));
    chk(f->y = f->alloc<float>(B * c.cout * N));
    chk(f->spec = f->alloc<float>(B * W * N));
    chk(f->gy = f->alloc<float>(B * c.cout * N));
    chk(f->ghpre = f->alloc<float>(B * H * N));
    chk(f->gA = f->alloc<float>(B * std::max(W, LH) * N));
    chk(f->gB = f->alloc<float>(B * std::max(W, LH) * N));
    chk(f->xin = f->alloc<float>(B * c.cin * N));
    chk(f->tin = f->alloc<float>(B * c.cout * N));
    chk(f->min = f->alloc<float>(B * N));
    const int64_t BC = B * W;
    chk(f->stA = f->alloc<float2>(std::max(BC * c.nz * c.ny * f->Kx, BC * c.nz * c.ny * f->Kx)));
    chk(f->stB = f->alloc<float2>(BC * c.nz * f->Ky * f->Kx));
    for (int l = 0; l < c.layers; ++l) { float2 *p = f->alloc<float2>(f->K * BC); chk(p); f->Vh.push_back(p); }
    chk(f->G = f->alloc<float2>(f->K * BC));
    chk(f->gG = f->alloc<float2>(f->K * BC));
    chk(f->gVh = f->alloc<float2>(f->K * BC));
    chk(f->twx = f->alloc<float2>((int64_t)c.nx * f->Kx));
    chk(f->twy = f->alloc<float2>((int64_t)c.ny * f->Ky));
    chk(f->twz = f->alloc<float2>((int64_t)c.nz * f->Kz));
    chk(f->scale_one = f->alloc<float>(16));
    chk(f->scale_inv = f->alloc<float>(16));
    f->nparts = gb300::sm_count() * 4;
    chk(f->part = f->alloc<double>(2 * f->nparts));
    chk(f->res = f->alloc<double>(2));
    chk(f->ustatus = f->alloc<int>(4));
    if (!ok) {
        g_fno_err = "device allocation failed";
        cudaGetLastError();
        fno_destroy(f);
        return LBM_ERR_OOM;
    }
    // twiddles (double precision angles) and inverse scales
    auto twiddle = [](int n, int K, bool half, float2 *dst_dev, cudaStream_t s) {
        std::vector<float2> t((size_t)n * K);
        for (int xx = 0; xx < n; ++xx)
            for (int j = 0; j < K; ++j) {
                const int k = half ? j : (j < K / 2 ? j : j - K);
                const double a = -2.0 * M_PI * (double)k * xx / n;
                t[(size_t)xx * K + j] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
        return cudaMemcpyAsync(dst_dev, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice, s) == cudaSuccess &&
               cudaStreamSynchronize(s) == cudaSuccess;
    };
    ok = twiddle(c.nx, f->Kx, false, f->twx, f->s) && twiddle(c.ny, f->Ky, false, f->twy, f->s) &&
         twiddle(c.nz, f->Kz, true, f->twz, f->s);
    float one[16], inv[16];
    for (int k = 0; k < 16; ++k) {
        one[k] = 1.f;
        const double ck = (k == 0 || (c.nz % 2 == 0 && k == c.nz / 2)) ? 1.0 : 2.0;
        inv[k] = (float)(ck / (double)N);
    }
    ok = ok && cudaMemcpy(f->scale_one, one, sizeof one, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(f->scale_inv, inv, sizeof inv, cudaMemcpyHostToDevice) == cudaSuccess;
    // initial parameters: uniform within 1/sqrt(fan-in); the SIREN projection
    // as Sitzmann et al. (first layer within 1/fan-in, output layer within
    // sqrt(6/fan-in)/omega0)
    std::vector<float> p0(o);
    uint64_t st = c.seed * 0x9E3779B97F4A7C15ull + 12345;
    auto fill = [&](int64_t off, int64_t cnt, double s) { for (int64_t k = 0; k < cnt; ++k) p0[off + k] = (float)(s * unif(st)); };
    fill(f->oP1_w, (int64_t)LH * c.cin, 1.0 / std::sqrt((double)c.cin));
    fill(f->oP1_b, LH, 1.0 / std::sqrt((double)c.cin));
    fill(f->oP2_w, (int64_t)W * LH, 1.0 / std::sqrt((double)LH));
    fill(f->oP2_b, W, 1.0 / std::sqrt((double)LH));
    for (int l = 0; l < c.layers; ++l) {
        fill(f->oR[l], 2 * f->K * W * W, 1.0 / ((double)W * W));
        fill(f->oW_w[l], (int64_t)W * W, 1.0 / std::sqrt((double)W));
        fill(f->oW_b[l], W, 1.0 / std::sqrt((double)W));
    }
    fill(f->oQ1_w, (int64_t)H * W, 1.0 / (double)W);
    fill(f->oQ1_b, H, 1.0 / std::sqrt((double)W));
    fill(f->oQ2_w, (int64_t)c.cout * H, std::sqrt(6.0 / (double)H) / (double)c.omega0);
    fill(f->oQ2_b, c.cout, 1.0 / std::sqrt((double)H));
    ok = ok && cudaMemcpy(f->params, p0.data(), o * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(f->m1, 0, o * sizeof(float)) == cudaSuccess && cudaMemset(f->m2, 0, o * sizeof(float)) == cudaSuccess &&
         cudaMemset(f->grads, 0, o * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMemset(f->ustatus, 0, 4 * sizeof(int)) == cudaSuccess;
    if (ok && c.umma) {
        // tensor maps of the layer inputs [max_batch * width * nz * ny rows][128]
        if (!(c.act_bf16 && c.nx == 128 && f->Kx == 32) || !umma_set_smem()) {
            g_fno_err = "umma needs BF16 activations, nx = 128 and 32 x modes, and a GPU that supports tcgen05";
            fno_destroy(f);
            return LBM_ERR_ARG;
        }
        const int64_t rows = (int64_t)c.max_batch * W * c.nz * c.ny;
        for (int l = 0; l < c.layers; ++l) {
            std::vector<unsigned char> m(128);
            if (!umma_make_row_map(m.data(), f->v[l], rows)) {
                g_fno_err = "tensor map encoding failed";
                fno_destroy(f);
                return LBM_ERR_CUDA;
            }
            f->vmaps.push_back(m);
        }
    }
    if (!ok) {
        g_fno_err = "initialisation failed";
        cudaGetLastError();
        fno_destroy(f);
        return LBM_ERR_CUDA;
    }
    *out = f;
    return LBM_OK;
}

extern "C" int64_t fno_num_params(const fno_ctx *f) { return f ? f->np : -1; }

extern "C" lbm_status fno_set_params(fno_ctx *f, const float *src)
{
    if (!f || !src) return LBM_ERR_ARG;
    FCK(cudaMemcpyAsync(f->params, src, f->np * sizeof(float), cudaMemcpyDefault, f->s));
    FCK(cudaStreamSynchronize(f->s));
    return LBM_OK;
}

extern "C" lbm_status fno_get_params(fno_ctx *f, float *dst)
{
    if (!f || !dst) return LBM_ERR_ARG;
    FCK(cudaMemcpyAsync(dst, f->params, f->np * sizeof(float), cudaMemcpyDefault, f->s));
    FCK(cudaStreamSynchronize(f->s));
    return LBM_OK;
}

extern "C" lbm_status fno_get_grads(fno_ctx *f, float *dst)
{
    if (!f || !dst) return LBM_ERR_ARG;
    FCK(cudaMemcpyAsync(dst, f->grads, f->np * sizeof(float), cudaMemcpyDefault, f->s));
    FCK(cudaStreamSynchronize(f->s));
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
namespace {

template <class T>
void pw_fwd(fno_ctx *f, const T *x, int ci, int co, int64_t oW, int64_t ob, const float *extra, T *pre, void *y,
            bool y_is_float, int act, int B)
{
    const float w0 = f->c.omega0;
    const bool pairs = f->N % 2 == 0;
    const int64_t units = pairs ? (int64_t)B * f->N / 2 : (int64_t)B * f->N;
    const float *W = f->params + oW, *bias = f->params + ob;
    if (ci <= 32 && !y_is_float) {
        const size_t sm = sizeof(float) * (co * ci + co);
        T *yt = static_cast<T *>(y);
        // 32 -> 128 (the training path of the projection's hidden layer): tensor
        // cores pay off.  32 -> 32 stays on the paired SIMT kernel: there the
        // per-element stores of the fragment layout (2 bytes into 4 channel
        // planes per warp instruction) cost more than the multiply-adds saved
        // (0.50 against 0.39 ms per layer at batch 8).
        if (std::is_same<T, __nv_bfloat16>::value && ci == PTC_CI && co == 128 && f->N % 16 == 0) {
            const int64_t warps = (int64_t)B * f->N / 16;
            const int blocks = (int)std::min<int64_t>((warps + TPB / 32 - 1) / (TPB / 32), gb300::sm_count() * 8);
            k_pw_tc<128><<<blocks, TPB, 0, f->s>>>(reinterpret_cast<const __nv_bfloat16 *>(x), W, bias, extra,
                                                   reinterpret_cast<__nv_bfloat16 *>(pre),
                                                   reinterpret_cast<__nv_bfloat16 *>(yt), act, w0, f->N, B);
        } else if (pairs && ci == 32 && co % 8 == 0)
            k_pw_fwd_in2<T, T, 32><<<grid_for(units), TPB, sm, f->s>>>(x, co, W, bias, extra, pre, yt, act, w0, f->N,
                                                                      B);
        else if (pairs && ci == 4 && co % 8 == 0)
            k_pw_fwd_in2<T, T, 4><<<grid_for(units), TPB, sm, f->s>>>(x, co, W, bias, extra, pre, yt, act, w0, f->N, B);
        else
            k_pw_fwd_in<T, T><<<grid_for(units), TPB, sm, f->s>>>(x, ci, co, W, bias, extra, pre, yt, act, w0, f->N, B);
    } else if (pairs && ci % 8 == 0) {
        k_pw_fwd_out2<T><<<grid_for(units), TPB, sizeof(float) * ci * 8, f->s>>>(x, ci, co, W, bias,
                                                                                static_cast<float *>(y), f->N, B);
    } else {
        k_pw_fwd_out<T><<<grid_for(units), TPB, sizeof(float) * (co * ci + co), f->s>>>(x, ci, co, W, bias,
                                                                                       static_cast<float *>(y), f->N, B);
    }
}

template <class T>
void pw_bwd_input(fno_ctx *f, const float *g, int co, int ci, int64_t oW, const T *pre_in, int act, float *gx, int B)
{
    const bool pairs = f->N % 2 == 0;
    const int64_t units = pairs ? (int64_t)B * f->N / 2 : (int64_t)B * f->N;
    const float *W = f->params + oW;
    const float w0 = f->c.omega0;
    if (pairs && ci == 32 && co % 8 == 0)
        k_pw_bwd_in2<T, 32><<<grid_for(units), TPB, sizeof(float) * co * ci, f->s>>>(g, co, W, pre_in, act, w0, gx,
                                                                                    f->N, B);
    else if (ci <= 32)
        k_pw_bwd_in<T><<<grid_for(units), TPB, sizeof(float) * co * ci, f->s>>>(g, co, ci, W, pre_in, act, w0, gx,
                                                                               f->N, B);
    else if (pairs && ci % 8 == 0)
        k_pw_bwd_out2<T><<<grid_for(units), TPB, sizeof(float) * ci * 8, f->s>>>(g, co, ci, W, pre_in, act, w0, gx,
                                                                                f->N, B);
    else
        k_pw_bwd_out<T><<<grid_for(units), TPB, sizeof(float) * co * ci, f->s>>>(g, co, ci, W, pre_in, act, w0, gx,
                                                                                f->N, B);
}

template <class T>
void outer(fno_ctx *f, const float *g, int co, const T *x, int ci, int64_t oW, int64_t ob, int B)
{
    if (std::is_same<T, __nv_bfloat16>::value && ci == 32 && co % 32 == 0 && f->N % 16 == 0) {
        const int64_t total = (int64_t)B * f->N;
        const dim3 grid((unsigned)((total + OUTER_CHUNK - 1) / OUTER_CHUNK), (unsigned)(co / 32));
        k_outer_tc<<<grid, TPB, 0, f->s>>>(g, co, reinterpret_cast<const __nv_bfloat16 *>(x), f->grads + oW,
                                           f->grads + ob, f->N, B);
        return;
    }
    const int64_t total = (int64_t)B * f->N;
    const int nb = (int)((total + OUTER_CHUNK - 1) / OUTER_CHUNK);
    const int units = outer_units(co, ci);
    int groups = 1;
    while (units * groups * 2 <= TPB && groups * 2 <= OUTER_TILE / 4) groups *= 2;
    const size_t sm = smem_outer(co, ci);
    if (f->N % OUTER_TILE == 0) {                           // whole tiles: double-buffered cp.async copies
        if (units <= TPB)
            k_outer_async<T, 1><<<nb, TPB, sm, f->s>>>(g, co, x, ci, f->grads + oW, f->grads + ob, f->N, B, groups);
        else
            k_outer_async<T, 2><<<nb, TPB, sm, f->s>>>(g, co, x, ci, f->grads + oW, f->grads + ob, f->N, B, groups);
    } else if (units <= TPB) {
        k_outer<T, 1><<<nb, TPB, sm, f->s>>>(g, co, x, ci, f->grads + oW, f->grads + ob, f->N, B, groups);
    } else {
        k_outer<T, 2><<<nb, TPB, sm, f->s>>>(g, co, x, ci, f->grads + oW, f->grads + ob, f->N, B, groups);
    }
}

// the y stages on tensor cores: BF16-activation configuration, whole
// m-tiles and k-steps of eight modes or rows, 32 x modes
bool ydft_tc(const fno_ctx *f, const Dims &d)
{
    return f->c.act_bf16 && d.ny % 8 == 0 && d.Ky % 8 == 0 && d.Kx == 32;
}
size_t smem_cdft(const Dims &d) { return 2 * sizeof(uint4) * (size_t)(d.Ky / 8) * (d.ny / 8) * 32; }

Dims dims(const fno_ctx *f, int B)
{
    return Dims{f->c.nx, f->c.ny, f->c.nz, f->Kx, f->Ky, f->Kz, (int64_t)B * f->c.width};
}

// forward truncated DFT of [B][W][N] fields into S[k][b*W + c] times scale[kz]
template <class T>
void dft_fwd(fno_ctx *f, const T *x, float2 *S, const float *scale, int B, int layer_map = -1)
{
    const Dims d = dims(f, B);
    const int64_t R = d.BC * d.nz * d.ny;
    // FP32 rows take the tensor-core stage in the BF16-activation
    // configuration only (whose tolerance covers its 2^-16 rounding); the
    // FP32 configuration keeps the FP32 stage
    const bool tc_input = std::is_same<T, __nv_bfloat16>::value || f->c.act_bf16;
    if (layer_map >= 0 && layer_map < (int)f->vmaps.size() && std::is_same<T, __nv_bfloat16>::value) {
        // BF16 layer inputs with a tensor map: tcgen05 with TMEM accumulators
        const int64_t tiles = (R + 127) / 128;
        const int blocks = (int)std::min<int64_t>(tiles, (int64_t)gb300::sm_count() * 2);
        umma_dftx_fwd(f->vmaps[layer_map].data(), f->twx, f->stA, R, f->ustatus, blocks, f->s);
    } else if (tc_input && d.nx == TCX_NX && d.Kx == TCX_KX && (reinterpret_cast<uintptr_t>(x) & 15u) == 0) {
        const int64_t warps = (R + 15) / 16;
        k_dftx_fwd_tc<T><<<(int)std::min<int64_t>((warps + TPB / 32 - 1) / (TPB / 32), gb300::sm_count() * 8), TPB, 0, f->s>>>(
            x, f->stA, f->twx, R);
    } else {
        k_dftx_fwd<T><<<(int)std::min<int64_t>((R + DFT_ROWS - 1) / DFT_ROWS, gb300::sm_count() * 8), TPB, smem_dftx_fwd(d),
                        f->s>>>(x, f->stA, f->twx, d, R);
    }
    const int64_t Sl = d.BC * d.nz;
    if (ydft_tc(f, d)) {
        k_cdft_tc<4><<<(int)std::min<int64_t>((Sl + TPB / 32 - 1) / (TPB / 32), gb300::sm_count() * 8), TPB,
                       smem_cdft(d), f->s>>>(f->stA, f->stB, f->twy, d.Ky, 0, d.Ky, d.ny, Sl);
    } else {
        const int SB = dfty_fwd_slabs(d);
        k_dfty_fwd<<<(int)std::min<int64_t>((Sl + SB - 1) / SB, gb300::sm_count() * 8), TPB, smem_dfty_fwd(d), f->s>>>(
            f->stA, f->stB, f->twy, d, Sl, SB);
    }
    k_dftz_fwd<<<dftz_blocks(d), ZW * 32, 0, f->s>>>(f->stB, S, f->twz, scale, d);
}

// inverse of S (times scale[kz]) into out [B][W][N]: store or add; then, if pre
// is given, multiply by gelu'(pre)
// z and y stages of the inverse of S (times scale[kz]) into stA: rows
// [B][W][z][y] of Kx complex x modes
void dft_inv_zy(fno_ctx *f, const float2 *S, const float *scale, int B)
{
    const Dims d = dims(f, B);
    k_dftz_inv<<<dftz_blocks(d), ZW * 32, 0, f->s>>>(S, f->stB, f->twz, scale, d);
    const int64_t Sl = d.BC * d.nz;
    if (ydft_tc(f, d)) {
        k_cdft_tc<4><<<(int)std::min<int64_t>((Sl + TPB / 32 - 1) / (TPB / 32), gb300::sm_count() * 8), TPB,
                       smem_cdft(d), f->s>>>(f->stB, f->stA, f->twy, d.Ky, 1, d.ny, d.Ky, Sl);
    } else {
        const int SB = dfty_inv_slabs(d);
        k_dfty_inv<<<(int)std::min<int64_t>((Sl + SB - 1) / SB, gb300::sm_count() * 8), TPB, smem_dfty_inv(d), f->s>>>(
            f->stB, f->stA, f->twy, d, Sl, SB);
    }
}

template <class TP>
void dft_inv(fno_ctx *f, const float2 *S, float *out, const float *scale, int accumulate, const TP *pre, int B)
{
    const Dims d = dims(f, B);
    dft_inv_zy(f, S, scale, B);
    const int64_t R = d.BC * d.nz * d.ny;
    if (std::is_same<TP, __nv_bfloat16>::value && d.nx == TCX_NX && d.Kx == TCX_KX &&
        (reinterpret_cast<uintptr_t>(out) & 7u) == 0) {
        const int64_t warps = (R + 15) / 16;
        k_dftx_inv_tc<TP><<<(int)std::min<int64_t>((warps + TPB / 32 - 1) / (TPB / 32), gb300::sm_count() * 8), TPB, 0, f->s>>>(
            f->stA, out, f->twx, R, accumulate, pre);
    } else {
        k_dftx_inv<TP><<<(int)std::min<int64_t>((R + DFT_ROWS - 1) / DFT_ROWS, gb300::sm_count() * 8), TPB, smem_dftx_inv(d),
                         f->s>>>(f->stA, out, f->twx, d, R, accumulate, pre);
    }
}

void contract(fno_ctx *f, const float2 *Vin, int64_t oR, float2 *Gout, bool adj, int B)
{
    const float2 *R = reinterpret_cast<const float2 *>(f->params + oR);
    const int C = f->c.width;
    if (f->c.tensor_cores) {
        const int blocks = (int)std::min<int64_t>((f->K * 32 + TPB - 1) / TPB, gb300::sm_count() * 8);
        if (adj) k_contract_tc<true><<<blocks, TPB, 0, f->s>>>(Vin, R, Gout, C, B, f->K);
        else k_contract_tc<false><<<blocks, TPB, 0, f->s>>>(Vin, R, Gout, C, B, f->K);
    } else {
        if (adj) k_contract_f32<true><<<grid_for(f->K * B * C), TPB, 0, f->s>>>(Vin, R, Gout, C, B, f->K);
        else k_contract_f32<false><<<grid_for(f->K * B * C), TPB, 0, f->s>>>(Vin, R, Gout, C, B, f->K);
    }
}

template <class T>
lbm_status forward_impl(fno_ctx *f, const float *x, int B, bool keep = true)
{
    const fno_config &c = f->c;
    const int W = c.width;
    T *xa = static_cast<T *>(f->xa);
    if (!keep && std::is_same<T, __nv_bfloat16>::value && c.cin == LIFT_CI && c.lift_hidden == LIFT_H &&
        W == LIFT_CO && f->N % 2 == 0) {
        // inference: the lift's two layers in one pass from the FP32 input
        k_lift_fused<<<grid_for((int64_t)B * f->N / 2), TPB, 0, f->s>>>(
            x, f->params + f->oP1_w, f->params + f->oP1_b, f->params + f->oP2_w, f->params + f->oP2_b,
            reinterpret_cast<__nv_bfloat16 *>(f->v[0]), f->N, B);
    } else {
        k_convert<T><<<grid_for((int64_t)B * c.cin * f->N), TPB, 0, f->s>>>(x, xa, (int64_t)B * c.cin * f->N);
        // feed-forward lift: v0 = P2 GELU(P1 x + b1) + b2
        pw_fwd<T>(f, xa, c.cin, c.lift_hidden, f->oP1_w, f->oP1_b, nullptr,
                  keep ? static_cast<T *>(f->apre) : nullptr, f->a, false, ACT_GELU, B);
        pw_fwd<T>(f, static_cast<T *>(f->a), c.lift_hidden, W, f->oP2_w, f->oP2_b, nullptr, nullptr, f->v[0], false,
                  ACT_NONE, B);
    }
    // the fused Fourier-layer output (inverse x stage and pointwise path in
    // one tensor-core pass) where its shape applies
    const bool fuse = std::is_same<T, __nv_bfloat16>::value && c.nx == TCX_NX && f->Kx == TCX_KX && W == FUSE_C;
    for (int l = 0; l < c.layers; ++l) {
        T *vin = static_cast<T *>(f->v[l]);
        dft_fwd<T>(f, vin, f->Vh[l], f->scale_one, B, c.umma ? l : -1);
        contract(f, f->Vh[l], f->oR[l], f->G, false, B);
        if (fuse) {
            dft_inv_zy(f, f->G, f->scale_inv, B);
            const int64_t lps = (int64_t)c.ny * c.nz;
            const int blocks = (int)std::min<int64_t>(((int64_t)B * lps + FUSE_WARPS - 1) / FUSE_WARPS,
                                                      (int64_t)gb300::sm_count() * 2);
            k_layer_tc<<<blocks, FUSE_WARPS * 32, FUSE_SMEM, f->s>>>(
                f->stA, reinterpret_cast<const __nv_bfloat16 *>(vin), f->params + f->oW_w[l], f->params + f->oW_b[l],
                f->twx, keep ? reinterpret_cast<__nv_bfloat16 *>(f->pre[l]) : nullptr,
                reinterpret_cast<__nv_bfloat16 *>(f->v[l + 1]), l < c.layers - 1 ? ACT_GELU : ACT_NONE, lps, f->N, B);
            continue;
        }
        dft_inv<T>(f, f->G, f->spec, f->scale_inv, 0, nullptr, B);
        pw_fwd<T>(f, vin, W, W, f->oW_w[l], f->oW_b[l], f->spec, keep ? static_cast<T *>(f->pre[l]) : nullptr,
                  f->v[l + 1], false,
                  l < c.layers - 1 ? ACT_GELU : ACT_NONE, B);
    }
    const int H = c.hidden;
    const size_t smf = sizeof(float) * ((size_t)H * 32 + ((H + 3) & ~3) + (size_t)H * 8);
    if (!keep && std::is_same<T, __nv_bfloat16>::value && W == PTC_CI && H == PTC_H && c.cout <= 8 &&
        f->N % 16 == 0) {
        // inference on tensor cores: projection fused, hidden activations in registers
        const int64_t warps = (int64_t)B * f->N / 16;
        k_proj_tc<<<(int)std::min<int64_t>((warps + TPB / 32 - 1) / (TPB / 32), gb300::sm_count() * 8), TPB, 0, f->s>>>(
            reinterpret_cast<const __nv_bfloat16 *>(f->v[c.layers]), c.cout, f->params + f->oQ1_w,
            f->params + f->oQ1_b, f->params + f->oQ2_w, f->params + f->oQ2_b, c.omega0, f->y, f->N, B);
        return LBM_OK;
    }
    if (!keep && W == 32 && f->N % 2 == 0 && smf <= 48 * 1024) {
        // inference: projection fused, hidden activations not stored
        const size_t sm = smf;
        k_proj_fused<T, 32><<<grid_for((int64_t)B * f->N / 2), TPB, sm, f->s>>>(
            static_cast<T *>(f->v[c.layers]), H, c.cout, f->params + f->oQ1_w, f->params + f->oQ1_b,
            f->params + f->oQ2_w, f->params + f->oQ2_b, c.omega0, f->y, f->N, B);
        return LBM_OK;
    }
    // SIREN projection: h = sin(omega0 (Q1 v + b1)) (cos kept for the backward), y = Q2 h + b2
    pw_fwd<T>(f, static_cast<T *>(f->v[c.layers]), W, c.hidden, f->oQ1_w, f->oQ1_b, nullptr, static_cast<T *>(f->hcos),
              f->h, false, ACT_SIREN, B);
    pw_fwd<T>(f, static_cast<T *>(f->h), c.hidden, c.cout, f->oQ2_w, f->oQ2_b, nullptr, nullptr, f->y, true, ACT_NONE,
              B);
    return LBM_OK;
}

template <class T>
lbm_status backward_impl(fno_ctx *f, int B)
{
    const fno_config &c = f->c;
    const int W = c.width, H = c.hidden;
    cudaMemsetAsync(f->grads, 0, f->np * sizeof(float), f->s);
    // projection: y = Q2 h + b2, h = sin(omega0 z), z = Q1 v_L + b1; dh/dz = omega0 cos(omega0 z)
    outer<T>(f, f->gy, c.cout, static_cast<T *>(f->h), H, f->oQ2_w, f->oQ2_b, B);
    pw_bwd_input<T>(f, f->gy, c.cout, H, f->oQ2_w, static_cast<T *>(f->hcos), ACT_SIREN, f->ghpre, B);
    outer<T>(f, f->ghpre, H, static_cast<T *>(f->v[c.layers]), W, f->oQ1_w, f->oQ1_b, B);
    float *gpre = f->gA, *gnext = f->gB;
    // gradient of v_L = pre_{L-1} (no activation after the last layer)
    pw_bwd_input<T>(f, f->ghpre, H, W, f->oQ1_w, static_cast<const T *>(nullptr), ACT_NONE, gpre, B);
    for (int l = c.layers - 1; l >= 0; --l) {
        T *vin = static_cast<T *>(f->v[l]);
        outer<T>(f, gpre, W, vin, W, f->oW_w[l], f->oW_b[l], B);
        // spectral branch: gG = (c/N) DFT(gpre); gR = sum_b gG conj(V); gV = gG R^H
        dft_fwd<float>(f, gpre, f->gG, f->scale_inv, B);
        k_grad_R<<<grid_for(f->K * W * W), TPB, 0, f->s>>>(f->gG, f->Vh[l],
                                                           reinterpret_cast<float2 *>(f->grads + f->oR[l]), W, B, f->K);
        contract(f, f->gG, f->oR[l], f->gVh, true, B);
        // gv_l = W_l^T gpre + adjoint DFT(gV), times gelu'(pre_{l-1}) for l > 0
        pw_bwd_input<T>(f, gpre, W, W, f->oW_w[l], static_cast<const T *>(nullptr), ACT_NONE, gnext, B);
        const T *pre_prev = l > 0 ? static_cast<T *>(f->pre[l - 1]) : nullptr;
        dft_inv<T>(f, f->gVh, gnext, f->scale_one, 1, pre_prev, B);
        std::swap(gpre, gnext);
    }
    // lift: v0 = P2 a + b2, a = GELU(P1 x + b1)
    outer<T>(f, gpre, W, static_cast<T *>(f->a), c.lift_hidden, f->oP2_w, f->oP2_b, B);
    pw_bwd_input<T>(f, gpre, W, c.lift_hidden, f->oP2_w, static_cast<T *>(f->apre), ACT_GELU, gnext, B);
    outer<T>(f, gnext, c.lift_hidden, static_cast<T *>(f->xa), c.cin, f->oP1_w, f->oP1_b, B);
    return LBM_OK;
}

}  // namespace

static lbm_status stage_input(fno_ctx *f, const float *src, float *dst, int64_t count)
{
    FCK(cudaMemcpyAsync(dst, src, count * sizeof(float), on_device(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        f->s));
    return LBM_OK;
}

extern "C" lbm_status fno_forward(fno_ctx *f, const float *x, float *y, int32_t batch)
{
    if (!f || !x || !y || batch < 1) return LBM_ERR_ARG;
    const fno_config &c = f->c;
    for (int b0 = 0; b0 < batch; b0 += c.max_batch) {
        const int B = std::min(c.max_batch, batch - b0);
        const float *xb = x + (int64_t)b0 * c.cin * f->N;
        lbm_status st = stage_input(f, xb, f->xin, (int64_t)B * c.cin * f->N);
        if (st != LBM_OK) return st;
        st = c.act_bf16 ? forward_impl<__nv_bfloat16>(f, f->xin, B, false) : forward_impl<float>(f, f->xin, B, false);
        if (st != LBM_OK) return st;
        FCK(cudaGetLastError());
        FCK(cudaMemcpyAsync(y + (int64_t)b0 * c.cout * f->N, f->y, (int64_t)B * c.cout * f->N * sizeof(float),
                            cudaMemcpyDefault, f->s));
    }
    if (!on_device(y)) FCK(cudaStreamSynchronize(f->s));
    return LBM_OK;
}

extern "C" lbm_status fno_loss_grad(fno_ctx *f, const float *x, const float *t, const float *m, int32_t batch,
                                    double *loss)
{
    if (!f || !x || !t || !m || batch < 1 || batch > f->c.max_batch) {
        if (f) f->err = "batch must be in [1, max_batch]";
        return LBM_ERR_ARG;
    }
    const fno_config &c = f->c;
    const int B = batch;
    lbm_status st = stage_input(f, x, f->xin, (int64_t)B * c.cin * f->N);
    if (st == LBM_OK) st = stage_input(f, t, f->tin, (int64_t)B * c.cout * f->N);
    if (st == LBM_OK) st = stage_input(f, m, f->min, (int64_t)B * f->N);
    if (st != LBM_OK) return st;
    st = c.act_bf16 ? forward_impl<__nv_bfloat16>(f, f->xin, B) : forward_impl<float>(f, f->xin, B);
    if (st != LBM_OK) return st;
    k_mse_partial<<<f->nparts, TPB, 0, f->s>>>(f->y, f->tin, f->min, c.cout, f->N, B, f->part);
    k_mse_final<<<1, 32, 0, f->s>>>(f->part, f->nparts, c.cout, f->res);
    k_mse_grad<<<grid_for((int64_t)B * c.cout * f->N), TPB, 0, f->s>>>(f->y, f->tin, f->min, c.cout, f->N, B, f->res,
                                                                       f->gy);
    st = c.act_bf16 ? backward_impl<__nv_bfloat16>(f, B) : backward_impl<float>(f, B);
    if (st != LBM_OK) return st;
    FCK(cudaGetLastError());
    if (loss) {
        double r[2];
        FCK(cudaMemcpyAsync(r, f->res, sizeof r, cudaMemcpyDeviceToHost, f->s));
        FCK(cudaStreamSynchronize(f->s));
        *loss = r[0];
    }
    return LBM_OK;
}

extern "C" lbm_status fno_adam_step(fno_ctx *f, float lr, float b1, float b2, float eps)
{
    if (!f) return LBM_ERR_ARG;
    f->adam_t++;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)f->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)f->adam_t)));
    k_adam<<<grid_for(f->np), TPB, 0, f->s>>>(f->params, f->grads, f->m1, f->m2, f->np, lr, b1, b2, eps, c1, c2);
    FCK(cudaGetLastError());
    return LBM_OK;
}

extern "C" lbm_status fno_train_step(fno_ctx *f, const float *x, const float *t, const float *m, int32_t batch,
                                     float lr, double *loss)
{
    lbm_status st = fno_loss_grad(f, x, t, m, batch, loss);
    if (st != LBM_OK) return st;
    return fno_adam_step(f, lr, 0.9f, 0.999f, 1e-8f);
}

namespace {
struct FnoCkpt {
    char magic[8];
    int32_t nx, ny, nz, cin, width, cout, mx, my, mz, layers, hidden, lift_hidden;
    float omega0;
    int32_t pad;
    int64_t np, adam_t;
};

FnoCkpt ckpt_header(const fno_ctx *f)
{
    FnoCkpt h{};
    std::memcpy(h.magic, "GBFNOCK1", 8);
    const fno_config &c = f->c;
    h.nx = c.nx; h.ny = c.ny; h.nz = c.nz; h.cin = c.cin; h.width = c.width; h.cout = c.cout;
    h.mx = c.mx; h.my = c.my; h.mz = c.mz; h.layers = c.layers; h.hidden = c.hidden; h.lift_hidden = c.lift_hidden;
    h.omega0 = c.omega0;
    h.np = f->np;
    h.adam_t = f->adam_t;
    return h;
}
}  // namespace

extern "C" lbm_status fno_save(fno_ctx *f, const char *path)
{
    if (!f || !path) return LBM_ERR_ARG;
    std::vector<float> buf(3 * (size_t)f->np);
    FCK(cudaStreamSynchronize(f->s));
    FCK(cudaMemcpy(buf.data(), f->params, f->np * sizeof(float), cudaMemcpyDeviceToHost));
    FCK(cudaMemcpy(buf.data() + f->np, f->m1, f->np * sizeof(float), cudaMemcpyDeviceToHost));
    FCK(cudaMemcpy(buf.data() + 2 * f->np, f->m2, f->np * sizeof(float), cudaMemcpyDeviceToHost));
    const FnoCkpt h = ckpt_header(f);
    FILE *fp = std::fopen(path, "wb");
    if (!fp) {
        f->err = std::string("cannot open ") + path;
        return LBM_ERR_IO;
    }
    bool ok = std::fwrite(&h, sizeof h, 1, fp) == 1 && std::fwrite(buf.data(), sizeof(float), buf.size(), fp) == buf.size();
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) f->err = "checkpoint write failed";
    return ok ? LBM_OK : LBM_ERR_IO;
}

extern "C" lbm_status fno_load(fno_ctx *f, const char *path)
{
    if (!f || !path) return LBM_ERR_ARG;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) {
        f->err = std::string("cannot open ") + path;
        return LBM_ERR_IO;
    }
    FnoCkpt h{};
    FnoCkpt mine = ckpt_header(f);
    const bool same = std::fread(&h, sizeof h, 1, fp) == 1 && std::memcmp(h.magic, mine.magic, 8) == 0 &&
                      std::memcmp(&h.nx, &mine.nx, offsetof(FnoCkpt, np) - offsetof(FnoCkpt, nx)) == 0 &&
                      h.np == mine.np;
    std::vector<float> buf(3 * (size_t)f->np);
    const bool ok = same && std::fread(buf.data(), sizeof(float), buf.size(), fp) == buf.size();
    std::fclose(fp);
    if (!ok) {
        f->err = same ? "checkpoint truncated" : "checkpoint does not match this network's shape";
        return LBM_ERR_IO;
    }
    FCK(cudaStreamSynchronize(f->s));
    FCK(cudaMemcpy(f->params, buf.data(), f->np * sizeof(float), cudaMemcpyHostToDevice));
    FCK(cudaMemcpy(f->m1, buf.data() + f->np, f->np * sizeof(float), cudaMemcpyHostToDevice));
    FCK(cudaMemcpy(f->m2, buf.data() + 2 * f->np, f->np * sizeof(float), cudaMemcpyHostToDevice));
    f->adam_t = h.adam_t;
    return LBM_OK;
}

extern "C" lbm_status fno_sync(fno_ctx *f)
{
    if (!f) return LBM_ERR_ARG;
    FCK(cudaStreamSynchronize(f->s));
    int st = 0;
    FCK(cudaMemcpy(&st, f->ustatus, sizeof st, cudaMemcpyDeviceToHost));
    if (st != 0) {
        FCK(cudaMemset(f->ustatus, 0, sizeof(int)));
        f->err = "a bounded wait of the tcgen05 x stage gave up (code " + std::to_string(st) + ")";
        return LBM_ERR_TIMEOUT;
    }
    return LBM_OK;
}

extern "C" const char *fno_last_error(const fno_ctx *f) { return f ? f->err.c_str() : g_fno_err.c_str(); }
