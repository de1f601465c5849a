// fno.cu -- kernels and host orchestration of the Fourier Neural Operator
// surrogate declared in include/fno.h (paper Sec. 4 and the appendix on the
// baseline models: FNO of Li et al. 2021 mapping mask and Re to the mean
// field).
//
// Kernels:
//   k_pw_fwd_*   pointwise layers (lift, W path, projection) with fused bias,
//                spectral-branch add and GELU; pre-activations kept for backward
//   k_pw_bwd_*   input gradients of pointwise layers with fused GELU'
//   k_outer      weight/bias gradients sum_{b,cell} gout x
//   k_dft*       truncated DFT in three separable stages (x, y, z) and the
//                inverse (z, y, x), FP32 with twiddle tables in shared memory
//   k_contract_tc  per-mode complex channel mixing on tensor cores
//                (mma.sync m16n8k16 BF16 operands, FP32 accumulation); complex
//                numbers enter as real 2x2 blocks, the batch is the n8 axis
//   k_contract_f32 the same contraction in FP32 (reference and small widths)
//   k_grad_R     spectral weight gradients sum_b gG conj(V)
//   k_mse_*      masked mean square error and its gradient (deterministic)
//   k_adam       Adam update of the flat parameter vector
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/fno.h"

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

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a conj(b)

int grid_for(int64_t n, int block = TPB) { return (int)std::min<int64_t>((n + block - 1) / block, 152 * 16); }

// ---------------------------------------------------------------------------
// pointwise layers
// ---------------------------------------------------------------------------
// y = act(W x + b + extra) for ci <= 32 (inputs cached in registers).
template <class TI, class TO>
__global__ void __launch_bounds__(TPB) k_pw_fwd_in(const TI *x, int ci, int co, const float *W, const float *bias,
                                                   const float *extra, TO *pre, TO *y, int act, int64_t N, int B)
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
            if (pre) stf(pre + off, acc);
            stf(y + off, act ? gelu(acc) : acc);
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

// gx = (W^T g) * (act ? gelu'(pre_in) : 1), ci <= 32 (gx accumulated in registers).
template <class TP>
__global__ void __launch_bounds__(TPB) k_pw_bwd_in(const float *g, int co, int ci, const float *W, const TP *pre_in,
                                                   float *gx, int64_t N, int B)
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
                gx[off] = pre_in ? acc[i] * gelu_grad(ldf(pre_in + off)) : acc[i];
            }
    }
}

// Same for co <= 8 and any ci (g cached in registers, inputs streamed).
template <class TP>
__global__ void __launch_bounds__(TPB) k_pw_bwd_out(const float *g, int co, int ci, const float *W, const TP *pre_in,
                                                    float *gx, int64_t N, int B)
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
            gx[off] = pre_in ? acc * gelu_grad(ldf(pre_in + off)) : acc;
        }
    }
}

// gW[o][i] += sum_{b,cell} g[b][o][cell] x[b][i][cell], gb[o] += sum g.  Each
// block reduces a chunk of cells through shared-memory tiles and adds its
// partial sums atomically.
constexpr int OUTER_TILE = 64;
constexpr int OUTER_LD = OUTER_TILE + 1;           // padded row: no bank conflicts
constexpr int OUTER_CHUNK = 8192;
constexpr int OUTER_PAIRS = 20;                     // pairs (o, i) per thread: co * (ci + 1) <= 5120

template <class TX>
__global__ void __launch_bounds__(TPB) k_outer(const float *g, int co, const TX *x, int ci, float *gW, float *gb,
                                               int64_t N, int B)
{
    extern __shared__ float sm[];
    float *sg = sm, *sx = sm + co * OUTER_LD;
    const int np = co * (ci + 1);                      // pairs (o, i), i = ci is the bias
    float acc[OUTER_PAIRS];
#pragma unroll
    for (int k = 0; k < OUTER_PAIRS; ++k) acc[k] = 0.f;
    const int64_t total = (int64_t)B * N;
    const int64_t c0 = (int64_t)blockIdx.x * OUTER_CHUNK;
    const int64_t c1 = c0 + OUTER_CHUNK < total ? c0 + OUTER_CHUNK : total;
    for (int64_t t0 = c0; t0 < c1; t0 += OUTER_TILE) {
        __syncthreads();
        for (int k = threadIdx.x; k < (co + ci) * OUTER_TILE; k += blockDim.x) {
            const int ch = k / OUTER_TILE, j = k % OUTER_TILE;
            const int64_t cell = t0 + j;
            float v = 0.f;
            if (cell < c1) {
                const int64_t b = cell / N, n = cell - b * N;
                v = ch < co ? g[(b * co + ch) * N + n] : ldf(x + (b * ci + (ch - co)) * N + n);
            }
            sm[ch * OUTER_LD + j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < OUTER_PAIRS; ++k) {
            const int pidx = threadIdx.x + k * TPB;
            if (pidx < np) {
                const int o = pidx / (ci + 1), i = pidx % (ci + 1);
                float s = 0.f;
                if (i < ci)
                    for (int j = 0; j < OUTER_TILE; ++j) s += sg[o * OUTER_LD + j] * sx[i * OUTER_LD + j];
                else
                    for (int j = 0; j < OUTER_TILE; ++j) s += sg[o * OUTER_LD + j];
                acc[k] += s;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < OUTER_PAIRS; ++k) {
        const int pidx = threadIdx.x + k * TPB;
        if (pidx < np) {
            const int o = pidx / (ci + 1), i = pidx % (ci + 1);
            atomicAdd(i < ci ? &gW[o * ci + i] : &gb[o], acc[k]);
        }
    }
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

// rows [R][nx] (real) -> A [R][Kx] (complex)
template <class TI>
__global__ void __launch_bounds__(TPB) k_dftx_fwd(const TI *x, float2 *A, const float2 *twx, Dims d, int64_t R)
{
    extern __shared__ float2 smc[];
    float2 *tw = smc;                                   // [nx][Kx]
    float *rows = reinterpret_cast<float *>(smc + d.nx * d.Kx);
    for (int k = threadIdx.x; k < d.nx * d.Kx; k += blockDim.x) tw[k] = twx[k];
    const int rpb = blockDim.x / d.Kx;                  // rows per group
    for (int64_t r0 = (int64_t)blockIdx.x * rpb; r0 < R; r0 += (int64_t)gridDim.x * rpb) {
        __syncthreads();
        for (int k = threadIdx.x; k < rpb * d.nx; k += blockDim.x) {
            const int64_t r = r0 + k / d.nx;
            rows[k] = r < R ? ldf(x + r0 * d.nx + k) : 0.f;
        }
        __syncthreads();
        const int lr = threadIdx.x / d.Kx, j = threadIdx.x % d.Kx;
        const int64_t r = r0 + lr;
        if (lr < rpb && r < R) {
            float2 acc = make_float2(0.f, 0.f);
            const float *row = rows + lr * d.nx;
            for (int xx = 0; xx < d.nx; ++xx) {
                const float2 t = tw[xx * d.Kx + j];
                acc.x += row[xx] * t.x;
                acc.y += row[xx] * t.y;
            }
            A[r * d.Kx + j] = acc;
        }
    }
}

// A [S][ny][Kx] -> B [S][Ky][Kx], S = BC*nz slabs
__global__ void __launch_bounds__(TPB) k_dfty_fwd(const float2 *A, float2 *Bt, const float2 *twy, Dims d, int64_t S)
{
    extern __shared__ float2 smc[];
    float2 *tw = smc;                                   // [ny][Ky]
    float2 *slab = smc + d.ny * d.Ky;                   // [ny][Kx]
    for (int k = threadIdx.x; k < d.ny * d.Ky; k += blockDim.x) tw[k] = twy[k];
    for (int64_t s = blockIdx.x; s < S; s += gridDim.x) {
        __syncthreads();
        for (int k = threadIdx.x; k < d.ny * d.Kx; k += blockDim.x) slab[k] = A[s * d.ny * d.Kx + k];
        __syncthreads();
        for (int o = threadIdx.x; o < d.Ky * d.Kx; o += blockDim.x) {
            const int jy = o / d.Kx, jx = o % d.Kx;
            float2 acc = make_float2(0.f, 0.f);
            for (int y = 0; y < d.ny; ++y) {
                const float2 v = cmul(slab[y * d.Kx + jx], tw[y * d.Ky + jy]);
                acc.x += v.x;
                acc.y += v.y;
            }
            Bt[s * d.Ky * d.Kx + o] = acc;
        }
    }
}

// B [BC][nz][Ky][Kx] -> S[k][bc] with factor scale[kz]
__global__ void __launch_bounds__(TPB) k_dftz_fwd(const float2 *Bt, float2 *Sp, const float2 *twz, const float *scale,
                                                  Dims d)
{
    const int64_t P = d.BC * d.Ky * d.Kx;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bc = t / (d.Ky * d.Kx);
        const int p = (int)(t % (d.Ky * d.Kx));
        float2 acc[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = make_float2(0.f, 0.f);
        for (int z = 0; z < d.nz; ++z) {
            const float2 v = Bt[(bc * d.nz + z) * d.Ky * d.Kx + p];
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < d.Kz) {
                    const float2 w = cmul(v, twz[z * d.Kz + k]);
                    acc[k].x += w.x;
                    acc[k].y += w.y;
                }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < d.Kz) Sp[((int64_t)k * d.Ky * d.Kx + p) * d.BC + bc] = make_float2(acc[k].x * scale[k], acc[k].y * scale[k]);
    }
}

// S[k][bc] (times scale[kz]) -> H [BC][nz][Ky][Kx] = sum_kz G exp(+i 2 pi kz z / nz)
__global__ void __launch_bounds__(TPB) k_dftz_inv(const float2 *Sp, float2 *Ht, const float2 *twz, const float *scale,
                                                  Dims d)
{
    const int64_t P = d.BC * d.Ky * d.Kx;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bc = t / (d.Ky * d.Kx);
        const int p = (int)(t % (d.Ky * d.Kx));
        float2 G[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            G[k] = make_float2(0.f, 0.f);
            if (k < d.Kz) {
                const float2 v = Sp[((int64_t)k * d.Ky * d.Kx + p) * d.BC + bc];
                G[k] = make_float2(v.x * scale[k], v.y * scale[k]);
            }
        }
        for (int z = 0; z < d.nz; ++z) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < d.Kz) {
                    const float2 w = cmulc(G[k], twz[z * d.Kz + k]);
                    acc.x += w.x;
                    acc.y += w.y;
                }
            Ht[(bc * d.nz + z) * d.Ky * d.Kx + p] = acc;
        }
    }
}

// H [S][Ky][Kx] -> I [S][ny][Kx] = sum_jy H exp(+i 2 pi ky y / ny)
__global__ void __launch_bounds__(TPB) k_dfty_inv(const float2 *Ht, float2 *It, const float2 *twy, Dims d, int64_t S)
{
    extern __shared__ float2 smc[];
    float2 *tw = smc;                                   // [ny][Ky]
    float2 *slab = smc + d.ny * d.Ky;                   // [Ky][Kx]
    for (int k = threadIdx.x; k < d.ny * d.Ky; k += blockDim.x) tw[k] = twy[k];
    for (int64_t s = blockIdx.x; s < S; s += gridDim.x) {
        __syncthreads();
        for (int k = threadIdx.x; k < d.Ky * d.Kx; k += blockDim.x) slab[k] = Ht[s * d.Ky * d.Kx + k];
        __syncthreads();
        for (int o = threadIdx.x; o < d.ny * d.Kx; o += blockDim.x) {
            const int y = o / d.Kx, jx = o % d.Kx;
            float2 acc = make_float2(0.f, 0.f);
            for (int jy = 0; jy < d.Ky; ++jy) {
                const float2 v = cmulc(slab[jy * d.Kx + jx], tw[y * d.Ky + jy]);
                acc.x += v.x;
                acc.y += v.y;
            }
            It[s * d.ny * d.Kx + o] = acc;
        }
    }
}

// I [R][Kx] -> out [R][nx] = Re sum_jx I exp(+i 2 pi kx x / nx); mode 0: store,
// mode 1: add to out; then, if pre is given, multiply by gelu'(pre).
template <class TP>
__global__ void __launch_bounds__(TPB) k_dftx_inv(const float2 *It, float *out, const float2 *twx, Dims d, int64_t R,
                                                  int accumulate, const TP *pre)
{
    extern __shared__ float2 smc[];
    float2 *tw = smc;                                   // [nx][Kx]
    float2 *rows = smc + d.nx * d.Kx;                   // [rpb][Kx]
    for (int k = threadIdx.x; k < d.nx * d.Kx; k += blockDim.x) tw[k] = twx[k];
    const int rpb = 8;
    for (int64_t r0 = (int64_t)blockIdx.x * rpb; r0 < R; r0 += (int64_t)gridDim.x * rpb) {
        __syncthreads();
        for (int k = threadIdx.x; k < rpb * d.Kx; k += blockDim.x) {
            const int64_t r = r0 + k / d.Kx;
            rows[k] = r < R ? It[r0 * d.Kx + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int o = threadIdx.x; o < rpb * d.nx; o += blockDim.x) {
            const int lr = o / d.nx, xx = o % d.nx;
            const int64_t r = r0 + lr;
            if (r >= R) continue;
            float acc = 0.f;
            const float2 *row = rows + lr * d.Kx;
            for (int j = 0; j < d.Kx; ++j) {
                const float2 t = tw[xx * d.Kx + j];
                acc += row[j].x * t.x + row[j].y * t.y;     // Re(I conj(t))
            }
            const int64_t off = r * d.nx + xx;
            float v = accumulate ? out[off] + acc : acc;
            if (pre) v *= gelu_grad(ldf(pre + off));
            out[off] = v;
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
    int64_t oP_w = 0, oP_b = 0, oQ1_w = 0, oQ1_b = 0, oQ2_w = 0, oQ2_b = 0;
    std::vector<int64_t> oR, oW_w, oW_b;
    float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
    int64_t adam_t = 0;
    // device buffers
    std::vector<void *> allocs;
    void *xa = nullptr;                       // converted input (act type)
    std::vector<void *> v, pre;               // activations
    void *hpre = nullptr, *h = nullptr;
    float *y = nullptr, *spec = nullptr, *gy = nullptr, *ghpre = nullptr, *gA = nullptr, *gB = nullptr;
    float *xin = nullptr, *tin = nullptr, *min = nullptr;
    float2 *stA = nullptr, *stB = nullptr;    // DFT stage temporaries
    std::vector<float2 *> Vh;                 // per-layer spectra of the layer inputs
    float2 *G = nullptr, *gG = nullptr, *gVh = nullptr;
    float2 *twx = nullptr, *twy = nullptr, *twz = nullptr;
    float *scale_one = nullptr, *scale_inv = nullptr;
    double *part = nullptr, *res = nullptr;
    int nparts = 0;
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
    if (c.mx < 1 || c.my < 1 || c.mz < 1 || 2 * c.mx > c.nx || 2 * c.my > c.ny || c.mz >= c.nz / 2 + 1 || c.mz > 16)
        return bad("modes must satisfy 2mx <= nx, 2my <= ny, mz <= nz/2, mz <= 16");
    if (c.tensor_cores && c.width % 8 != 0) return bad("tensor-core contraction needs width % 8 == 0");
    if (2 * c.mx > 256) return bad("2mx must be <= 256");
    const size_t smx = sizeof(float2) * c.nx * 2 * c.mx + sizeof(float) * (256 / (2 * c.mx)) * c.nx;
    const size_t smi = sizeof(float2) * (c.nx * 2 * c.mx + 8 * 2 * c.mx);
    const size_t smy = sizeof(float2) * (c.ny * 2 * c.my + c.ny * 2 * c.mx);
    const int outer_ch = std::max(std::max(c.hidden + c.width, c.cout + c.hidden), std::max(2 * c.width, c.width + c.cin));
    const size_t smo = sizeof(float) * outer_ch * (OUTER_TILE + 1);
    if (smx > 48 * 1024 || smi > 48 * 1024 || smy > 48 * 1024 || smo > 48 * 1024)
        return bad("grid x modes too large for the shared-memory twiddle tables");
    if ((int64_t)c.hidden * (c.width + 1) > OUTER_PAIRS * TPB || (int64_t)c.cout * (c.hidden + 1) > OUTER_PAIRS * TPB ||
        (int64_t)c.width * (c.width + 1) > OUTER_PAIRS * TPB)
        return bad("layer too wide for the gradient reduction");
    fno_ctx *f = new fno_ctx();
    f->c = c;
    f->s = static_cast<cudaStream_t>(stream);
    f->N = (int64_t)c.nx * c.ny * c.nz;
    f->Kx = 2 * c.mx; f->Ky = 2 * c.my; f->Kz = c.mz;
    f->K = (int64_t)f->Kx * f->Ky * f->Kz;
    const int W = c.width, H = c.hidden;
    // spectral weights first: every R_l starts at an even float index, so
    // its complex entries are 8-byte aligned
    int64_t o = 0;
    for (int l = 0; l < c.layers; ++l) { f->oR.push_back(o); o += 2 * f->K * W * W; }
    f->oP_w = o; o += (int64_t)W * c.cin;
    f->oP_b = o; o += W;
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
    chk(f->hpre = f->alloc<char>(B * H * N * es));
    chk(f->h = f->alloc<char>(B * H * N * es));
    chk(f->y = f->alloc<float>(B * c.cout * N));
    chk(f->spec = f->alloc<float>(B * W * N));
    chk(f->gy = f->alloc<float>(B * c.cout * N));
    chk(f->ghpre = f->alloc<float>(B * H * N));
    chk(f->gA = f->alloc<float>(B * W * N));
    chk(f->gB = f->alloc<float>(B * W * N));
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
    f->nparts = 152 * 4;
    chk(f->part = f->alloc<double>(2 * f->nparts));
    chk(f->res = f->alloc<double>(2));
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
    // initial parameters (same scales as a 1/sqrt(fan-in) uniform init)
    std::vector<float> p0(o);
    uint64_t st = c.seed * 0x9E3779B97F4A7C15ull + 12345;
    auto fill = [&](int64_t off, int64_t cnt, double s) { for (int64_t k = 0; k < cnt; ++k) p0[off + k] = (float)(s * unif(st)); };
    fill(f->oP_w, (int64_t)W * c.cin, 1.0 / std::sqrt((double)c.cin));
    fill(f->oP_b, W, 1.0 / std::sqrt((double)c.cin));
    for (int l = 0; l < c.layers; ++l) {
        fill(f->oR[l], 2 * f->K * W * W, 1.0 / ((double)W * W));
        fill(f->oW_w[l], (int64_t)W * W, 1.0 / std::sqrt((double)W));
        fill(f->oW_b[l], W, 1.0 / std::sqrt((double)W));
    }
    fill(f->oQ1_w, (int64_t)H * W, 1.0 / std::sqrt((double)W));
    fill(f->oQ1_b, H, 1.0 / std::sqrt((double)W));
    fill(f->oQ2_w, (int64_t)c.cout * H, 1.0 / std::sqrt((double)H));
    fill(f->oQ2_b, c.cout, 1.0 / std::sqrt((double)H));
    ok = ok && cudaMemcpy(f->params, p0.data(), o * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(f->m1, 0, o * sizeof(float)) == cudaSuccess && cudaMemset(f->m2, 0, o * sizeof(float)) == cudaSuccess &&
         cudaMemset(f->grads, 0, o * sizeof(float)) == cudaSuccess;
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
    const size_t sm = sizeof(float) * (co * ci + co);
    if (ci <= 32 && !y_is_float) {
        k_pw_fwd_in<T, T><<<grid_for((int64_t)B * f->N), TPB, sm, f->s>>>(x, ci, co, f->params + oW, f->params + ob, extra,
                                                                        pre, static_cast<T *>(y), act, f->N, B);
    } else {
        k_pw_fwd_out<T><<<grid_for((int64_t)B * f->N), TPB, sm, f->s>>>(x, ci, co, f->params + oW, f->params + ob,
                                                                      static_cast<float *>(y), f->N, B);
    }
}

template <class T>
void pw_bwd_input(fno_ctx *f, const float *g, int co, int ci, int64_t oW, const T *pre_in, float *gx, int B)
{
    const size_t sm = sizeof(float) * co * ci;
    if (ci <= 32)
        k_pw_bwd_in<T><<<grid_for((int64_t)B * f->N), TPB, sm, f->s>>>(g, co, ci, f->params + oW, pre_in, gx, f->N, B);
    else
        k_pw_bwd_out<T><<<grid_for((int64_t)B * f->N), TPB, sm, f->s>>>(g, co, ci, f->params + oW, pre_in, gx, f->N, B);
}

template <class T>
void outer(fno_ctx *f, const float *g, int co, const T *x, int ci, int64_t oW, int64_t ob, int B)
{
    const int64_t total = (int64_t)B * f->N;
    const int nb = (int)((total + OUTER_CHUNK - 1) / OUTER_CHUNK);
    const size_t sm = sizeof(float) * (co + ci) * OUTER_LD;
    k_outer<T><<<nb, TPB, sm, f->s>>>(g, co, x, ci, f->grads + oW, f->grads + ob, f->N, B);
}

Dims dims(const fno_ctx *f, int B)
{
    return Dims{f->c.nx, f->c.ny, f->c.nz, f->Kx, f->Ky, f->Kz, (int64_t)B * f->c.width};
}

// forward truncated DFT of [B][W][N] fields into S[k][b*W + c] times scale[kz]
template <class T>
void dft_fwd(fno_ctx *f, const T *x, float2 *S, const float *scale, int B)
{
    const Dims d = dims(f, B);
    const int64_t R = d.BC * d.nz * d.ny;
    const int rpb = TPB / d.Kx;
    const size_t smx = sizeof(float2) * d.nx * d.Kx + sizeof(float) * rpb * d.nx;
    k_dftx_fwd<T><<<(int)std::min<int64_t>((R + rpb - 1) / rpb, 152 * 8), TPB, smx, f->s>>>(x, f->stA, f->twx, d, R);
    const int64_t Sl = d.BC * d.nz;
    const size_t smy = sizeof(float2) * (d.ny * d.Ky + d.ny * d.Kx);
    k_dfty_fwd<<<(int)std::min<int64_t>(Sl, 152 * 8), TPB, smy, f->s>>>(f->stA, f->stB, f->twy, d, Sl);
    k_dftz_fwd<<<grid_for(d.BC * d.Ky * d.Kx), TPB, 0, f->s>>>(f->stB, S, f->twz, scale, d);
}

// inverse of S (times scale[kz]) into out [B][W][N]: store or add; then, if pre
// is given, multiply by gelu'(pre)
template <class TP>
void dft_inv(fno_ctx *f, const float2 *S, float *out, const float *scale, int accumulate, const TP *pre, int B)
{
    const Dims d = dims(f, B);
    k_dftz_inv<<<grid_for(d.BC * d.Ky * d.Kx), TPB, 0, f->s>>>(S, f->stB, f->twz, scale, d);
    const int64_t Sl = d.BC * d.nz;
    const size_t smy = sizeof(float2) * (d.ny * d.Ky + d.Ky * d.Kx);
    k_dfty_inv<<<(int)std::min<int64_t>(Sl, 152 * 8), TPB, smy, f->s>>>(f->stB, f->stA, f->twy, d, Sl);
    const int64_t R = d.BC * d.nz * d.ny;
    const size_t smx = sizeof(float2) * (d.nx * d.Kx + 8 * d.Kx);
    k_dftx_inv<TP><<<(int)std::min<int64_t>((R + 7) / 8, 152 * 8), TPB, smx, f->s>>>(f->stA, out, f->twx, d, R, accumulate,
                                                                                    pre);
}

void contract(fno_ctx *f, const float2 *Vin, int64_t oR, float2 *Gout, bool adj, int B)
{
    const float2 *R = reinterpret_cast<const float2 *>(f->params + oR);
    const int C = f->c.width;
    if (f->c.tensor_cores) {
        const int blocks = (int)std::min<int64_t>((f->K * 32 + TPB - 1) / TPB, 152 * 8);
        if (adj) k_contract_tc<true><<<blocks, TPB, 0, f->s>>>(Vin, R, Gout, C, B, f->K);
        else k_contract_tc<false><<<blocks, TPB, 0, f->s>>>(Vin, R, Gout, C, B, f->K);
    } else {
        if (adj) k_contract_f32<true><<<grid_for(f->K * B * C), TPB, 0, f->s>>>(Vin, R, Gout, C, B, f->K);
        else k_contract_f32<false><<<grid_for(f->K * B * C), TPB, 0, f->s>>>(Vin, R, Gout, C, B, f->K);
    }
}

template <class T>
lbm_status forward_impl(fno_ctx *f, const float *x, int B)
{
    const fno_config &c = f->c;
    const int W = c.width;
    T *xa = static_cast<T *>(f->xa);
    k_convert<T><<<grid_for((int64_t)B * c.cin * f->N), TPB, 0, f->s>>>(x, xa, (int64_t)B * c.cin * f->N);
    pw_fwd<T>(f, xa, c.cin, W, f->oP_w, f->oP_b, nullptr, nullptr, f->v[0], false, 0, B);
    for (int l = 0; l < c.layers; ++l) {
        T *vin = static_cast<T *>(f->v[l]);
        dft_fwd<T>(f, vin, f->Vh[l], f->scale_one, B);
        contract(f, f->Vh[l], f->oR[l], f->G, false, B);
        dft_inv<T>(f, f->G, f->spec, f->scale_inv, 0, nullptr, B);
        pw_fwd<T>(f, vin, W, W, f->oW_w[l], f->oW_b[l], f->spec, static_cast<T *>(f->pre[l]), f->v[l + 1], false,
                  l < c.layers - 1 ? 1 : 0, B);
    }
    pw_fwd<T>(f, static_cast<T *>(f->v[c.layers]), W, c.hidden, f->oQ1_w, f->oQ1_b, nullptr, static_cast<T *>(f->hpre),
              f->h, false, 1, B);
    pw_fwd<T>(f, static_cast<T *>(f->h), c.hidden, c.cout, f->oQ2_w, f->oQ2_b, nullptr, nullptr, f->y, true, 0, B);
    return LBM_OK;
}

template <class T>
lbm_status backward_impl(fno_ctx *f, int B)
{
    const fno_config &c = f->c;
    const int W = c.width, H = c.hidden;
    cudaMemsetAsync(f->grads, 0, f->np * sizeof(float), f->s);
    // projection: y = Q2 h + b2, h = GELU(hpre), hpre = Q1 v_L + b1
    outer<T>(f, f->gy, c.cout, static_cast<T *>(f->h), H, f->oQ2_w, f->oQ2_b, B);
    pw_bwd_input<T>(f, f->gy, c.cout, H, f->oQ2_w, static_cast<T *>(f->hpre), f->ghpre, B);
    outer<T>(f, f->ghpre, H, static_cast<T *>(f->v[c.layers]), W, f->oQ1_w, f->oQ1_b, B);
    float *gpre = f->gA, *gnext = f->gB;
    // gradient of v_L = pre_{L-1} (no activation after the last layer)
    pw_bwd_input<T>(f, f->ghpre, H, W, f->oQ1_w, static_cast<const T *>(nullptr), gpre, B);
    for (int l = c.layers - 1; l >= 0; --l) {
        T *vin = static_cast<T *>(f->v[l]);
        outer<T>(f, gpre, W, vin, W, f->oW_w[l], f->oW_b[l], B);
        // spectral branch: gG = (c/N) DFT(gpre); gR = sum_b gG conj(V); gV = gG R^H
        dft_fwd<float>(f, gpre, f->gG, f->scale_inv, B);
        k_grad_R<<<grid_for(f->K * W * W), TPB, 0, f->s>>>(f->gG, f->Vh[l],
                                                           reinterpret_cast<float2 *>(f->grads + f->oR[l]), W, B, f->K);
        contract(f, f->gG, f->oR[l], f->gVh, true, B);
        // gv_l = W_l^T gpre + adjoint DFT(gV), times gelu'(pre_{l-1}) for l > 0
        pw_bwd_input<T>(f, gpre, W, W, f->oW_w[l], static_cast<const T *>(nullptr), gnext, B);
        const T *pre_prev = l > 0 ? static_cast<T *>(f->pre[l - 1]) : nullptr;
        dft_inv<T>(f, f->gVh, gnext, f->scale_one, 1, pre_prev, B);
        std::swap(gpre, gnext);
    }
    outer<T>(f, gpre, W, static_cast<T *>(f->xa), c.cin, f->oP_w, f->oP_b, B);
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
        st = c.act_bf16 ? forward_impl<__nv_bfloat16>(f, f->xin, B) : forward_impl<float>(f, f->xin, B);
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

extern "C" const char *fno_last_error(const fno_ctx *f) { return f ? f->err.c_str() : g_fno_err.c_str(); }
