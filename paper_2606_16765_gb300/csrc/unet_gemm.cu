// unet_gemm.cu -- the U-Net's 3x3x3 convolutions on the fifth-generation
// tensor cores (tcgen05.mma, kind::f16, BF16 operands, FP32 accumulators in
// tensor memory), fed by tensor-map copies (cp.async.bulk.tensor).
//
// Forward and input gradient: an implicit GEMM with M = 128 output cells (a
// box of the channel-last activation: bx x by x bz cells x bb samples), N =
// output channels (<= 256 per tile) and K = 27 taps x input channels.  For
// tap (dz, dy, dx) the A tile is the same box shifted by (dz-1, dy-1, dx-1):
// one 5-D tensor-map copy whose out-of-range cells arrive as zeros, which is
// the convolution's zero padding.  The B tile is the tap's [N][K-chunk] slice
// of the weights.  Both operands are K-major, 64 channels per 128-byte
// swizzled row (or 32 channels per 64-byte row when the channel count is not a
// multiple of 64).  The input gradient is the same product with the weights
// transposed and the taps reversed.
//
// Weight gradient: G[(tap, i)][o] = sum over cells of X[cell + tap - 1][i] *
// GZ[cell][o]: M = 128 (tap, input-channel) rows taken as four 32-channel
// atoms, N = output channels, K = cells.  Here both operands are MN-major: the
// same channel-last boxes, 64-byte rows of 32 channels, consecutive cells
// the contraction index.  The cell range is split over CTAs, each adding its
// FP32 tile into G atomically.
//
// A persistent CTA of six warps: warp 0 issues the copies into a ring of
// stages, warp 1 (after allocating tensor memory) issues the MMAs and commits
// each stage back to the producer, warps 2-5 read the accumulator (two
// accumulators alternate, so the epilogue of one tile overlaps the products of
// the next) and write the outputs.  Every mbarrier wait is bounded (about a
// second): on expiry the CTA records a status code, every role stops, the
// copies in flight and the issued products are waited for (bounded again),
// tensor memory is freed and the kernel returns.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "unet_gemm.h"

namespace unet {
namespace {

constexpr int NT = 192;                                // six warps
constexpr long long WAIT_CYCLES = 2000000000LL;        // about a second at the SM clock
constexpr size_t SMEM_MAX = 232448;                    // 227 KB
constexpr size_t SMEM_ONE_CTA = 120 * 1024;            // at least this much: one CTA per SM

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity`; false after WAIT_CYCLES or, when
// `abort` is given, as soon as another role has set it.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int *abort)
{
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (abort && *abort) return false;
        if (clock64() - t0 > WAIT_CYCLES) return false;
    }
    return true;
}

__device__ __forceinline__ void fail(volatile int *abort, int *status, int code)
{
    *abort = 1;
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ void tma5(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                     uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma3(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor, K-major, swizzled rows of `row_bytes`
// (128: swizzle mode 2; 64: mode 4); 8-row atoms row_bytes * 8 apart (stride
// field), leading field unused by these layouts, version 1 (bit 46).
__device__ __forceinline__ uint64_t desc_k(uint32_t addr, uint32_t row_bytes)
{
    const uint64_t mode = row_bytes == 128 ? 2 : 4;
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((row_bytes * 8) >> 4) << 32) |
           ((uint64_t)1 << 46) | (mode << 61);
}

// MN-major with the 64-byte swizzle: atoms of 32 MN elements x 8 K rows
// (512 bytes); `lbo` bytes between atoms along MN (leading field), 512 bytes
// between 8-row groups along K (stride field).
__device__ __forceinline__ uint64_t desc_mn64(uint32_t addr, uint32_t lbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void store16(float *dst, const float *v)
{
    float4 *d = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ void store16(__nv_bfloat16 *dst, const float *v)
{
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t *>(&h);
    }
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

struct Box {
    int x0, y0, z0, b0;
};

__device__ __forceinline__ Box box_origin(int64_t mt, int tx, int ty, int tz, int bx, int by, int bz, int bb)
{
    Box o;
    o.x0 = (int)(mt % tx) * bx;
    mt /= tx;
    o.y0 = (int)(mt % ty) * by;
    mt /= ty;
    o.z0 = (int)(mt % tz) * bz;
    o.b0 = (int)(mt / tz) * bb;
    return o;
}

// Shared memory after the 1024-aligned operand ring: barriers, the tensor
// memory address, the abort flag.
struct Ctl {
    uint64_t *full, *empty, *accf, *acce, *drain;
    uint32_t *tslot;
    volatile int *abort;
};

__device__ __forceinline__ Ctl ctl_at(unsigned char *p, int S)
{
    Ctl c;
    uint64_t *b = reinterpret_cast<uint64_t *>(p);
    c.full = b;
    c.empty = b + S;
    c.accf = b + 2 * S;
    c.acce = b + 2 * S + 2;
    c.drain = b + 2 * S + 4;
    c.tslot = reinterpret_cast<uint32_t *>(b + 2 * S + 5);
    c.abort = reinterpret_cast<volatile int *>(c.tslot + 1);
    return c;
}

__device__ __forceinline__ void ctl_init(const Ctl &c, int S, uint32_t tmem_cols)
{
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(saddr(&c.full[s]), 1);
            mbar_init(saddr(&c.empty[s]), 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(saddr(&c.accf[q]), 1);
            mbar_init(saddr(&c.acce[q]), 128);
        }
        mbar_init(saddr(c.drain), 1);
        *c.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(c.tslot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
}

__device__ __forceinline__ void ctl_finish(const Ctl &c, uint32_t tmem, uint32_t tmem_cols)
{
    tc_before();
    __syncthreads();
    tc_after();
    if ((threadIdx.x >> 5) == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// The producer's copies still in flight must land before the CTA exits.
__device__ __forceinline__ void drain_loads(const Ctl &c, uint32_t issued, int S, int *status)
{
    for (uint32_t j = issued > (uint32_t)S ? issued - S : 0; j < issued; ++j)
        if (!wait_bar(saddr(&c.full[j % S]), (j / S) & 1, nullptr)) atomicCAS(status, 0, 3);
}

// Every product issued must complete before tensor memory is freed.
__device__ __forceinline__ void drain_mma(const Ctl &c, int *status)
{
    commit(saddr(c.drain));
    if (!wait_bar(saddr(c.drain), 0, nullptr)) atomicCAS(status, 0, 4);
}

// ---------------------------------------------------------------------------
// forward / input-gradient convolution
// ---------------------------------------------------------------------------
template <int CK, class TO>
__global__ void __launch_bounds__(NT, 1) k_conv_umma(const __grid_constant__ CUtensorMap amap,
                                                     const __grid_constant__ CUtensorMap wmap, const ConvArgs a,
                                                     TO *__restrict__ out, int *status)
{
    extern __shared__ unsigned char raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    const int S = a.stages;
    unsigned char *sA = sm;
    unsigned char *sB = sm + (size_t)S * a.a_bytes;
    const Ctl c = ctl_at(sB + (size_t)S * a.b_bytes, S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ctl_init(c, S, a.tmem_cols);
    const uint32_t tmem = *c.tslot;
    const int nk = a.ntaps * a.kchunks;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; ok && w < a.nwork; w += gridDim.x) {
                const Box o = box_origin(w / a.nntiles, a.tx, a.ty, a.tz, a.bx, a.by, a.bz, a.bb);
                const int n0 = (int)(w % a.nntiles) * a.ntile;
                for (int q = 0; q < nk; ++q) {
                    const int tap = q / a.kchunks, kc = q % a.kchunks;
                    const int dz = a.ntaps == 1 ? 1 : tap / 9, dy = a.ntaps == 1 ? 1 : (tap / 3) % 3,
                              dx = a.ntaps == 1 ? 1 : tap % 3;
                    const uint32_t s = it % S;
                    if (!wait_bar(saddr(&c.empty[s]), ((it / S) & 1) ^ 1, c.abort)) {
                        fail(c.abort, status, 1);
                        ok = false;
                        break;
                    }
                    const uint32_t fb = saddr(&c.full[s]);
                    mbar_expect_tx(fb, a.a_bytes + a.b_bytes);
                    tma5(saddr(sA + (size_t)s * a.a_bytes), &amap, kc * CK, o.x0 + dx - 1, o.y0 + dy - 1,
                         o.z0 + dz - 1, o.b0, fb);
                    tma3(saddr(sB + (size_t)s * a.b_bytes), &wmap, kc * CK, n0, tap, fb);
                    ++it;
                }
            }
            drain_loads(c, it, S, status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, tc = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; ok && w < a.nwork; w += gridDim.x, ++tc) {
                const uint32_t acc = tc & 1;
                if (!wait_bar(saddr(&c.acce[acc]), ((tc >> 1) & 1) ^ 1, c.abort)) {
                    fail(c.abort, status, 2);
                    break;
                }
                tc_after();
                const uint32_t d = tmem + acc * (uint32_t)a.ntile;
                for (int q = 0; q < nk; ++q) {
                    const uint32_t s = it % S;
                    if (!wait_bar(saddr(&c.full[s]), (it / S) & 1, c.abort)) {
                        fail(c.abort, status, 2);
                        ok = false;
                        break;
                    }
                    tc_after();
                    const uint64_t ad = desc_k(saddr(sA + (size_t)s * a.a_bytes), CK * 2);
                    const uint64_t bd = desc_k(saddr(sB + (size_t)s * a.b_bytes), CK * 2);
#pragma unroll
                    for (int k = 0; k < CK / 16; ++k)      // K = 16 per product: 32 bytes along the row
                        umma(d, ad + 2 * k, bd + 2 * k, a.idesc, (q > 0 || k > 0) ? 1u : 0u);
                    commit(saddr(&c.empty[s]));
                    ++it;
                }
                if (ok) commit(saddr(&c.accf[acc]));
            }
            drain_mma(c, status);
        }
    } else {
        const int quad = warp & 3;                 // tensor-memory lanes 32 quad .. 32 quad + 31
        const int row = quad * 32 + lane;
        const int rx = row % a.bx, ry = (row / a.bx) % a.by, rz = (row / (a.bx * a.by)) % a.bz,
                  rb = row / (a.bx * a.by * a.bz);
        uint32_t tc = 0;
        for (int64_t w = blockIdx.x; w < a.nwork; w += gridDim.x, ++tc) {
            const uint32_t acc = tc & 1;
            if (!wait_bar(saddr(&c.accf[acc]), (tc >> 1) & 1, c.abort)) {
                fail(c.abort, status, 5);
                break;
            }
            tc_after();
            const Box o = box_origin(w / a.nntiles, a.tx, a.ty, a.tz, a.bx, a.by, a.bz, a.bb);
            const int n0 = (int)(w % a.nntiles) * a.ntile;
            const int b = o.b0 + rb;
            const bool valid = b < a.B;
            TO *dst = out + ((((int64_t)(valid ? b : 0) * a.Z + o.z0 + rz) * a.Y + o.y0 + ry) * a.X + o.x0 + rx) * a.ldo +
                      a.ooff + n0;
            const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + acc * (uint32_t)a.ntile;
            for (int cc = 0; cc < a.ntile; cc += 16) {
                float v[16];
                tmem_ld16(base + cc, v);
                if (valid) store16(dst + cc, v);
            }
            tc_before();
            mbar_arrive(saddr(&c.acce[acc]));
        }
    }
    ctl_finish(c, tmem, a.tmem_cols);
}

// ---------------------------------------------------------------------------
// weight gradient
// ---------------------------------------------------------------------------
struct WItem {
    int mt, nt;
    int64_t c0, c1;
};

__device__ __forceinline__ WItem witem(const WgradArgs &a, int64_t w)
{
    WItem it;
    const int ks = (int)(w % a.ksplit);
    const int64_t r = w / a.ksplit;
    it.nt = (int)(r % a.nntiles);
    it.mt = (int)(r / a.nntiles);
    it.c0 = a.nchunks * ks / a.ksplit;
    it.c1 = a.nchunks * (ks + 1) / a.ksplit;
    return it;
}

__global__ void __launch_bounds__(NT, 1) k_wgrad_umma(const __grid_constant__ CUtensorMap xmap,
                                                      const __grid_constant__ CUtensorMap gmap, const WgradArgs a,
                                                      float *__restrict__ g, int *status)
{
    extern __shared__ unsigned char raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    const int S = a.stages;
    unsigned char *sA = sm;
    unsigned char *sB = sm + (size_t)S * a.a_bytes;
    const Ctl c = ctl_at(sB + (size_t)S * a.b_bytes, S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ctl_init(c, S, a.tmem_cols);
    const uint32_t tmem = *c.tslot;
    constexpr uint32_t ATOM = 128 * 64;            // 128 cells x 32 channels

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; ok && w < a.nwork; w += gridDim.x) {
                const WItem wi = witem(a, w);
                for (int64_t ch = wi.c0; ch < wi.c1; ++ch) {
                    const Box o = box_origin(ch, a.tx, a.ty, a.tz, a.bx, a.by, a.bz, a.bb);
                    const uint32_t s = it % S;
                    if (!wait_bar(saddr(&c.empty[s]), ((it / S) & 1) ^ 1, c.abort)) {
                        fail(c.abort, status, 1);
                        ok = false;
                        break;
                    }
                    const uint32_t fb = saddr(&c.full[s]);
                    mbar_expect_tx(fb, a.a_bytes + a.b_bytes);
                    for (int at = 0; at < 4; ++at) {
                        const int ga = wi.mt * 4 + at;
                        // rows past 27 * cin load a valid tap and are discarded
                        const int tap = min(ga / a.cin_blocks, 26), cb = ga / a.cin_blocks > 26 ? 0 : ga % a.cin_blocks;
                        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                        tma5(saddr(sA + (size_t)s * a.a_bytes + at * ATOM), &xmap, cb * 32, o.x0 + dx - 1,
                             o.y0 + dy - 1, o.z0 + dz - 1, o.b0, fb);
                    }
                    for (int j = 0; j < a.ntile / 32; ++j)
                        tma5(saddr(sB + (size_t)s * a.b_bytes + j * ATOM), &gmap, wi.nt * a.ntile + j * 32, o.x0, o.y0,
                             o.z0, o.b0, fb);
                    ++it;
                }
            }
            drain_loads(c, it, S, status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, tc = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; ok && w < a.nwork; w += gridDim.x) {
                const WItem wi = witem(a, w);
                if (wi.c1 <= wi.c0) continue;
                const uint32_t acc = tc & 1;
                if (!wait_bar(saddr(&c.acce[acc]), ((tc >> 1) & 1) ^ 1, c.abort)) {
                    fail(c.abort, status, 2);
                    break;
                }
                tc_after();
                const uint32_t d = tmem + acc * (uint32_t)a.ntile;
                for (int64_t ch = wi.c0; ch < wi.c1; ++ch) {
                    const uint32_t s = it % S;
                    if (!wait_bar(saddr(&c.full[s]), (it / S) & 1, c.abort)) {
                        fail(c.abort, status, 2);
                        ok = false;
                        break;
                    }
                    tc_after();
                    const uint32_t a0 = saddr(sA + (size_t)s * a.a_bytes), b0 = saddr(sB + (size_t)s * a.b_bytes);
#pragma unroll
                    for (int k = 0; k < 8; ++k)            // 16 cells (two 8-row groups) per product
                        umma(d, desc_mn64(a0 + k * 1024, ATOM), desc_mn64(b0 + k * 1024, ATOM), a.idesc,
                             (ch > wi.c0 || k > 0) ? 1u : 0u);
                    commit(saddr(&c.empty[s]));
                    ++it;
                }
                if (ok) commit(saddr(&c.accf[acc]));
                ++tc;
            }
            drain_mma(c, status);
        }
    } else {
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        uint32_t tc = 0;
        for (int64_t w = blockIdx.x; w < a.nwork; w += gridDim.x) {
            const WItem wi = witem(a, w);
            if (wi.c1 <= wi.c0) continue;
            const uint32_t acc = tc & 1;
            if (!wait_bar(saddr(&c.accf[acc]), (tc >> 1) & 1, c.abort)) {
                fail(c.abort, status, 5);
                break;
            }
            tc_after();
            const int m = wi.mt * 128 + row;
            float *dst = g + (int64_t)(m < a.m_total ? m : 0) * a.ldg + wi.nt * a.ntile;
            const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + acc * (uint32_t)a.ntile;
            for (int cc = 0; cc < a.ntile; cc += 16) {
                float v[16];
                tmem_ld16(base + cc, v);
                if (m < a.m_total) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        atomicAdd(reinterpret_cast<float4 *>(dst + cc) + q,
                                  make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
                }
            }
            tc_before();
            mbar_arrive(saddr(&c.acce[acc]));
            ++tc;
        }
    }
    ctl_finish(c, tmem, a.tmem_cols);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

bool encode(unsigned char *dst, int rank, const void *base, const cuuint64_t *dims, const cuuint64_t *strides,
            const cuuint32_t *box, CUtensorMapSwizzle sw)
{
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15u)) return false;
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUtensorMap m;
    const CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void *>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    std::memcpy(dst, &m, sizeof m);
    return true;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// A tile of 128 cells: whole rows of x first, then rows of y, planes of z,
// samples (grids with power-of-two sides).
void box_for(int X, int Y, int Z, int &bx, int &by, int &bz, int &bb)
{
    bx = std::min(X, 128);
    by = std::min(Y, 128 / bx);
    bz = std::min(Z, 128 / (bx * by));
    bb = 128 / (bx * by * bz);
}

int pick_ntile(int N)
{
    for (int t = std::min(N, 256); t >= 32; t -= 32)
        if (N % t == 0) return t;
    return 0;
}

uint32_t tmem_cols_for(int ntile)
{
    uint32_t c = 32;
    while (c < 2u * (uint32_t)ntile) c <<= 1;
    return c;
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, M = 128.
uint32_t idesc_for(int ntile, bool a_mn, bool b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(ntile >> 3) << 17) | ((128u >> 4) << 24);
}

size_t ctl_bytes(int S) { return (size_t)(2 * S + 5) * 8 + 16; }

}  // namespace

bool conv_plan(ConvPlan &p, const void *act, int lda, int k, int X, int Y, int Z, int B, const void *w, int N,
               int ntaps, int ldo, int ooff, int sms, const char **err)
{
    auto bad = [&](const char *m) {
        if (err) *err = m;
        return false;
    };
    if (!pow2(X) || !pow2(Y) || !pow2(Z) || B < 1) return bad("conv: grid sides must be powers of two");
    if (k < 32 || k % 32 || lda < k || lda % 8) return bad("conv: input channels must be a multiple of 32");
    if (N < 32 || N % 32 || ooff % 16 || ldo % 8 || ldo < ooff + N) return bad("conv: output channels");
    if (ntaps != 1 && ntaps != 27) return bad("conv: taps must be 1 or 27");
    ConvArgs &a = p.a;
    std::memset(&a, 0, sizeof a);
    p.ck = (k % 64 == 0) ? 64 : 32;
    a.X = X; a.Y = Y; a.Z = Z; a.B = B;
    box_for(X, Y, Z, a.bx, a.by, a.bz, a.bb);
    a.tx = X / a.bx; a.ty = Y / a.by; a.tz = Z / a.bz; a.tb = (B + a.bb - 1) / a.bb;
    a.ntaps = ntaps;
    a.kchunks = k / p.ck;
    a.ntile = pick_ntile(N);
    a.nntiles = N / a.ntile;
    a.ldo = ldo; a.ooff = ooff;
    a.a_bytes = 128u * p.ck * 2;
    a.b_bytes = (uint32_t)a.ntile * p.ck * 2;
    a.stages = (int)std::min<size_t>(8, (SMEM_MAX - 2048 - ctl_bytes(8)) / (a.a_bytes + a.b_bytes));
    if (a.stages < 2) return bad("conv: tile does not fit in shared memory");
    a.nwork = (int64_t)a.tx * a.ty * a.tz * a.tb * a.nntiles;
    a.idesc = idesc_for(a.ntile, false, false);
    a.tmem_cols = tmem_cols_for(a.ntile);
    p.smem = std::max(SMEM_ONE_CTA, 1024 + (size_t)a.stages * (a.a_bytes + a.b_bytes) + ctl_bytes(a.stages));
    p.grid = (int)std::min<int64_t>(a.nwork, std::max(1, sms));
    const CUtensorMapSwizzle sw = p.ck == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    const cuuint64_t adims[5] = {(cuuint64_t)lda, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)Z, (cuuint64_t)B};
    const cuuint64_t astr[4] = {(cuuint64_t)lda * 2, (cuuint64_t)lda * 2 * X, (cuuint64_t)lda * 2 * X * Y,
                                (cuuint64_t)lda * 2 * X * Y * Z};
    const cuuint32_t abox[5] = {(cuuint32_t)p.ck, (cuuint32_t)a.bx, (cuuint32_t)a.by, (cuuint32_t)a.bz,
                                (cuuint32_t)a.bb};
    if (!encode(p.amap, 5, act, adims, astr, abox, sw)) return bad("conv: activation tensor map rejected");
    const cuuint64_t wdims[3] = {(cuuint64_t)k, (cuuint64_t)N, (cuuint64_t)ntaps};
    const cuuint64_t wstr[2] = {(cuuint64_t)k * 2, (cuuint64_t)k * 2 * N};
    const cuuint32_t wbox[3] = {(cuuint32_t)p.ck, (cuuint32_t)a.ntile, 1};
    if (!encode(p.wmap, 3, w, wdims, wstr, wbox, sw)) return bad("conv: weight tensor map rejected");
    return true;
}

void conv_launch(const ConvPlan &p, void *out, bool out_f32, int *status, cudaStream_t s)
{
    CUtensorMap am, wm;
    std::memcpy(&am, p.amap, sizeof am);
    std::memcpy(&wm, p.wmap, sizeof wm);
    if (p.ck == 64) {
        if (out_f32)
            k_conv_umma<64, float><<<p.grid, NT, p.smem, s>>>(am, wm, p.a, static_cast<float *>(out), status);
        else
            k_conv_umma<64, __nv_bfloat16><<<p.grid, NT, p.smem, s>>>(am, wm, p.a, static_cast<__nv_bfloat16 *>(out),
                                                                      status);
    } else {
        if (out_f32)
            k_conv_umma<32, float><<<p.grid, NT, p.smem, s>>>(am, wm, p.a, static_cast<float *>(out), status);
        else
            k_conv_umma<32, __nv_bfloat16><<<p.grid, NT, p.smem, s>>>(am, wm, p.a, static_cast<__nv_bfloat16 *>(out),
                                                                      status);
    }
}

bool wgrad_plan(WgradPlan &p, const void *x, int ldx, int cin, const void *gz, int ldgz, int N, int X, int Y, int Z,
                int B, int sms, const char **err)
{
    auto bad = [&](const char *m) {
        if (err) *err = m;
        return false;
    };
    if (!pow2(X) || !pow2(Y) || !pow2(Z) || B < 1) return bad("wgrad: grid sides must be powers of two");
    if (cin < 32 || cin % 32 || ldx < cin || ldx % 8) return bad("wgrad: input channels must be a multiple of 32");
    if (N < 32 || N % 32 || ldgz < N || ldgz % 8) return bad("wgrad: output channels must be a multiple of 32");
    WgradArgs &a = p.a;
    std::memset(&a, 0, sizeof a);
    a.X = X; a.Y = Y; a.Z = Z; a.B = B;
    box_for(X, Y, Z, a.bx, a.by, a.bz, a.bb);
    a.tx = X / a.bx; a.ty = Y / a.by; a.tz = Z / a.bz; a.tb = (B + a.bb - 1) / a.bb;
    a.cin_blocks = cin / 32;
    a.m_total = 27 * cin;
    a.mtiles = (a.m_total + 127) / 128;
    a.ntile = pick_ntile(N);
    a.nntiles = N / a.ntile;
    a.nchunks = (int64_t)a.tx * a.ty * a.tz * a.tb;
    const int64_t items = (int64_t)a.mtiles * a.nntiles;
    int64_t ks = (2 * (int64_t)std::max(1, sms) + items - 1) / items;
    ks = std::min<int64_t>(ks, std::max<int64_t>(1, a.nchunks / 4));
    a.ksplit = (int)std::max<int64_t>(1, ks);
    a.nwork = items * a.ksplit;
    a.a_bytes = 4u * 128 * 64;
    a.b_bytes = (uint32_t)(a.ntile / 32) * 128 * 64;
    a.stages = (int)std::min<size_t>(6, (SMEM_MAX - 2048 - ctl_bytes(6)) / (a.a_bytes + a.b_bytes));
    if (a.stages < 2) return bad("wgrad: tile does not fit in shared memory");
    a.idesc = idesc_for(a.ntile, true, true);
    a.tmem_cols = tmem_cols_for(a.ntile);
    a.ldg = N;
    p.smem = std::max(SMEM_ONE_CTA, 1024 + (size_t)a.stages * (a.a_bytes + a.b_bytes) + ctl_bytes(a.stages));
    p.grid = (int)std::min<int64_t>(a.nwork, std::max(1, sms));
    const cuuint32_t box[5] = {32, (cuuint32_t)a.bx, (cuuint32_t)a.by, (cuuint32_t)a.bz, (cuuint32_t)a.bb};
    const cuuint64_t xd[5] = {(cuuint64_t)ldx, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)Z, (cuuint64_t)B};
    const cuuint64_t xs[4] = {(cuuint64_t)ldx * 2, (cuuint64_t)ldx * 2 * X, (cuuint64_t)ldx * 2 * X * Y,
                              (cuuint64_t)ldx * 2 * X * Y * Z};
    if (!encode(p.xmap, 5, x, xd, xs, box, CU_TENSOR_MAP_SWIZZLE_64B)) return bad("wgrad: input tensor map rejected");
    const cuuint64_t gd[5] = {(cuuint64_t)ldgz, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)Z, (cuuint64_t)B};
    const cuuint64_t gs[4] = {(cuuint64_t)ldgz * 2, (cuuint64_t)ldgz * 2 * X, (cuuint64_t)ldgz * 2 * X * Y,
                              (cuuint64_t)ldgz * 2 * X * Y * Z};
    if (!encode(p.gmap, 5, gz, gd, gs, box, CU_TENSOR_MAP_SWIZZLE_64B)) return bad("wgrad: gradient tensor map rejected");
    return true;
}

void wgrad_launch(const WgradPlan &p, float *g, int *status, cudaStream_t s)
{
    CUtensorMap xm, gm;
    std::memcpy(&xm, p.xmap, sizeof xm);
    std::memcpy(&gm, p.gmap, sizeof gm);
    k_wgrad_umma<<<p.grid, NT, p.smem, s>>>(xm, gm, p.a, g, status);
}

bool gemm_set_attrs()
{
    static int done = 0;
    if (done) return done > 0;
    const int v = (int)SMEM_MAX;
    const auto a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const bool ok = cudaFuncSetAttribute(k_conv_umma<64, float>, a, v) == cudaSuccess &&
                    cudaFuncSetAttribute(k_conv_umma<64, __nv_bfloat16>, a, v) == cudaSuccess &&
                    cudaFuncSetAttribute(k_conv_umma<32, float>, a, v) == cudaSuccess &&
                    cudaFuncSetAttribute(k_conv_umma<32, __nv_bfloat16>, a, v) == cudaSuccess &&
                    cudaFuncSetAttribute(k_wgrad_umma, a, v) == cudaSuccess;
    done = ok ? 1 : -1;
    return ok;
}

}  // namespace unet
