// fno_umma.cu -- the forward x stage of the FNO transforms on the fifth-
// generation tensor cores: tcgen05.mma with the accumulator in tensor memory
// (TMEM), the row tiles brought into shared memory by the tensor-memory-
// access unit (cp.async.bulk.tensor with a 128-byte-swizzled tensor map).
//
// The stage is the dense contraction A[r][n] = sum_x rows[r][x] T[x][n] of the
// real rows (BF16 activations, nx = 128 samples) against the twiddle table of
// 32 retained x modes, T[x][2j + p] = (p ? Im : Re) exp(-i 2 pi k_j x / nx).
// One tcgen05.mma shape serves the whole tile: M = 128 rows, N = 128, K = 16,
// eight instructions over the 128 samples.  The N = 128 columns are the 64
// reals of the table as BF16 hi parts followed by their lo parts
// (lo = bf16(t - hi)), so that the epilogue adds the two halves and the result
// keeps about 2^-16 relative error, as the mma.sync stage does (BF16 rows are
// exact).  Both operands are K-major with the 128-byte swizzle: 64-sample
// panels of 128-byte rows, 8-row atoms 1024 bytes apart.
//
// A persistent CTA of four warps takes tiles tile = blockIdx.x, + gridDim.x,
// ...: thread 0 issues the tensor-map loads (two 16 KB panels per tile, into
// one of two stages, the next tile's load in flight while the current tile is
// multiplied and written) and the MMAs, whose completion tcgen05.commit
// signals on an mbarrier; then each warp reads its 32 accumulator lanes
// (tcgen05.ld 32x32b) and stores its rows.  Every wait is bounded: after
// about a second the CTA records a status code, waits (bounded again) for the
// loads it issued, frees its tensor memory and returns.
#include <cstdint>
#include <cstring>
#include <string>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fno_umma.h"

namespace {

constexpr int UM_ROWS = 128;                 // M: rows per tile
constexpr uint32_t UM_PANEL = 128 * 128;     // one 64-sample panel of 128 rows (bytes)
constexpr uint32_t UM_TILE = 2 * UM_PANEL;   // a tile's rows (128 samples)
constexpr uint32_t UM_TCOLS = 128;           // TMEM columns (the FP32 accumulator, N = 128)
constexpr long long UM_WAIT_CYCLES = 2000000000LL;   // about a second at the SM clock

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
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

// Wait for phase `parity` of the barrier, giving up after UM_WAIT_CYCLES.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > UM_WAIT_CYCLES) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand with the 128-byte
// swizzle: start address >> 4 (bits 0-13), leading-dimension offset
// (unused by this layout; 16 bytes), stride between 8-row atoms 1024 bytes
// (bits 32-45), descriptor version 1 (bit 46), swizzle mode 2 = 128 bytes
// (bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
constexpr uint32_t UM_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem), "l"(a), "l"(b), "r"(UM_IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__global__ void __launch_bounds__(128, 1) k_dftx_fwd_umma(const __grid_constant__ CUtensorMap rows, const float2 *twx,
                                                          float2 *out, int64_t R, int *status)
{
    extern __shared__ unsigned char um_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(um_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sa = sm;                                   // two stages of a tile's rows
    unsigned char *sb = sm + 2 * UM_TILE;                     // the twiddle operand
    uint64_t *bars = reinterpret_cast<uint64_t *>(sb + UM_TILE);   // full[0], full[1], done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // B: row n of 128 samples, n < 64 the hi parts of T[.][n], n >= 64 the lo
    // parts of T[.][n - 64]; sample x in panel x / 64, 16-byte chunk
    // (x % 64) / 8 stored at chunk ^ (n % 8)
    for (int idx = threadIdx.x; idx < 128 * 128; idx += blockDim.x) {
        const int n = idx >> 7, x = idx & 127;
        const int nn = n & 63;
        const float2 t = twx[x * 32 + (nn >> 1)];
        const float v = (nn & 1) ? t.y : t.x;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 val = n < 64 ? hi : __float2bfloat16_rn(v - __bfloat162float(hi));
        const int xi = x & 63;
        *reinterpret_cast<__nv_bfloat16 *>(sb + (x >> 6) * UM_PANEL + n * 128 + ((((xi >> 3) ^ (n & 7)) & 7) << 4) +
                                           (xi & 7) * 2) = val;
    }
    if (threadIdx.x == 0) {
        mbar_init(saddr(&bars[0]), 1);
        mbar_init(saddr(&bars[1]), 1);
        mbar_init(saddr(&bars[2]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tslot)),
                     "r"(UM_TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    // the twiddle operand, written by the threads, is read by the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;

    const int64_t ntiles = (R + UM_ROWS - 1) / UM_ROWS;
    int pending[2] = {0, 0};                                  // stage has a load in flight (thread 0)
    uint32_t nload[2] = {0, 0};                               // loads issued into each stage
    auto issue = [&](int64_t tile, int s) {
        const uint32_t bar = saddr(&bars[s]);
        mbar_expect_tx(bar, UM_TILE);
        const uint32_t dst = saddr(sa + s * UM_TILE);
        tma_load_2d(dst, &rows, 0, (int)(tile * UM_ROWS), bar);
        tma_load_2d(dst + UM_PANEL, &rows, 64, (int)(tile * UM_ROWS), bar);
        pending[s] = 1;
        ++nload[s];
    };
    if (threadIdx.x == 0 && (int64_t)blockIdx.x < ntiles) issue(blockIdx.x, 0);
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int s = it & 1;
        if (threadIdx.x == 0) {
            const int64_t nxt = tile + gridDim.x;
            if (nxt < ntiles) issue(nxt, s ^ 1);
            if (!mbar_wait(saddr(&bars[s]), (it >> 1) & 1)) {
                atomicExch(status, 1);                        // operand load timed out
                *abort_flag = 1;
            } else {
                pending[s] = 0;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a0 = saddr(sa + s * UM_TILE), b0 = saddr(sb);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t off = (k >> 2) * UM_PANEL + (k & 3) * 32;
                    umma(tmem, sdesc(a0 + off), sdesc(b0 + off), k > 0 ? 1u : 0u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 saddr(&bars[2]))
                             : "memory");
            }
        }
        __syncthreads();
        if (*abort_flag) break;
        if (!mbar_wait(saddr(&bars[2]), it & 1)) {
            atomicExch(status, 2);                            // the products did not complete
            *abort_flag = 1;
        }
        __syncthreads();
        if (*abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // warp w holds accumulator lanes (tile rows) 32 w .. 32 w + 31
        const int64_t row = tile * UM_ROWS + warp * 32 + lane;
        const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float h[16], l[16];
            tmem_ld16(base + c, h);
            tmem_ld16(base + 64 + c, l);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row < R) {
                float4 *dst = reinterpret_cast<float4 *>(out + row * 32 + c / 2);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    dst[q] = make_float4(h[4 * q] + l[4 * q], h[4 * q + 1] + l[4 * q + 1], h[4 * q + 2] + l[4 * q + 2],
                                         h[4 * q + 3] + l[4 * q + 3]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();                                      // the accumulator is free for the next tile
    }
    // loads still in flight (after an abort) must land before the CTA's
    // shared memory goes away
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s)
            if (pending[s] && !mbar_wait(saddr(&bars[s]), (nload[s] - 1) & 1)) atomicExch(status, 3);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UM_TCOLS) : "memory");
}

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

}  // namespace

size_t umma_dftx_smem() { return 1024 + 3 * (size_t)UM_TILE + 64; }

bool umma_make_row_map(void *map, const void *rows, int64_t R)
{
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || !rows || R < 1 || (reinterpret_cast<uintptr_t>(rows) & 15u)) return false;
    const cuuint64_t dims[2] = {128, (cuuint64_t)R};
    const cuuint64_t strides[1] = {256};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t estr[2] = {1, 1};
    CUtensorMap m;
    const CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(rows), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    std::memcpy(map, &m, sizeof m);
    return true;
}

bool umma_set_smem()
{
    return cudaFuncSetAttribute(k_dftx_fwd_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)umma_dftx_smem()) ==
           cudaSuccess;
}

void umma_dftx_fwd(const void *map, const float2 *twx, float2 *out, int64_t R, int *status, int blocks,
                   cudaStream_t s)
{
    CUtensorMap m;
    std::memcpy(&m, map, sizeof m);
    k_dftx_fwd_umma<<<blocks, 128, umma_dftx_smem(), s>>>(m, twx, out, R, status);
}
