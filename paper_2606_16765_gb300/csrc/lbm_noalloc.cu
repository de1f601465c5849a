// lbm_noalloc.cu -- mass and momentum totals of a caller-owned population
// array without allocating any device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// totals: a monitor thread that checks conservation between the steps of a
// solver it does not own (cudaMalloc/cudaFree may synchronise the whole
// device and stall that solver), or an application whose device memory is
// owned entirely by a host framework's pool (a side allocation can fail or
// fragment it).  This entry point serves them: its only scratch is a
// fixed-size array compiled into the library, g_totals_scratch below.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (512 KiB + 32 B) until the process exits.  Host code must
// not pass its name to a kernel: on the host the name is only a stand-in, not
// a device address.  The first call on each device looks the device address
// up with cudaGetSymbolAddress while that device is current and caches it.
// All calls share the array and it keeps the last call's contents; every
// partial slot a call reads is written by the same call first, so nothing
// needs clearing, but calls that overlap on the GPU race.
#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {
void set_global_error(const std::string &m);   // lbm_api.cu
}

using namespace lbm;

namespace {
constexpr int NA_THREADS = 256;
constexpr int64_t NA_CELLS_PER_BLOCK = 65536;
constexpr int NA_MAX_BLOCKS = 16384;
constexpr int64_t NA_MAX_CELLS = NA_CELLS_PER_BLOCK * NA_MAX_BLOCKS;   // 2^30 cells
constexpr int NA_MAX_DEVICES = 64;
}  // namespace

// 4 partial sums per block of the first pass, then the 4 totals.
static __device__ __align__(256) double g_totals_scratch[4 * NA_MAX_BLOCKS + 4];

namespace {

// Pass 1: block b sums cells [b * NA_CELLS_PER_BLOCK, (b + 1) * NA_CELLS_PER_BLOCK)
// in a fixed order and writes its 4 partial sums.
template <class S>
__global__ void __launch_bounds__(NA_THREADS) k_na_partial(const S *pdf, int64_t slot, const uint8_t *mask, int64_t n,
                                                           double *scratch)
{
    using T = Store<S>;
    __shared__ double sh[4][NA_THREADS];
    double acc[4] = {0, 0, 0, 0};
    const int64_t begin = (int64_t)blockIdx.x * NA_CELLS_PER_BLOCK;
    const int64_t end = begin + NA_CELLS_PER_BLOCK < n ? begin + NA_CELLS_PER_BLOCK : n;
    for (int64_t c = begin + threadIdx.x; c < end; c += NA_THREADS) {
        if (mask && mask[c]) continue;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double v = (double)T::ld(pdf + (int64_t)i * slot + c);
            acc[0] += v;
            acc[1] += cx_of(i) * v;
            acc[2] += cy_of(i) * v;
            acc[3] += cz_of(i) * v;
        }
    }
    for (int d = 0; d < 4; ++d) sh[d][threadIdx.x] = acc[d];
    __syncthreads();
    for (int h = NA_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int d = 0; d < 4; ++d) sh[d][threadIdx.x] += sh[d][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 4; ++d) scratch[4 * (int64_t)blockIdx.x + d] = sh[d][0];
}

// Pass 2: one block adds the partials in a fixed order into the 4 totals.
__global__ void __launch_bounds__(NA_THREADS) k_na_final(double *scratch, int nblocks)
{
    __shared__ double sh[4][NA_THREADS];
    double acc[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += NA_THREADS)
        for (int d = 0; d < 4; ++d) acc[d] += scratch[4 * b + d];
    for (int d = 0; d < 4; ++d) sh[d][threadIdx.x] = acc[d];
    __syncthreads();
    for (int h = NA_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int d = 0; d < 4; ++d) sh[d][threadIdx.x] += sh[d][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 4; ++d) scratch[4 * NA_MAX_BLOCKS + d] = sh[d][0];
}

std::mutex g_addr_mu;
double *g_addr[NA_MAX_DEVICES] = {};

// Device address of g_totals_scratch on the current device (looked up once
// per device, with that device current).
lbm_status scratch_address(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        set_global_error("lbm_totals_noalloc: no usable current CUDA device");
        return LBM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_totals_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_global_error(std::string("lbm_totals_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return LBM_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return LBM_OK;
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

}  // namespace

extern "C" lbm_status lbm_totals_noalloc(const void *pdf, int32_t storage, int64_t slot_stride,
                                         const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz,
                                         void *cuda_stream, double *out)
{
    if (!pdf || !out || storage < LBM_F64 || storage > LBM_F16C || nx < 1 || ny < 1 || nz < 1) {
        set_global_error("lbm_totals_noalloc: null pointer, unknown storage or empty grid");
        return LBM_ERR_ARG;
    }
    // a host pdf or mask would reach the kernel as an address the GPU may not
    // translate: refuse it here, before anything is launched
    if (!on_device(pdf) || (mask && !on_device(mask))) {
        set_global_error("lbm_totals_noalloc: pdf and mask must be device (or managed) memory");
        return LBM_ERR_ARG;
    }
    const int64_t n = (int64_t)nx * ny * nz;
    if (n > NA_MAX_CELLS) {
        set_global_error("lbm_totals_noalloc: grid of " + std::to_string(n) + " cells exceeds the " +
                         std::to_string(NA_MAX_CELLS) + "-cell capacity of its static scratch");
        return LBM_ERR_ARG;
    }
    if (slot_stride < n) {
        set_global_error("lbm_totals_noalloc: slot_stride is smaller than nx*ny*nz");
        return LBM_ERR_ARG;
    }
    double *scratch = nullptr;
    lbm_status st = scratch_address(&scratch);
    if (st != LBM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nblocks = (int)((n + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    switch (storage) {
    case LBM_F64: k_na_partial<double><<<nblocks, NA_THREADS, 0, s>>>((const double *)pdf, slot_stride, mask, n, scratch); break;
    case LBM_F32: k_na_partial<float><<<nblocks, NA_THREADS, 0, s>>>((const float *)pdf, slot_stride, mask, n, scratch); break;
    case LBM_F16S: k_na_partial<__half><<<nblocks, NA_THREADS, 0, s>>>((const __half *)pdf, slot_stride, mask, n, scratch); break;
    case LBM_BF16S: k_na_partial<__nv_bfloat16><<<nblocks, NA_THREADS, 0, s>>>((const __nv_bfloat16 *)pdf, slot_stride, mask, n, scratch); break;
    default: k_na_partial<F16C><<<nblocks, NA_THREADS, 0, s>>>((const F16C *)pdf, slot_stride, mask, n, scratch); break;
    }
    k_na_final<<<1, NA_THREADS, 0, s>>>(scratch, nblocks);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        if (on_device(out)) {
            e = cudaMemcpyAsync(out, scratch + 4 * NA_MAX_BLOCKS, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        } else {
            e = cudaMemcpyAsync(out, scratch + 4 * NA_MAX_BLOCKS, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
    }
    if (e != cudaSuccess) {
        set_global_error(std::string("lbm_totals_noalloc: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
