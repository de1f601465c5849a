// resample.cu -- cell-centred trilinear resampling of mean fields onto the
// surrogate's grid (App. B: the simulated fields are scaled down to
// 128x64x64 before training).
//
// Output cell o of an axis with n source and m target cells samples the
// source at s = (o + 1/2) n/m - 1/2, clamped to [0, n - 1], linearly between
// floor(s) and floor(s) + 1; the 3D map is the product of the three axes.
// One thread per output value; the source (a few MB per field) stays in L2.
#include <string>

#include "../../include/lbm.h"
#include "sm_count.h"

namespace lbm {
void set_global_error(const std::string &m);   // lbm_api.cu
}

namespace {

struct Axis {
    int i0, i1;
    float t;
};

__device__ __forceinline__ Axis axis_map(int o, int n, int m)
{
    float s = ((float)o + 0.5f) * ((float)n / (float)m) - 0.5f;
    s = fminf(fmaxf(s, 0.f), (float)(n - 1));
    const int i0 = (int)floorf(s);
    return Axis{i0, min(i0 + 1, n - 1), s - (float)i0};
}

// src: [nz][ny][nx][C] (cell-major, layout 0) or [C][nz][ny][nx] (layout 1);
// dst: [C][mz][my][mx].
__global__ void k_resample(const float *src, int nx, int ny, int nz, int C, int layout, float *dst, int mx, int my,
                           int mz)
{
    const int64_t total = (int64_t)C * mz * my * mx;
    const int64_t nxyz = (int64_t)nx * ny * nz;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int ox = (int)(k % mx);
        const int oy = (int)((k / mx) % my);
        const int oz = (int)((k / ((int64_t)mx * my)) % mz);
        const int c = (int)(k / ((int64_t)mx * my * mz));
        const Axis ax = axis_map(ox, nx, mx), ay = axis_map(oy, ny, my), az = axis_map(oz, nz, mz);
        auto at = [&](int x, int y, int z) {
            const int64_t cell = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
            return layout == 0 ? src[cell * C + c] : src[(int64_t)c * nxyz + cell];
        };
        const float wx[2] = {1.f - ax.t, ax.t}, wy[2] = {1.f - ay.t, ay.t}, wz[2] = {1.f - az.t, az.t};
        const int xs[2] = {ax.i0, ax.i1}, ys[2] = {ay.i0, ay.i1}, zs[2] = {az.i0, az.i1};
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int e = 0; e < 2; ++e) acc += wz[a] * wy[b] * wx[e] * at(xs[e], ys[b], zs[a]);
        dst[k] = acc;
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

}  // namespace

extern "C" lbm_status lbm_resample(const float *src, int32_t nx, int32_t ny, int32_t nz, int32_t channels,
                                   int32_t src_layout, float *dst, int32_t mx, int32_t my, int32_t mz,
                                   void *cuda_stream)
{
    if (!src || !dst || nx < 1 || ny < 1 || nz < 1 || mx < 1 || my < 1 || mz < 1 || channels < 1 ||
        (src_layout != 0 && src_layout != 1)) {
        lbm::set_global_error("lbm_resample: null pointer, empty grid or unknown layout");
        return LBM_ERR_ARG;
    }
    if (!on_device(src) || !on_device(dst)) {
        lbm::set_global_error("lbm_resample: src and dst must be device (or managed) memory");
        return LBM_ERR_ARG;
    }
    const int64_t total = (int64_t)channels * mz * my * mx;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)gb300::sm_count() * 16);
    k_resample<<<blocks, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(src, nx, ny, nz, channels, src_layout,
                                                                          dst, mx, my, mz);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        lbm::set_global_error(std::string("lbm_resample: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
