// sm_count.h -- multiprocessor count of the current device, read once per
// device from cudaDevAttrMultiProcessorCount.  Grid-stride launches size
// their grids as a multiple of it (152 on a GB300).
#pragma once
#include <atomic>

#include <cuda_runtime.h>

namespace gb300 {

inline int sm_count()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            return 152;
        }
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

}  // namespace gb300
