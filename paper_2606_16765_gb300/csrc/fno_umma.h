// fno_umma.h -- host side of the tcgen05 forward x stage (fno_umma.cu).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

// Dynamic shared memory of the kernel (bytes).
size_t umma_dftx_smem();
// Raise the kernel's shared-memory limit; false on failure.
bool umma_set_smem();
// Encode the 128-byte-swizzled tensor map of R BF16 rows of 128 samples at
// `rows` (16-byte aligned) into map[128 bytes]; false if the driver entry
// point is missing or refuses.
bool umma_make_row_map(void *map, const void *rows, int64_t R);
// out[R][32] (complex) = rows[R][128] times the twiddle table twx[128][32],
// the first R rows of the map; status receives a nonzero code if a bounded
// wait gave up.
void umma_dftx_fwd(const void *map, const float2 *twx, float2 *out, int64_t R, int *status, int blocks,
                   cudaStream_t s);
