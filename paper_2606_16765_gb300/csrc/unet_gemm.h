// unet_gemm.h -- the U-Net's 3x3x3 convolutions as implicit GEMMs on the
// tcgen05 tensor cores (unet_gemm.cu): the plans (tensor maps, tile shapes,
// launch sizes) and their launches.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace unet {

// One convolution y[cell][n] = sum_tap sum_k A[cell + tap - 1][k] W[tap][n][k]
// over a channel-last BF16 activation A [B][Z][Y][X][lda] (K = the first
// `k` channels) and BF16 weights W [taps][N][k]; taps 27 (3x3x3) or 1.
struct ConvArgs {
    int X, Y, Z, B;              // grid of the activation (= output grid)
    int bx, by, bz, bb;          // a tile of 128 cells: bx * by * bz * bb = 128
    int tx, ty, tz, tb;          // tiles along each axis
    int ntaps;                   // 27 or 1
    int kchunks;                 // K per tap / chunk width
    int ntile, nntiles;          // output channels per tile, tiles
    int ldo, ooff;               // output row stride and channel offset
    int stages;                  // pipeline depth
    int64_t nwork;               // cell tiles x channel tiles
    uint32_t a_bytes, b_bytes;   // shared-memory bytes of one stage's operands
    uint32_t idesc;              // instruction descriptor
    uint32_t tmem_cols;          // tensor-memory columns (two accumulators)
};

struct ConvPlan {
    alignas(64) unsigned char amap[128];
    alignas(64) unsigned char wmap[128];
    ConvArgs a;
    int ck = 0;                  // chunk width: 64 (128-byte swizzle) or 32 (64-byte)
    size_t smem = 0;
    int grid = 0;
};

// Weight gradient G[m][n] += sum_cell X[cell + tap(m) - 1][ci(m)] GZ[cell][n],
// m = tap * cin + ci, as a GEMM with both operands MN-major (cells are the
// contraction index); FP32 result accumulated atomically.
struct WgradArgs {
    int X, Y, Z, B;
    int bx, by, bz, bb;
    int tx, ty, tz, tb;
    int cin_blocks;              // cin / 32
    int m_total;                 // 27 * cin
    int mtiles;                  // ceil(m_total / 128)
    int ntile, nntiles;
    int64_t nchunks;             // cell tiles
    int ksplit;                  // slices of the cell range
    int stages;
    int64_t nwork;
    uint32_t a_bytes, b_bytes;
    uint32_t idesc;
    uint32_t tmem_cols;
    int ldg;                     // row stride of G (= N)
};

struct WgradPlan {
    alignas(64) unsigned char xmap[128];
    alignas(64) unsigned char gmap[128];
    WgradArgs a;
    size_t smem = 0;
    int grid = 0;
};

// false: unsupported shape or tensor-map encoding failed (message in err).
bool conv_plan(ConvPlan &p, const void *act, int lda, int k, int X, int Y, int Z, int B, const void *w, int N,
               int ntaps, int ldo, int ooff, int sms, const char **err);
void conv_launch(const ConvPlan &p, void *out, bool out_f32, int *status, cudaStream_t s);

bool wgrad_plan(WgradPlan &p, const void *x, int ldx, int cin, const void *gz, int ldg, int N, int X, int Y, int Z,
                int B, int sms, const char **err);
void wgrad_launch(const WgradPlan &p, float *g, int *status, cudaStream_t s);

// Raise the kernels' dynamic shared-memory limits (once per process).
bool gemm_set_attrs();

}  // namespace unet
