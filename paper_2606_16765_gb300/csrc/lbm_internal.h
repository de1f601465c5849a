// lbm_internal.h -- declarations shared by the translation units of the
// library (kernel launchers and the auxiliary-operation argument block).
#pragma once

#include <algorithm>
#include <cstdint>

#include "lbm_device.cuh"
#include "sm_count.h"

namespace lbm {

// fused step (bulk + edge kernels) for one storage type
void launch_step_f64(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, int block_y,
                    cudaStream_t s, cudaEvent_t ev_interior, cudaEvent_t ev_bulk);
void launch_batch_step_f64(const BatchLaunch &L, bool odd, bool epi, bool plain, cudaStream_t s);
void launch_outflow_record_f64(const StepArgs &a, bool odd, cudaStream_t s);
void launch_step_f32(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, int block_y,
                    cudaStream_t s, cudaEvent_t ev_interior, cudaEvent_t ev_bulk);
void launch_batch_step_f32(const BatchLaunch &L, bool odd, bool epi, bool plain, cudaStream_t s);
void launch_outflow_record_f32(const StepArgs &a, bool odd, cudaStream_t s);
void launch_step_f16(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, int block_y,
                    cudaStream_t s, cudaEvent_t ev_interior, cudaEvent_t ev_bulk);
void launch_batch_step_f16(const BatchLaunch &L, bool odd, bool epi, bool plain, cudaStream_t s);
void launch_outflow_record_f16(const StepArgs &a, bool odd, cudaStream_t s);
void launch_step_bf16(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, int block_y,
                    cudaStream_t s, cudaEvent_t ev_interior, cudaEvent_t ev_bulk);
void launch_batch_step_bf16(const BatchLaunch &L, bool odd, bool epi, bool plain, cudaStream_t s);
void launch_outflow_record_bf16(const StepArgs &a, bool odd, cudaStream_t s);
void launch_step_f16c(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, int block_y,
                    cudaStream_t s, cudaEvent_t ev_interior, cudaEvent_t ev_bulk);
void launch_batch_step_f16c(const BatchLaunch &L, bool odd, bool epi, bool plain, cudaStream_t s);
void launch_outflow_record_f16c(const StepArgs &a, bool odd, cudaStream_t s);

enum AuxOp { AUX_NOISE, AUX_GATHER, AUX_SET, AUX_MACROS, AUX_TOTALS, AUX_PROBE, AUX_EQUILIBRIUM, AUX_PLANE };

struct AuxArgs {
    uint64_t seed = 0;
    double amp = 0;
    const int64_t *cells = nullptr;
    int64_t count = 0;
    double *out = nullptr, *out2 = nullptr;
    float *fout = nullptr;
    const float *fsrc = nullptr;
    int64_t si = 0, sc = 0;
    const double *src = nullptr;
    double *partials = nullptr;
    int nblocks = 0;
};

// boundary-cell records on the device (lbm_aux.cu): counts per chunk of
// EB_CHUNK cells [blocks][4] = fluid, bulk, wall, record cells; then the
// records at the chunks' exclusive-scan offsets, and the solid links per
// direction heading into the obstacle
constexpr int EB_CHUNK = 8192;
constexpr int EB_THREADS = 256;
int64_t record_blocks(int64_t n);
void launch_record_count(const uint8_t *flags, int64_t n, int *counts, cudaStream_t s);
void launch_record_write(const uint8_t *flags, int nx, int ny, int nz, int fxlo, int fxhi, int fy, int fz,
                         const int64_t *offsets, uint4 *edge, unsigned long long *solid, cudaStream_t s);

// flags[idx[k]] -> out[k] (the cell classes a host-side check needs)
void launch_gather_flags(const uint8_t *flags, const int64_t *idx, int64_t m, uint8_t *out, cudaStream_t s);

void launch_flags(const uint8_t *mask, uint8_t *flags, int nx, int ny, int nz, bool xface_lo, bool xface_hi,
                  bool wall_y, bool wall_z, cudaStream_t s);
void launch_aux(int storage, AuxOp op, const StepArgs &a, bool odd, const AuxArgs &x, cudaStream_t s);
void launch_mean_out(const double *msum, int64_t n, double inv_samples, bool f32, void *out, cudaStream_t s);
void launch_stats_out(const double *msum, int64_t n, double inv_samples, bool f32, void *out, cudaStream_t s);
void launch_halfres(const void *in, int nx, int ny, int nz, bool f32, void *out, cudaStream_t s);

}  // namespace lbm
