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

void launch_flags(const uint8_t *mask, uint8_t *flags, int nx, int ny, int nz, bool xface_lo, bool xface_hi,
                  bool wall_y, bool wall_z, cudaStream_t s);
void launch_aux(int storage, AuxOp op, const StepArgs &a, bool odd, const AuxArgs &x, cudaStream_t s);
void launch_mean_out(const double *msum, int64_t n, double inv_samples, bool f32, void *out, cudaStream_t s);
void launch_stats_out(const double *msum, int64_t n, double inv_samples, bool f32, void *out, cudaStream_t s);
void launch_halfres(const void *in, int nx, int ny, int nz, bool f32, void *out, cudaStream_t s);

}  // namespace lbm
