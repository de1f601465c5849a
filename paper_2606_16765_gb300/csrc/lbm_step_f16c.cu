// lbm_step_f16c.cu -- step kernels instantiated for the 16-bit custom float
// storage (F16C) of the shifted populations.
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbm {
void launch_step_f16c(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, int block_y,
                    cudaStream_t s, cudaEvent_t ev_interior, cudaEvent_t ev_bulk)
{
    launch_step_t<F16C>(a, odd, epi, plain, block_x, block_y, s, ev_interior, ev_bulk);
}

void launch_batch_step_f16c(const BatchLaunch &L, bool odd, bool epi, bool plain, cudaStream_t s)
{
    launch_batch_step_t<F16C>(L, odd, epi, plain, s);
}

void launch_outflow_record_f16c(const StepArgs &a, bool odd, cudaStream_t s)
{
    launch_outflow_record_t<F16C>(a, odd, s);
}
}  // namespace lbm
