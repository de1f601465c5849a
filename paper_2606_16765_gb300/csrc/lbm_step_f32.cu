// lbm_step_f32.cu -- step kernels instantiated for float storage of the shifted
// populations (one translation unit per storage type for parallel builds).
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbm {
void launch_step_f32(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, int block_y,
                    cudaStream_t s, cudaEvent_t ev_interior, cudaEvent_t ev_bulk)
{
    launch_step_t<float>(a, odd, epi, plain, block_x, block_y, s, ev_interior, ev_bulk);
}

void launch_batch_step_f32(const BatchLaunch &L, bool odd, bool epi, bool plain, cudaStream_t s)
{
    launch_batch_step_t<float>(L, odd, epi, plain, s);
}

void launch_outflow_record_f32(const StepArgs &a, bool odd, cudaStream_t s)
{
    launch_outflow_record_t<float>(a, odd, s);
}
}  // namespace lbm
