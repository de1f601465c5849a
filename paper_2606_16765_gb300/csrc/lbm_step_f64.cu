// lbm_step_f64.cu -- step kernels instantiated for double storage of the shifted
// populations (one translation unit per storage type for parallel builds).
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbm {
void launch_step_f64(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, int block_y,
                    cudaStream_t s, cudaEvent_t ev_interior, cudaEvent_t ev_bulk)
{
    launch_step_t<double>(a, odd, epi, plain, block_x, block_y, s, ev_interior, ev_bulk);
}

void launch_batch_step_f64(const BatchLaunch &L, bool odd, bool epi, bool plain, cudaStream_t s)
{
    launch_batch_step_t<double>(L, odd, epi, plain, s);
}

void launch_outflow_record_f64(const StepArgs &a, bool odd, cudaStream_t s)
{
    launch_outflow_record_t<double>(a, odd, s);
}
}  // namespace lbm
