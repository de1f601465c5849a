// lbm_step_f16c.cu -- step kernels instantiated for the 16-bit custom float
// storage (F16C) of the shifted populations.
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbm {
void launch_step_f16c(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, cudaStream_t s,
                      cudaEvent_t ev_interior, cudaEvent_t ev_bulk)
{
    launch_step_t<F16C>(a, odd, epi, plain, block_x, s, ev_interior, ev_bulk);
}
}  // namespace lbm
