// Forward stage kernels of the BOCF model with its tanh terms as smoothed steps
// (instantiations of cg_stepper.cuh).
#include "cg_stepper.cuh"

namespace cgk {

const void *fwd_kernel_bocfh(int stencil, int scheme, int cx)
{
    return pick_fwd_kernel<MODEL_BOCFH>(stencil, scheme, cx);
}

}  // namespace cgk
