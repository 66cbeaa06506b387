// Forward stage kernels of the BOCF model (instantiations of cg_stepper.cuh).
#include "cg_stepper.cuh"

namespace cgk {

const void *fwd_kernel_bocf(int stencil, int scheme, int cx)
{
    return pick_fwd_kernel<MODEL_BOCF>(stencil, scheme, cx);
}

}  // namespace cgk
