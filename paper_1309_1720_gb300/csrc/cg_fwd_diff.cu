// Forward stage kernels of the DIFF model (instantiations of cg_stepper.cuh).
#include "cg_stepper.cuh"

namespace cgk {

const void *fwd_kernel_diff(int stencil, int scheme, int cx)
{
    return pick_fwd_kernel<MODEL_DIFF>(stencil, scheme, cx);
}

}  // namespace cgk
