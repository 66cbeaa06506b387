// Forward stage kernels of the FHN model (instantiations of cg_stepper.cuh).
#include "cg_stepper.cuh"

namespace cgk {

const void *fwd_kernel_fhn(int stencil, int scheme, int cx)
{
    return pick_fwd_kernel<MODEL_FHN>(stencil, scheme, cx);
}

}  // namespace cgk
