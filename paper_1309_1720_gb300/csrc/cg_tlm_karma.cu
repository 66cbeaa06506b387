// Tangent-linear kernels of the Karma model (instantiations of cg_tlm.cuh).
#include "cg_tlm.cuh"

namespace cgk {

const void *tlm_kernel_karma(int stencil, int scheme, int cx)
{
    return pick_tlm_kernel<MODEL_KARMA>(stencil, scheme, cx);
}

}  // namespace cgk
