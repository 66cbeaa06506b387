// Tangent-linear kernels of the DIFF model (instantiations of cg_tlm.cuh).
#include "cg_tlm.cuh"

namespace cgk {

const void *tlm_kernel_diff(int stencil, int scheme, int cx)
{
    return pick_tlm_kernel<MODEL_DIFF>(stencil, scheme, cx);
}

}  // namespace cgk
