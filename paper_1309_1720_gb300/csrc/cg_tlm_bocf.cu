// Tangent-linear kernels of the BOCF model (instantiations of cg_tlm.cuh).
#include "cg_tlm.cuh"

namespace cgk {

const void *tlm_kernel_bocf(int stencil, int scheme, int cx)
{
    return pick_tlm_kernel<MODEL_BOCF>(stencil, scheme, cx);
}

}  // namespace cgk
