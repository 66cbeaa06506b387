// Tangent-linear kernels of the BOCF model with its tanh terms as smoothed steps
// (instantiations of cg_tlm.cuh).
#include "cg_tlm.cuh"

namespace cgk {

const void *tlm_kernel_bocfh(int stencil, int scheme, int cx)
{
    return pick_tlm_kernel<MODEL_BOCFH>(stencil, scheme, cx);
}

}  // namespace cgk
