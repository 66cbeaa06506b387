// Tangent-linear kernels of the FHN model (instantiations of cg_tlm.cuh).
#include "cg_tlm.cuh"

namespace cgk {

const void *tlm_kernel_fhn(int stencil, int scheme, int cx)
{
    return pick_tlm_kernel<MODEL_FHN>(stencil, scheme, cx);
}

}  // namespace cgk
