// Adjoint kernels of the BOCF model (instantiations of cg_adjoint.cuh).
#include "cg_adjoint.cuh"

namespace cgk {

const void *adj_kernel_bocf(int stencil, int scheme, int cx)
{
    return pick_adj_kernel<MODEL_BOCF>(stencil, scheme, cx);
}

}  // namespace cgk
