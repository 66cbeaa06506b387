// Adjoint kernels of the BOCF model with its tanh terms as smoothed steps
// (instantiations of cg_adjoint.cuh).
#include "cg_adjoint.cuh"

namespace cgk {

const void *adj_kernel_bocfh(int stencil, int scheme, int cx)
{
    return pick_adj_kernel<MODEL_BOCFH>(stencil, scheme, cx);
}

}  // namespace cgk
