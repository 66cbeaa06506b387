// Adjoint kernels of the Karma model (instantiations of cg_adjoint.cuh).
#include "cg_adjoint.cuh"

namespace cgk {

const void *adj_kernel_karma(int stencil, int scheme, int cx)
{
    return pick_adj_kernel<MODEL_KARMA>(stencil, scheme, cx);
}

}  // namespace cgk
