// Adjoint kernels of the DIFF model (instantiations of cg_adjoint.cuh).
#include "cg_adjoint.cuh"

namespace cgk {

const void *adj_kernel_diff(int stencil, int scheme, int cx)
{
    return pick_adj_kernel<MODEL_DIFF>(stencil, scheme, cx);
}

}  // namespace cgk
