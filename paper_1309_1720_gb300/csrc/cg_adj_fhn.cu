// Adjoint kernels of the FHN model (instantiations of cg_adjoint.cuh).
#include "cg_adjoint.cuh"

namespace cgk {

const void *adj_kernel_fhn(int stencil, int scheme, int cx)
{
    return pick_adj_kernel<MODEL_FHN>(stencil, scheme, cx);
}

}  // namespace cgk
