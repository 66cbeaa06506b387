// Forward stage kernels of the Karma model (instantiations of cg_stepper.cuh and
// cg_tblock.cuh).
#include "cg_tblock.cuh"

namespace cgk {

const void *fwd_kernel_karma(int stencil, int scheme, int cx)
{
    return pick_fwd_kernel<MODEL_KARMA>(stencil, scheme, cx);
}

const void *tb_kernel_karma(int stencil, int scheme)
{
    return pick_tb_kernel<MODEL_KARMA>(stencil, scheme);
}

}  // namespace cgk
