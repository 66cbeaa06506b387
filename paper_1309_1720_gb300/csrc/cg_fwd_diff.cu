// Forward stage kernels of the DIFF model (instantiations of cg_stepper.cuh and
// cg_tblock.cuh).
#include "cg_tblock.cuh"

namespace cgk {

const void *fwd_kernel_diff(int stencil, int scheme, int cx)
{
    return pick_fwd_kernel<MODEL_DIFF>(stencil, scheme, cx);
}

const void *tb_kernel_diff(int stencil, int scheme)
{
    return pick_tb_kernel<MODEL_DIFF>(stencil, scheme);
}

}  // namespace cgk
