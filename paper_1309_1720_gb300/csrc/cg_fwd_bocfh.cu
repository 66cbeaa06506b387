// Forward stage kernels of the BOCF model with its tanh terms as smoothed steps
// (instantiations of cg_stepper.cuh and cg_tblock.cuh).
#include "cg_tblock.cuh"

namespace cgk {

const void *fwd_kernel_bocfh(int stencil, int scheme, int cx)
{
    return pick_fwd_kernel<MODEL_BOCFH>(stencil, scheme, cx);
}

const void *tb_kernel_bocfh(int stencil, int scheme)
{
    return pick_tb_kernel<MODEL_BOCFH>(stencil, scheme);
}

}  // namespace cgk
