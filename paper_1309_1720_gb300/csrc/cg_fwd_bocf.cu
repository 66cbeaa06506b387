// Forward stage kernels of the BOCF model (instantiations of cg_stepper.cuh and
// cg_tblock.cuh).
#include "cg_tblock.cuh"

namespace cgk {

const void *fwd_kernel_bocf(int stencil, int scheme, int cx)
{
    return pick_fwd_kernel<MODEL_BOCF>(stencil, scheme, cx);
}

const void *tb_kernel_bocf(int stencil, int scheme)
{
    return pick_tb_kernel<MODEL_BOCF>(stencil, scheme);
}

namespace {

__global__ void k_rcp_consts(double ts1, double dts, double *out)
{
    out[0] = fast_rcp(ts1);
    out[1] = fast_rcp(fma(1.0, dts, ts1));
}

}  // namespace

cudaError_t bocf_rcp_constants(double ts1, double dts, double *out)
{
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(double));
    if (e == cudaSuccess) {
        k_rcp_consts<<<1, 1>>>(ts1, dts, d);
        e = cudaMemcpy(out, d, 2 * sizeof(double), cudaMemcpyDeviceToHost);
    }
    if (d) cudaFree(d);
    return e;
}

}  // namespace cgk
