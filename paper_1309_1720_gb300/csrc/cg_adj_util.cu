// Small helper kernels of the adjoint driver.
#include "cg_adjoint.cuh"

namespace cgk {

__global__ void k_scale(double *dst, const double *src, double c, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = c * src[i];
}

// One thread per diffusive field sums the per-warp partials in index order,
// so the result does not depend on scheduling, then scales by 1/Dxx_f.
__global__ void k_reduce_partials(const double *partial, int nw, int nd, Inv4 inv, double *out)
{
    const int f = threadIdx.x;
    if (f >= nd) return;
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += partial[(int64_t)w * nd + f];
    out[f] = s * inv.v[f];
}

}  // namespace cgk
