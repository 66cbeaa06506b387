// Small helper kernels of the adjoint driver.
#include "cg_adjoint.cuh"

namespace cgk {

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
