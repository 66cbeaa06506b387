// Newton-Krylov step on the period-T flow map with exact Jacobian-vector
// products (the use the paper gives for double precision, Sect. 1), plus the
// deterministic vector kernels it needs.
//
// Solves (J_T - I) dz = -(Phi_T(z0) - z0) by restarted GMRES with modified
// Gram-Schmidt; J_T v comes from the tangent-linear kernels, every vector
// operation runs on the device, only the small Hessenberg least-squares
// problem (Givens rotations) is solved on the host.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cardiac_gb300.h"
#include "cg_internal.h"

#define CG_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr int DOT_BLOCKS = 256, DOT_THREADS = 256;

// Each block sums a fixed strided subset in a fixed order, then a fixed tree;
// the second kernel adds the block sums in index order.  Same inputs, same
// bits, whatever the scheduling.
__global__ void k_dot_partial(const double *x, const double *y, int64_t n, double *part)
{
    __shared__ double sh[DOT_THREADS];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * DOT_THREADS + threadIdx.x; i < n; i += (int64_t)DOT_BLOCKS * DOT_THREADS)
        s = fma(x[i], y[i], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = DOT_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(const double *part, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < DOT_BLOCKS; ++b) s += part[b];
        out[0] = s;
    }
}

// y = a x + b y
__global__ void k_axpby(double a, const double *x, double b, double *y, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], b * y[i]);
}

}  // namespace

namespace {

// Status with a message for cg_last_error().
cg_status err(cg_status st, const char *msg)
{
    return cgk::set_last_error(st, msg);
}

cg_status cuda_err(cudaError_t e)
{
    return e == cudaSuccess ? CG_OK : cgk::set_last_error(CG_ECUDA, cudaGetErrorString(e));
}

}  // namespace

CG_API cg_status cg_dot(const double *x, const double *y, int64_t n, double *result, void *workspace, void *stream)
{
    if (!x || !y || !result || !workspace || n < 0) return err(CG_EINVAL, "cg_dot: NULL buffer or n < 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double *part = reinterpret_cast<double *>(workspace);
    k_dot_partial<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(x, y, n, part);
    k_dot_final<<<1, 32, 0, s>>>(part, result);
    return cuda_err(cudaGetLastError());
}

CG_API cg_status cg_axpby(double a, const double *x, double b, double *y, int64_t n, void *stream)
{
    if (!x || !y || n < 0) return err(CG_EINVAL, "cg_axpby: NULL buffer or n < 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t blocks = std::min<int64_t>(4096, (n + 255) / 256 + 1);
    k_axpby<<<(unsigned)blocks, 256, 0, s>>>(a, x, b, y, n);
    return cuda_err(cudaGetLastError());
}

namespace {

struct Dev {
    cudaStream_t s;
    double *dpart, *dres;
    cg_status dot(const double *x, const double *y, int64_t n, double *out)
    {
        k_dot_partial<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(x, y, n, dpart);
        k_dot_final<<<1, 32, 0, s>>>(dpart, dres);
        cudaError_t e = cudaMemcpyAsync(out, dres, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return cuda_err(e);
    }
    cg_status axpby(double a, const double *x, double b, double *y, int64_t n)
    {
        const int64_t blocks = std::min<int64_t>(4096, (n + 255) / 256 + 1);
        k_axpby<<<(unsigned)blocks, 256, 0, s>>>(a, x, b, y, n);
        return cuda_err(cudaGetLastError());
    }
};

}  // namespace

// Bytes of the tangent-linear workspace at the front of the Newton workspace:
// one stage Jacobian reused (lin = false) or every stage's kept (lin = true).
static cg_status newton_sizes(cg_plan plan, int32_t restart, bool lin, int64_t period_steps, size_t *tws,
                              size_t *total)
{
    int64_t off[2];
    if (cg_plan_n_instances(plan) != 1) return err(CG_EUNSUPPORTED, "Newton steps need a single-instance plan");
    cg_status st = cg_batch_offsets(plan, off);
    if (st != CG_OK) return st;
    st = lin ? cg_tlm_linearized_workspace_size(plan, 1, period_steps, tws) : cg_tlm_workspace_size(plan, 1, tws);
    if (st != CG_OK) return st;
    *tws = (*tws + 255) / 256 * 256;
    const size_t vec = ((size_t)off[1] + 31) / 32 * 32 * sizeof(double);
    *total = *tws + vec * (size_t)(restart + 4) + 4096;
    if ((double)*tws + (double)vec * ((double)restart + 4.0) + 4096.0 >= 4611686018427387904.0)   // 2^62
        return err(CG_EINVAL, "Newton workspace size overflows");
    return CG_OK;
}

CG_API cg_status cg_newton_workspace_size(cg_plan plan, int32_t restart, size_t *bytes)
{
    if (!plan || !bytes || restart < 1) return err(CG_EINVAL, "cg_newton_workspace_size: bad argument");
    size_t tws = 0;
    return newton_sizes(plan, restart, false, 0, &tws, bytes);
}

CG_API cg_status cg_newton_linearized_workspace_size(cg_plan plan, int32_t restart, int64_t period_steps,
                                                     size_t *bytes)
{
    if (!plan || !bytes || restart < 1 || period_steps < 1 || period_steps > CG_MAX_STEPS)
        return err(CG_EINVAL, "cg_newton_linearized_workspace_size: bad argument");
    size_t tws = 0;
    return newton_sizes(plan, restart, true, period_steps, &tws, bytes);
}

// One GMRES Newton step.  lin = false: every J v is a tangent-linear run that
// recomputes the primal trajectory; lin = true: one linearizing run keeps
// every stage's Jacobian, and each J v advances the tangent alone.  Both
// apply the same arithmetic to every tangent, so their results agree bit for
// bit.
static cg_status gmres_step(cg_plan plan, const double *z0, int64_t period_steps, int32_t restart,
                            int32_t max_restarts, double rtol, double *dz, double *res_hist, int32_t *n_iter,
                            void *workspace, void *stream, bool lin)
{
    if (!plan || !z0 || !dz || !workspace || period_steps < 1 || period_steps > CG_MAX_STEPS || restart < 1 ||
        max_restarts < 1 || !(rtol > 0))
        return err(CG_EINVAL, "cg_newton_gmres_step: bad argument");
    int64_t off[2];
    cg_status st = cg_batch_offsets(plan, off);
    if (st != CG_OK) return st;
    const int64_t n = off[1];
    size_t tws = 0, total = 0;
    st = newton_sizes(plan, restart, lin, period_steps, &tws, &total);
    if (st != CG_OK) return st;
    (void)total;
    const size_t vec = (size_t)(n + 31) / 32 * 32;
    char *base = reinterpret_cast<char *>(workspace);
    double *V = reinterpret_cast<double *>(base + tws);              // restart + 1 basis vectors
    double *w = V + vec * (restart + 1);
    double *phi = w + vec;                                            // Phi_T(z0), then scratch
    double *zT = phi + vec;
    Dev d;
    d.s = reinterpret_cast<cudaStream_t>(stream);
    d.dpart = zT + vec;
    d.dres = d.dpart + DOT_BLOCKS;
    const int m = restart;

    // J v: vout = J_T(z0) vin
    auto jvp = [&](const double *vin, double *vout) {
        return lin ? cg_tlm_apply(plan, vin, vout, 1, period_steps, base, stream)
                   : cg_tlm_run(plan, z0, vin, zT, vout, 1, period_steps, base, stream);
    };

    // b = -(Phi_T(z0) - z0), stored in w
    st = lin ? cg_tlm_linearize(plan, z0, phi, period_steps, base, stream)
             : cg_run(plan, z0, phi, period_steps, base, stream);
    if (st != CG_OK) return st;
    cudaError_t e = cudaMemcpyAsync(w, z0, sizeof(double) * n, cudaMemcpyDeviceToDevice, d.s);
    if (e != cudaSuccess) return cuda_err(e);
    if ((st = d.axpby(-1.0, phi, 1.0, w, n)) != CG_OK) return st;          // w = z0 - Phi
    e = cudaMemsetAsync(dz, 0, sizeof(double) * n, d.s);
    if (e != cudaSuccess) return cuda_err(e);
    double bnorm2 = 0;
    if ((st = d.dot(w, w, n, &bnorm2)) != CG_OK) return st;
    const double bnorm = std::sqrt(bnorm2);
    int iters = 0;
    if (res_hist) res_hist[0] = bnorm;
    if (bnorm == 0.0) {
        if (n_iter) *n_iter = 0;
        return CG_OK;
    }
    // r lives in phi: r = b - A dz (dz = 0 at start)
    e = cudaMemcpyAsync(phi, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, d.s);
    if (e != cudaSuccess) return cuda_err(e);
    double rnorm = bnorm;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    for (int cycle = 0; cycle < max_restarts && rnorm > rtol * bnorm; ++cycle) {
        // V0 = r / |r|
        e = cudaMemcpyAsync(V, phi, sizeof(double) * n, cudaMemcpyDeviceToDevice, d.s);
        if (e != cudaSuccess) return cuda_err(e);
        if ((st = d.axpby(0.0, V, 1.0 / rnorm, V, n)) != CG_OK) return st;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = rnorm;
        int j = 0;
        for (; j < m; ++j) {
            double *vj = V + vec * j;
            double *vn = V + vec * (j + 1);
            // vn = J_T vj - vj
            st = jvp(vj, vn);
            if (st != CG_OK) return st;
            if ((st = d.axpby(-1.0, vj, 1.0, vn, n)) != CG_OK) return st;
            for (int i = 0; i <= j; ++i) {
                double h = 0;
                if ((st = d.dot(vn, V + vec * i, n, &h)) != CG_OK) return st;
                H[(size_t)i * m + j] = h;
                if ((st = d.axpby(-h, V + vec * i, 1.0, vn, n)) != CG_OK) return st;
            }
            double hn2 = 0;
            if ((st = d.dot(vn, vn, n, &hn2)) != CG_OK) return st;
            const double hn = std::sqrt(hn2);
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0) {
                if ((st = d.axpby(0.0, vn, 1.0 / hn, vn, n)) != CG_OK) return st;
            }
            // apply the previous rotations, then a new one
            for (int i = 0; i < j; ++i) {
                const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
            const double r = std::hypot(a, b);
            cs[j] = r > 0 ? a / r : 1.0;
            sn[j] = r > 0 ? b / r : 0.0;
            H[(size_t)j * m + j] = r;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++iters;
            rnorm = std::fabs(g[j + 1]);
            if (res_hist) res_hist[iters] = rnorm;
            if (rnorm <= rtol * bnorm || hn == 0) {
                ++j;
                break;
            }
        }
        // back substitution and dz += V y
        for (int i = j - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
            y[i] = H[(size_t)i * m + i] != 0 ? s / H[(size_t)i * m + i] : 0.0;
        }
        for (int i = 0; i < j; ++i)
            if ((st = d.axpby(y[i], V + vec * i, 1.0, dz, n)) != CG_OK) return st;
        if (rnorm <= rtol * bnorm) break;
        // true residual for the restart: r = b - A dz
        st = jvp(dz, phi);
        if (st != CG_OK) return st;
        if ((st = d.axpby(1.0, dz, -1.0, phi, n)) != CG_OK) return st;      // phi = dz - J dz
        if ((st = d.axpby(1.0, w, 1.0, phi, n)) != CG_OK) return st;        // + b
        double r2 = 0;
        if ((st = d.dot(phi, phi, n, &r2)) != CG_OK) return st;
        rnorm = std::sqrt(r2);
    }
    if (n_iter) *n_iter = iters;
    return cuda_err(cudaStreamSynchronize(d.s));
}

CG_API cg_status cg_newton_gmres_step(cg_plan plan, const double *z0, int64_t period_steps, int32_t restart,
                                      int32_t max_restarts, double rtol, double *dz, double *res_hist,
                                      int32_t *n_iter, void *workspace, void *stream)
{
    cgk::NvtxRange nvtx_range("cg_newton_gmres_step");
    return gmres_step(plan, z0, period_steps, restart, max_restarts, rtol, dz, res_hist, n_iter, workspace, stream,
                      false);
}

CG_API cg_status cg_newton_gmres_step_linearized(cg_plan plan, const double *z0, int64_t period_steps,
                                                 int32_t restart, int32_t max_restarts, double rtol, double *dz,
                                                 double *res_hist, int32_t *n_iter, void *workspace, void *stream)
{
    cgk::NvtxRange nvtx_range("cg_newton_gmres_step_linearized");
    return gmres_step(plan, z0, period_steps, restart, max_restarts, rtol, dz, res_hist, n_iter, workspace, stream,
                      true);
}
