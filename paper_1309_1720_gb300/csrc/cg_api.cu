// Host side of libcardiac_gb300.so: plan validation, stencil and model
// coefficient folding, tile tables, workspace layout, kernel launches and
// the device status word.  Declarations: include/cardiac_gb300.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "cg_internal.h"
#include "cg_tlm.cuh"
#include "cg_adjoint.cuh"
#include "cg_tblock.cuh"

#define CG_API extern "C" __attribute__((visibility("default")))

using cgk::Inst;
using cgk::RunArgs;

namespace {

thread_local std::string g_err;
// Longest run any entry point accepts: stage counters (n_steps x stages)
// and per-step byte counts stay far from int64 / size_t overflow.
constexpr int64_t MAX_STEPS = CG_MAX_STEPS;
// Relative extra cost of a cell on the adjoint's scaled boundary path (the
// W^-1 / W factors of mirror ghosts): about 38 FP64 instructions per cell
// and reverse stage there against 27 in the interior.
constexpr double ADJ_BOUNDARY_COST = 0.4;

cg_status fail(cg_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

cg_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(CG_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int n_fields(int model)
{
    switch (model) {
    case CG_FHN: return 2;
    case CG_BOCF: return 4;
    case CG_KARMA: return 2;
    case CG_DIFFUSION: return 1;
    default: return -1;
    }
}

int n_diffusive(int model)
{
    switch (model) {
    case CG_FHN: return 2;
    case CG_BOCF: return 1;
    case CG_KARMA: return 1;
    case CG_DIFFUSION: return 1;
    default: return 0;
    }
}

int n_params(int model)
{
    switch (model) {
    case CG_FHN: return 3;
    case CG_BOCF: return 29;
    case CG_KARMA: return 8;
    case CG_DIFFUSION: return 0;
    default: return -1;
    }
}

int n_stages(int scheme)
{
    return scheme == CG_HEUN ? 2 : scheme == CG_RK4 ? 4 : 1;
}

// Rush-Larsen / implicit Euler on the gates (no Butcher tableau, no
// tangent-linear or adjoint kernels).
bool gate_scheme(int scheme)
{
    return scheme == CG_RUSH_LARSEN || scheme == CG_IMPLICIT_EULER;
}

// Kernel family of a problem: the model, or the tanh-as-smoothed-step
// variant of the four-field model.
int kernel_model(int model, uint32_t flags)
{
    return (model == CG_BOCF && (flags & CG_FLAG_TANH_AS_HK)) ? cgk::MODEL_BOCFH : model;
}

// Default constants.  FHN: (eps, a1, a0) of Sect. 2.  BOCF: epicardial set
// of the minimal model cited in Sect. 2 (order: uo uu thv thw thvm tho tv1m
// tv2m tvp tw1m tw2m kwm uwm twp tfi to1 to2 tso1 tso2 kso uso ts1 ts2 ks us
// tsi twinf winfstar), then the H_k sharpness k = 28.4 of Sect. 2.  Karma
// (order tau_u tau_v u* u_h u_v Re M k): (Re, M) = (1, 6) and k = 28.4 of
// Sect. 2, the others the values of the model paper it cites.
void default_params(int model, double *out)
{
    if (model == CG_FHN) {
        const double p[3] = {0.05, 1.5, -0.1};
        std::memcpy(out, p, sizeof p);
    } else if (model == CG_BOCF) {
        const double p[29] = {0.0,    1.55,   0.3,     0.13,   0.006,  0.006, 60.0, 1150.0,
                              1.4506, 60.0,   15.0,    65.0,   0.03,   200.0, 0.11, 400.0,
                              6.0,    30.0181, 0.9957, 2.0458, 0.65,   2.7342, 16.0, 2.0994,
                              0.9087, 1.8875, 0.07,    0.94,   28.4};
        std::memcpy(out, p, sizeof p);
    } else if (model == CG_KARMA) {
        const double p[8] = {2.5, 250.0, 1.5415, 3.0, 1.0, 1.0, 6.0, 28.4};
        std::memcpy(out, p, sizeof p);
    }
}

bool finite(double x) { return std::isfinite(x); }

}  // namespace

struct cg_plan_s {
    int32_t model = 0, stencil = 0, bc = 0, scheme = 0, nv = 0, ns = 0;
    int32_t kmodel = 0;              // kernel family (kernel_model)
    uint32_t flags = 0;
    double dt = 0;
    int device = 0;
    int num_sms = 0;
    std::vector<Inst> inst;          // in tile order
    std::vector<int64_t> offsets;    // packed offsets in user order (n_inst + 1)
    std::vector<int32_t> order;      // user index -> tile-order index
    Inst *d_inst = nullptr;
    std::vector<cgk::Seg> segs;      // static schedule
    std::vector<int32_t> warp_seg;
    cgk::Seg *d_segs = nullptr;
    int32_t *d_warp_seg = nullptr;
    // the adjoint's static schedule, cost-balanced for its boundary path
    // (single-instance mirror plans with grid barriers; else the one above)
    std::vector<cgk::Seg> segs_adj;
    std::vector<int32_t> warp_seg_adj;
    cgk::Seg *d_segs_adj = nullptr;
    int32_t *d_warp_seg_adj = nullptr;
    int32_t sched = cgk::SCHED_STATIC;
    int32_t n_tiles = 0;
    int32_t cx = 2, rows = 4, threads = 512, bpsm = 1;
    int64_t scratch_elems = 0;
    double mp[cgk::NMP] = {};
    double cacc[4] = {}, cy[4] = {};
    uint64_t timeout_ns = 0;
    const void *kernel = nullptr;
    // temporal blocking of cg_run (tuning.schedule = 2): steps per pass (0 =
    // off), tile size, tiles along x, blocks, threads, window cells, kernel
    int32_t tb_k = 0, tb_tx = 0, tb_ty = 0, tb_tiles = 0, tb_blocks = 0, tb_threads = 0, tb_wmax = 0;
    int32_t tb_nbr = 0, tb_tiles_x = 0, tb_tiles_y = 0;   // neighbour waits between passes (one instance)
    size_t tb_smem = 0;
    const void *tb_kernel = nullptr;
    int nblocks = 0;
    double dxx[4] = {};              // Dxx of the first instance (gradient normalisation)
    std::vector<int2> deps;          // halo owners of each block (neighbour sync)
    int2 *d_deps = nullptr;
    int32_t sync_mode = cgk::SYNC_GRID;
    double *d_tab = nullptr;         // 2^(j/4096) table of the exponential
    // workspace and stream of the latest run issued with this plan (for
    // cg_get_device_status; the plan's numerical content stays immutable)
    std::mutex last_mu;
    const void *last_ws = nullptr;
    void *last_stream = nullptr;
    // workspaces linearized with this plan and their step counts (the latest
    // 16), so that cg_tlm_apply can reject a workspace it never filled
    std::vector<std::pair<const void *, int64_t>> linearized;
    // checkpoint buffers filled by cg_adjoint_forward with this plan, with
    // their step counts and checkpoint intervals (the latest 16), so that
    // cg_adjoint_reverse can reject a buffer it never filled
    struct Ckpt {
        const void *buf;
        int64_t n_steps, c;
    };
    std::vector<Ckpt> checkpointed;
};

namespace cgk {

void exp_table(double *tab, int n)
{
    for (int j = 0; j < n; ++j) tab[j] = (double)std::exp2((long double)j / (long double)n);
}

}  // namespace cgk

namespace {

// Remember the workspace and stream of a run for cg_get_device_status.
void note_run(cg_plan P, const void *ws, cudaStream_t s)
{
    std::lock_guard<std::mutex> g(P->last_mu);
    P->last_ws = ws;
    P->last_stream = reinterpret_cast<void *>(s);
}

const void *lookup_tb_kernel(int kmodel, int stencil, int scheme)
{
    switch (kmodel) {
    case CG_FHN: return cgk::tb_kernel_fhn(stencil, scheme);
    case CG_BOCF: return cgk::tb_kernel_bocf(stencil, scheme);
    case CG_DIFFUSION: return cgk::tb_kernel_diff(stencil, scheme);
    case CG_KARMA: return cgk::tb_kernel_karma(stencil, scheme);
    case cgk::MODEL_BOCFH: return cgk::tb_kernel_bocfh(stencil, scheme);
    default: return nullptr;
    }
}

const void *lookup_kernel(int kmodel, int stencil, int scheme, int cx)
{
    switch (kmodel) {
    case CG_FHN: return cgk::fwd_kernel_fhn(stencil, scheme, cx);
    case CG_BOCF: return cgk::fwd_kernel_bocf(stencil, scheme, cx);
    case CG_DIFFUSION: return cgk::fwd_kernel_diff(stencil, scheme, cx);
    case CG_KARMA: return cgk::fwd_kernel_karma(stencil, scheme, cx);
    case cgk::MODEL_BOCFH: return cgk::fwd_kernel_bocfh(stencil, scheme, cx);
    default: return nullptr;
    }
}

// Weights of D_f L for one field: Dxx d_xx + Dyy d_yy + kappa h^2 d_xx d_yy
// with kappa = alpha_d (a + b) / 2 (Eq. diffusion; isotropic D recovers the
// paper's alpha_a = 1 - 2 alpha_d, alpha_00 = -4 (alpha_a + alpha_d)).
void stencil_weights(const cg_problem &p, int f, double &wx, double &wy, double &wd, double &wc)
{
    const double a = p.Dxx[f] / (p.dx * p.dx);
    const double b = p.Dyy[f] / (p.dy * p.dy);
    const double kappa = (p.stencil == CG_STENCIL9) ? p.alpha_d * (a + b) / 2.0 : 0.0;
    wx = a - 2.0 * kappa;
    wy = b - 2.0 * kappa;
    wd = kappa;
    wc = -2.0 * a - 2.0 * b + 4.0 * kappa;
}

// Largest |eigenvalue| of D_f L: the symbol a ex + b ey + kappa ex ey with
// ex, ey in [-4, 0] is bilinear, so the extremes sit at the corners.
double spectral_radius(const cg_problem &p, int f)
{
    const double a = p.Dxx[f] / (p.dx * p.dx);
    const double b = p.Dyy[f] / (p.dy * p.dy);
    const double kappa = (p.stencil == CG_STENCIL9) ? p.alpha_d * (a + b) / 2.0 : 0.0;
    return std::max({4.0 * a, 4.0 * b, std::fabs(-4.0 * a - 4.0 * b + 16.0 * kappa)});
}

cg_status validate(const cg_problem *p, int idx)
{
    if (!p) return fail(CG_EINVAL, "problem %d is NULL", idx);
    if (p->abi_version != CG_ABI_VERSION)
        return fail(CG_EINVAL, "problem %d: abi_version %d, library speaks %d", idx, p->abi_version,
                    CG_ABI_VERSION);
    const int nv = n_fields(p->model);
    if (nv < 0) return fail(CG_EINVAL, "problem %d: unknown model %d", idx, p->model);
    if (p->nx < 2 || p->ny < 2 || p->nx > (1 << 28) || p->ny > (1 << 28))
        return fail(CG_EINVAL, "problem %d: grid %lld x %lld outside [2, 2^28]", idx, (long long)p->nx,
                    (long long)p->ny);
    if ((double)p->nx * (double)p->ny * nv > 4.0e12)
        return fail(CG_EINVAL, "problem %d: grid too large", idx);
    if (!(p->dx > 0) || !(p->dy > 0) || !finite(p->dx) || !finite(p->dy))
        return fail(CG_EINVAL, "problem %d: dx, dy must be positive and finite", idx);
    if (!(p->dt > 0) || !finite(p->dt)) return fail(CG_EINVAL, "problem %d: dt must be positive", idx);
    if (p->stencil != CG_STENCIL5 && p->stencil != CG_STENCIL9)
        return fail(CG_EINVAL, "problem %d: unknown stencil %d", idx, p->stencil);
    if (p->stencil == CG_STENCIL9 && (!finite(p->alpha_d) || p->alpha_d < 0 || p->alpha_d > 0.25))
        return fail(CG_EINVAL, "problem %d: alpha_d %g outside [0, 1/4]", idx, p->alpha_d);
    if (p->bc != CG_BC_MIRROR && p->bc != CG_BC_CLAMP && p->bc != CG_BC_PERIODIC)
        return fail(CG_EINVAL, "problem %d: unknown boundary mode %d", idx, p->bc);
    if (p->scheme != CG_EULER && p->scheme != CG_HEUN && p->scheme != CG_RK4 && !gate_scheme(p->scheme))
        return fail(CG_EINVAL, "problem %d: unknown scheme %d", idx, p->scheme);
    if (gate_scheme(p->scheme) && p->model != CG_BOCF)
        return fail(CG_EUNSUPPORTED, "problem %d: Rush-Larsen and implicit Euler integrate the gates of the "
                                     "four-field model only", idx);
    if ((p->flags & CG_FLAG_TANH_AS_HK) && p->model != CG_BOCF && p->model != CG_KARMA)
        return fail(CG_EUNSUPPORTED, "problem %d: CG_FLAG_TANH_AS_HK applies to the four-field and Karma models "
                                     "only", idx);
    if (gate_scheme(p->scheme) && p->params) {
        // the gate coefficients al are negative when these time constants are
        // positive: tv1m tv2m tvp tw1m tw2m twp ts1 ts2
        const int tau[] = {6, 7, 8, 9, 10, 13, 21, 22};
        for (int i : tau)
            if (!(p->params[i] > 0))
                return fail(CG_EINVAL, "problem %d: the gate integrators need positive time constants "
                                       "(param %d = %g)", idx, i, p->params[i]);
    }
    const int nd = n_diffusive(p->model);
    for (int f = 0; f < 4; ++f) {
        if (!finite(p->Dxx[f]) || !finite(p->Dyy[f]) || p->Dxx[f] < 0 || p->Dyy[f] < 0)
            return fail(CG_EINVAL, "problem %d: D of field %d must be finite and >= 0", idx, f);
        if (f >= nd && (p->Dxx[f] != 0 || p->Dyy[f] != 0))
            return fail(CG_EUNSUPPORTED, "problem %d: field %d of this model does not diffuse", idx, f);
    }
    if (p->params && p->n_params != n_params(p->model))
        return fail(CG_EINVAL, "problem %d: %d params given, model takes %d", idx, p->n_params,
                    n_params(p->model));
    if (p->params)
        for (int i = 0; i < p->n_params; ++i)
            if (!finite(p->params[i])) return fail(CG_EINVAL, "problem %d: param %d not finite", idx, i);
    if (p->model == CG_BOCF && p->params && !(p->params[28] > 0))
        return fail(CG_EINVAL, "problem %d: the smoothed-step sharpness k must be positive", idx);
    if (p->model == CG_KARMA && p->params) {
        // tau_u, tau_v divide; Re = 0 makes 1/(1 - e^-Re) infinite
        if (p->params[0] == 0 || p->params[1] == 0 || p->params[5] == 0)
            return fail(CG_EINVAL, "problem %d: Karma tau_u, tau_v and Re must be non-zero", idx);
    }
    if (!(p->flags & CG_FLAG_ALLOW_UNSTABLE)) {
        const double bound = (p->scheme == CG_RK4) ? 2.785 : 2.0;
        double rho = 0;
        for (int f = 0; f < nd; ++f) rho = std::max(rho, spectral_radius(*p, f));
        if (rho * p->dt > bound * (1.0 + 1e-12))
            return fail(CG_EUNSTABLE, "problem %d: dt %g exceeds the linear diffusive bound %g", idx, p->dt,
                        bound / rho);
    }
    return CG_OK;
}

void fold_constants(cg_plan_s &P, const cg_problem &p, Inst &I)
{
    double prm[32] = {};
    if (p.params) std::memcpy(prm, p.params, sizeof(double) * p.n_params);
    else default_params(p.model, prm);
    for (int f = 0; f < cgk::MAXF; ++f) {
        if (f < n_diffusive(p.model)) stencil_weights(p, f, I.wx[f], I.wy[f], I.wd[f], I.wc[f]);
        else I.wx[f] = I.wy[f] = I.wd[f] = I.wc[f] = 0.0;
        I.wt[f] = (I.wd[f] != 0.0) ? I.wy[f] / I.wd[f] : 0.0;
    }
    std::memset(I.mi, 0, sizeof I.mi);
    std::memset(P.mp, 0, sizeof P.mp);
    if (p.model == CG_FHN) {
        const double eps = prm[0], a1 = prm[1], a0 = prm[2];
        P.mp[0] = eps;
        P.mp[1] = -eps * a0;
        I.mi[0] = 1.0 + I.wc[0];
        I.mi[1] = I.wc[1] - eps * a1;
    } else if (p.model == CG_DIFFUSION) {
        I.mi[0] = I.wc[0];
    } else if (p.model == CG_KARMA) {  // layout of cg_stepper.cuh
        const double tu = prm[0], tv = prm[1], ustar = prm[2], uh = prm[3], uv = prm[4], re = prm[5], M = prm[6],
                     k = prm[7];
        const double a = 1.0 / (1.0 - std::exp(-re));
        P.mp[cgk::KP_ITU] = 1.0 / tu;
        P.mp[cgk::KP_ITV] = 1.0 / tv;
        P.mp[cgk::KP_USTAR] = ustar;
        P.mp[cgk::KP_SA] = 2.0 * uh;
        P.mp[cgk::KP_HA] = 0.5 + uh / 3.0;
        P.mp[cgk::KP_AITV] = a / tv;
        P.mp[cgk::KP_K] = k;
        P.mp[cgk::KP_CV] = 0.5 - k * uv;
        P.mp[cgk::KP_6KA] = 6.0 * k * a / tv;
        P.mp[cgk::KP_M] = M;
        const int64_t mi = (M >= 0 && M <= 64 && M == std::floor(M)) ? (int64_t)M : -1;
        std::memcpy(&P.mp[cgk::KP_MI], &mi, sizeof mi);
        P.mp[cgk::KP_TH] = (p.flags & CG_FLAG_TANH_AS_HK) ? 1.0 : 0.0;
        static_assert(cgk::KP_N <= cgk::NMP, "model constant table too small");
        I.mi[0] = I.wc[0] - 1.0 / tu;
    } else {  // BOCF, layout of cg_stepper.cuh
        for (int i = 0; i < 29; ++i) P.mp[i] = prm[i];
        const double k = prm[28];
        P.mp[29] = 0.5 - k * prm[2];    // thv
        P.mp[30] = 0.5 - k * prm[3];    // thw
        P.mp[31] = 0.5 - k * prm[4];    // thvm
        P.mp[32] = 0.5 - k * prm[5];    // tho
        P.mp[33] = prm[7] - prm[6];     // tv2m - tv1m
        P.mp[34] = prm[16] - prm[15];   // to2 - to1
        P.mp[35] = prm[22] - prm[21];   // ts2 - ts1
        P.mp[36] = 1.0 / prm[14];       // 1/tfi
        P.mp[37] = 1.0 / prm[25];       // 1/tsi
        P.mp[38] = 1.0 / prm[8];        // 1/tvp
        P.mp[39] = 1.0 / prm[13];       // 1/twp
        P.mp[40] = 1.0 / prm[26];       // 1/twinf
        // (1 + tanh(a))/2 = sigmoid(2 a): the arguments are pre-doubled
        P.mp[cgk::BD_AW2] = -2.0 * prm[11] * prm[12];
        P.mp[cgk::BD_KW2] = 2.0 * prm[11];
        P.mp[cgk::BD_ASO2] = -2.0 * prm[19] * prm[20];
        P.mp[cgk::BD_KSO2] = 2.0 * prm[19];
        P.mp[cgk::BD_AS2] = -2.0 * prm[23] * prm[24];
        P.mp[cgk::BD_KS2] = 2.0 * prm[23];
        P.mp[cgk::BD_DTW] = prm[10] - prm[9];
        P.mp[cgk::BD_DTSO] = prm[18] - prm[17];
        P.mp[cgk::BD_6K] = 6.0 * k;
        // tanh variant: H_{kk/3}(u - cc) with t = kk/3 u + 1/2 - kk cc/3
        P.mp[cgk::BD_KWH] = prm[11] / 3.0;
        P.mp[cgk::BD_AWH] = 0.5 - prm[11] * prm[12] / 3.0;
        P.mp[cgk::BD_KSOH] = prm[19] / 3.0;
        P.mp[cgk::BD_ASOH] = 0.5 - prm[19] * prm[20] / 3.0;
        P.mp[cgk::BD_KSH] = prm[23] / 3.0;
        P.mp[cgk::BD_ASH] = 0.5 - prm[23] * prm[24] / 3.0;
        // shortcut bounds of the kernel's switches t = clamp(k u + c): the
        // largest u with fma(k, u, c) <= 0 and the smallest with >= 1
        // (fma is correctly rounded here as on the device, and monotone in u)
        // Bisection over the order keys of all doubles from -inf to +inf
        // (the key map is its own inverse); k > 0 is validated.
        auto key_of = [](double x) {
            int64_t b;
            std::memcpy(&b, &x, sizeof b);
            return b ^ ((b >> 63) & INT64_C(0x7FFFFFFFFFFFFFFF));
        };
        auto from_key = [&](int64_t q) {
            const int64_t b = q ^ ((q >> 63) & INT64_C(0x7FFFFFFFFFFFFFFF));
            double x;
            std::memcpy(&x, &b, sizeof x);
            return x;
        };
        auto boundary = [&](auto pred_hi) {       // smallest key where the monotone pred_hi holds
            int64_t lo = key_of(-INFINITY), hi = key_of(INFINITY);
            // the key range spans almost 2^64: differences in unsigned arithmetic
            while ((uint64_t)hi - (uint64_t)lo > 1) {
                const int64_t mid = (int64_t)((uint64_t)lo + ((uint64_t)hi - (uint64_t)lo) / 2);
                if (pred_hi(from_key(mid))) hi = mid; else lo = mid;
            }
            return hi;
        };
        auto last_zero = [&](double c) {
            return from_key(boundary([&](double u) { return std::fma(k, u, c) > 0; }) - 1);
        };
        auto first_one = [&](double c) {
            return from_key(boundary([&](double u) { return std::fma(k, u, c) >= 1; }));
        };
        auto key_bits = [&](double x) {
            const int64_t q = key_of(x);
            double d;
            std::memcpy(&d, &q, sizeof d);
            return d;
        };
        const double u_rest = std::min(last_zero(P.mp[cgk::BD_CV]), last_zero(P.mp[cgk::BD_CW]));
        const double u_exc = std::max({first_one(P.mp[cgk::BD_CV]), first_one(P.mp[cgk::BD_CW]),
                                       first_one(P.mp[cgk::BD_CVM]), first_one(P.mp[cgk::BD_CO])});
        P.mp[cgk::BD_KREST] = key_bits(u_rest);
        P.mp[cgk::BD_KEXC] = key_bits(u_exc);
        {
            // exact savings the constants allow (cg_stepper.cuh, BF_*)
            long long fl = 0;
            if (std::memcmp(&P.mp[cgk::BD_CVM], &P.mp[cgk::BD_CO], sizeof(double)) == 0) fl |= cgk::BF_SAME_VMO;
            std::memcpy(&P.mp[cgk::BD_FLAGS], &fl, sizeof fl);
        }
        static_assert(cgk::BD_N <= cgk::NMP, "model constant table too small");
        I.mi[0] = I.wc[0];
    }
}

bool same_config(const cg_problem &a, const cg_problem &b)
{
    if (a.model != b.model || a.stencil != b.stencil || a.bc != b.bc || a.scheme != b.scheme ||
        a.dt != b.dt || a.flags != b.flags || a.barrier_timeout_s != b.barrier_timeout_s)
        return false;
    if (a.stencil == CG_STENCIL9 && a.alpha_d != b.alpha_d) return false;
    if ((a.params == nullptr) != (b.params == nullptr)) return false;
    if (a.params)
        for (int i = 0; i < a.n_params; ++i)
            if (a.params[i] != b.params[i]) return false;
    return true;
}

// Block ranges of the static schedule: G + 1 monotone cell offsets from 0 to
// the total cell count of the instances (in plan order, row-major inside an
// instance).  Every offset is the start of a strip-row (the 32*cx cells of a
// row's column strip, which one warp runs in one pass of its row loop) or
// the end, chosen so that the blocks' summed strip-row costs are equal to
// within one strip-row: each boundary is the strip-row start whose
// cumulative cost is nearest to b/G of the total.  A warp takes a strip-row
// in the same time however many of its cells it holds (the FP64 pipe is
// warp-granular), so a cut inside a strip would charge both blocks a whole
// strip-row.  cost(k, y, x0): the cost of strip-row (y, x0) of instance k.
template <class Cost>
std::vector<int64_t> strip_ranges(const std::vector<int32_t> &nxs, const std::vector<int32_t> &nys, int tw, int G,
                                  Cost cost)
{
    const int n = (int)nxs.size();
    double total = 0.0;
    int64_t N = 0;
    for (int k = 0; k < n; ++k) {
        N += (int64_t)nxs[k] * nys[k];
        for (int y = 0; y < nys[k]; ++y)
            for (int x0 = 0; x0 < nxs[k]; x0 += tw) total += cost(k, y, x0);
    }
    std::vector<int64_t> cb(G + 1, N);
    cb[0] = 0;
    int b = 1;
    double acc = 0.0;
    int64_t base = 0;
    for (int k = 0; k < n && b < G; ++k) {
        for (int y = 0; y < nys[k] && b < G; ++y)
            for (int x0 = 0; x0 < nxs[k]; x0 += tw) {
                const double w = cost(k, y, x0);
                while (b < G && total * b / G <= acc + 0.5 * w) cb[b++] = base + (int64_t)y * nxs[k] + x0;
                acc += w;
            }
        base += (int64_t)nxs[k] * nys[k];
    }
    return cb;
}

// Equal strip-row counts (the forward and tangent stage kernels).
std::vector<int64_t> static_ranges(const std::vector<int32_t> &nxs, const std::vector<int32_t> &nys, int tw, int G)
{
    return strip_ranges(nxs, nys, tw, G, [](int, int, int) { return 1.0; });
}

// The adjoint's ranges for a single nx x ny instance: a strip-row that its
// scaled (mirror boundary) path handles costs 1 + beta.  Those are the
// strip-rows of rows 0, 1, ny-2, ny-1 and of the column strips that start
// at column <= 1 or reach column nx-2, the adjoint kernel's per-segment
// test applied row by row.
std::vector<int64_t> cost_balanced_ranges(int nx, int ny, int tw, int G, double beta)
{
    return strip_ranges(std::vector<int32_t>{nx}, std::vector<int32_t>{ny}, tw, G, [&](int, int y, int x0) {
        const bool scaled = y <= 1 || y >= ny - 2 || x0 <= 1 || x0 + tw >= nx - 1;
        return scaled ? 1.0 + beta : 1.0;
    });
}

// Static schedule: the cells of all instances (in plan order, row-major
// inside an instance) are cut into G ranges at strip-row starts, one per
// block (static_ranges: equal strip-row counts; cost_balanced_ranges for
// the adjoint); a block's range becomes column strips of 32*cx cells by row
// ranges, and those are cut into NW pieces with equal numbers of
// strip-rows, one per warp.  Every SM therefore gets the same FP64 work per
// stage, and so does each of its warps (to within one row).  With
// split_boundary_rows (the adjoint's schedule) no segment mixes the two
// first or last rows of an instance with its interior rows, so that the
// adjoint kernel's per-segment choice of its scaled boundary path matches
// the per-row cost of cost_balanced_ranges.
void static_schedule(const std::vector<int32_t> &nxs, const std::vector<int32_t> &nys, int cx, int G, int NW,
                     std::vector<cgk::Seg> &segs, std::vector<int32_t> &warp_seg,
                     const std::vector<int64_t> &ranges, bool split_boundary_rows = false)
{
    const int n = (int)nxs.size();
    std::vector<int64_t> cstart(n + 1, 0);
    for (int k = 0; k < n; ++k) cstart[k + 1] = cstart[k] + (int64_t)nxs[k] * nys[k];
    const int64_t N = cstart[n];
    const int tw = 32 * cx;
    segs.clear();
    warp_seg.assign((size_t)G * NW + 1, 0);
    int k0 = 0;
    for (int b = 0; b < G; ++b) {
        const int64_t c0 = ranges[b], c1 = ranges[b + 1];
        std::vector<cgk::Seg> bs;
        while (k0 < n && cstart[k0 + 1] <= c0) ++k0;
        for (int k = k0; k < n && cstart[k] < c1; ++k) {
            const int64_t l0 = std::max(c0, cstart[k]) - cstart[k];
            const int64_t l1 = std::min(c1, cstart[k + 1]) - cstart[k];
            if (l0 >= l1) continue;
            const int nx = nxs[k];
            const int ya = (int)(l0 / nx), yb = (int)((l1 - 1) / nx);
            const int fa0 = (int)(l0 % nx), fa1 = (ya == yb) ? (int)((l1 - 1) % nx) + 1 : nx;
            const int fb0 = 0, fb1 = (int)((l1 - 1) % nx) + 1;
            for (int x0 = 0; x0 < nx; x0 += tw) {
                const int x1 = std::min(nx, x0 + tw);
                const bool in_a = x1 > fa0 && x0 < fa1;
                const bool in_b = (yb > ya) ? (x1 > fb0 && x0 < fb1) : in_a;
                int r0 = in_a ? ya : ya + 1, r1 = in_b ? yb : yb - 1;
                if (ya == yb) {
                    if (!in_a) continue;
                    r0 = r1 = ya;
                }
                if (r0 > r1) continue;
                cgk::Seg sg;
                sg.inst = k; sg.x0 = x0; sg.y0 = r0; sg.y1 = r1;
                sg.mrow_a = ya; sg.ma0 = fa0; sg.ma1 = fa1;
                sg.mrow_b = (yb > ya) ? yb : -1; sg.mb0 = fb0; sg.mb1 = fb1;
                if (split_boundary_rows) {
                    // pieces that never mix rows 0, 1 or ny-2, ny-1 with
                    // interior rows (same rows, same order)
                    const int ny = nys[k];
                    for (int p : {2, ny - 2}) {
                        if (p > sg.y0 && p <= sg.y1) {
                            cgk::Seg head = sg;
                            head.y1 = p - 1;
                            bs.push_back(head);
                            sg.y0 = p;
                        }
                    }
                }
                bs.push_back(sg);
            }
        }
        int64_t total = 0;
        for (const auto &sg : bs) total += sg.y1 - sg.y0 + 1;
        // cut the block's strip-rows into NW consecutive shares
        size_t si = 0;
        int cur = bs.empty() ? 0 : bs[0].y0;     // next unassigned row of bs[si]
        int64_t pos = 0;
        for (int w = 0; w < NW; ++w) {
            warp_seg[(size_t)b * NW + w] = (int32_t)segs.size();
            const int64_t end = total * (w + 1) / NW;
            while (pos < end && si < bs.size()) {
                cgk::Seg sg = bs[si];
                const int64_t avail = sg.y1 - cur + 1;
                const int64_t take = std::min<int64_t>(avail, end - pos);
                sg.y0 = cur;
                sg.y1 = (int)(cur + take - 1);
                segs.push_back(sg);
                pos += take;
                cur += (int)take;
                if (cur > bs[si].y1) {
                    ++si;
                    if (si < bs.size()) cur = bs[si].y0;
                }
            }
        }
    }
    warp_seg[(size_t)G * NW] = (int32_t)segs.size();
}

// For each block of the static schedule, the range of blocks that own its
// one-cell halo: every cell within one row and one column of the block's
// cells, inside the same instance.  Block b owns global cells
// [ranges[b], ranges[b+1]); the owner of cell c is the last block whose
// range starts at or before c.
void halo_dependencies(const std::vector<int32_t> &nxs, const std::vector<int32_t> &nys, int G,
                       const std::vector<int64_t> &ranges, std::vector<int2> &deps)
{
    const int n = (int)nxs.size();
    std::vector<int64_t> cstart(n + 1, 0);
    for (int k = 0; k < n; ++k) cstart[k + 1] = cstart[k] + (int64_t)nxs[k] * nys[k];
    auto owner = [&](int64_t c) {
        return (int)(std::upper_bound(ranges.begin(), ranges.begin() + G, c) - ranges.begin()) - 1;
    };
    deps.assign(G, make_int2(0, -1));
    int k0 = 0;
    for (int b = 0; b < G; ++b) {
        const int64_t c0 = ranges[b], c1 = ranges[b + 1];
        int lo = b, hi = b;
        while (k0 < n && cstart[k0 + 1] <= c0) ++k0;
        for (int k = k0; k < n && cstart[k] < c1; ++k) {
            const int64_t l0 = std::max(c0, cstart[k]) - cstart[k];
            const int64_t l1 = std::min(c1, cstart[k + 1]) - cstart[k];
            if (l0 >= l1) continue;
            const int64_t nx = nxs[k], cells = (int64_t)nxs[k] * nys[k];
            const int64_t h0 = std::max<int64_t>(0, l0 - nx - 1), h1 = std::min<int64_t>(cells, l1 + nx + 1);
            lo = std::min(lo, owner(cstart[k] + h0));
            hi = std::max(hi, owner(cstart[k] + h1 - 1));
        }
        deps[b] = make_int2(lo, hi);
    }
}

// Tiles of the temporally blocked kernel: about one tile per SM, square
// unless the grid is thinner than that, every tile resident at once (the
// launch is cooperative), the window (tile plus k n_s halo cells, clipped
// at the ghost layer) in shared memory.
// Tiles of the temporally blocked kernel: one uniform tile size for all
// instances (clipped at their edges), windows (tile + halo) that fit shared
// memory.  One instance: one tile per block, the tiles grown until they are
// all resident together.  A batch: the largest square tile whose window
// fits, blocks looping over the tiles.
cg_status tb_setup(cg_plan_s *P)
{
    P->tb_kernel = lookup_tb_kernel(P->kmodel, P->stencil, P->scheme);
    if (!P->tb_kernel) return fail(CG_EUNSUPPORTED, "no temporally blocked kernel for this problem");
    const int H = P->tb_k * P->ns;
    int dev_smem = 0;
    cudaError_t e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
    if (e != cudaSuccess) return cuda_fail(e, "device attribute");
    const bool single = P->inst.size() == 1;
    int maxnx = 1, maxny = 1;
    int64_t cells = 0;
    for (const Inst &I : P->inst) {
        maxnx = std::max(maxnx, I.nx);
        maxny = std::max(maxny, I.ny);
        cells += (int64_t)I.nx * I.ny;
    }
    // largest window of tiles tx x ty over all instances, and the tile count
    auto windows = [&](int tx, int ty, int &wmax, int64_t &ntiles) {
        wmax = 0;
        ntiles = 0;
        for (const Inst &I : P->inst) {
            const int tiles_x = (I.nx + tx - 1) / tx, tiles_y = (I.ny + ty - 1) / ty;
            ntiles += (int64_t)tiles_x * tiles_y;
            // a window's width and height depend on its column and row alone
            int wx = 0, wy = 0;
            for (int bx = 0; bx < tiles_x; ++bx) {
                int w0, w1;
                cgk::tb_window(bx * tx, std::min(bx * tx + tx, I.nx), I.nx, H, w0, w1);
                wx = std::max(wx, w1 - w0);
            }
            for (int by = 0; by < tiles_y; ++by) {
                int h0, h1;
                cgk::tb_window(by * ty, std::min(by * ty + ty, I.ny), I.ny, H, h0, h1);
                wy = std::max(wy, h1 - h0);
            }
            wmax = std::max(wmax, wx * wy);
        }
    };
    auto finish = [&](int tx, int ty, int wmax, int64_t ntiles, int blocks, size_t smem) {
        P->tb_tx = tx;
        P->tb_ty = ty;
        P->tb_wmax = wmax;
        P->tb_smem = smem;
        P->tb_tiles = (int32_t)ntiles;
        P->tb_blocks = blocks;
        int32_t begin = 0;
        for (Inst &I : P->inst) {
            I.tb_tiles_x = (I.nx + tx - 1) / tx;
            I.tb_tile_begin = begin;
            begin += I.tb_tiles_x * ((I.ny + ty - 1) / ty);
        }
        return CG_OK;
    };
    auto occupancy = [&](size_t smem, int &occ) -> cg_status {
        cudaError_t err = cudaFuncSetAttribute(P->tb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return cuda_fail(err, "shared memory attribute");
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, P->tb_kernel, P->tb_threads, smem);
        if (err != cudaSuccess) return cuda_fail(err, "occupancy query");
        return CG_OK;
    };
    const size_t inst_smem = sizeof(Inst) + 16;
    const int64_t per = (cells + P->num_sms - 1) / P->num_sms;
    if (single) {
        const int nx = P->inst[0].nx, ny = P->inst[0].ny;
        // Tile shape with the least FP64 time on the busiest SM.  Stage g of
        // a pass (H stages) evaluates the tile grown by H - g cells on each
        // side, clipped to the domain and, where it reaches an edge, with
        // its ghost ring (not at the last stage), packed into whole warps;
        // the FP64 pipe takes a warp instruction in the same time whatever
        // its active lanes, so a pass costs the busiest tile's sum over the
        // stages of ceil(cells / 32) warp-evaluations.  Among the shapes from
        // 3/4 to 3/2 of the square side that give at most one tile per SM,
        // the cheapest wins (then the fewer tiles, then the squarer); small
        // grids only (side <= 48), else the search below.
        const int s0 = (int)std::ceil(std::sqrt((double)per));
        if (s0 <= 48) {
            auto widths = [&](int n, int t, std::vector<int> &w) {        // [tile][g - 1]
                const int nt = (n + t - 1) / t;
                w.assign((size_t)nt * H, 0);
                for (int b = 0; b < nt; ++b)
                    for (int g = 1; g <= H; ++g) {
                        const int rad = H - g, t0 = b * t, t1 = std::min(n, t0 + t);
                        const bool gr = g < H;
                        const int lo = std::max(t0 - rad, 0), hi = std::min(t1 + rad, n);
                        w[(size_t)b * H + g - 1] = (hi + (gr && hi == n)) - (lo - (gr && lo == 0));
                    }
                return nt;
            };
            int64_t best = -1;
            int btx = 0, bty = 0, bn = 0;
            std::vector<int> wx, wy;
            for (int tx = std::max(1, s0 * 3 / 4); tx <= std::min(nx, s0 * 3 / 2); ++tx) {
                const int ntx = widths(nx, tx, wx);
                for (int ty = std::max(1, s0 * 3 / 4); ty <= std::min(ny, s0 * 3 / 2); ++ty) {
                    const int nty = (ny + ty - 1) / ty;
                    if ((int64_t)ntx * nty > P->num_sms) continue;
                    widths(ny, ty, wy);
                    int64_t worst = 0;
                    for (int bx = 0; bx < ntx; ++bx)
                        for (int by = 0; by < nty; ++by) {
                            int64_t c = 0;
                            for (int g = 0; g < H; ++g)
                                c += ((int64_t)wx[(size_t)bx * H + g] * wy[(size_t)by * H + g] + 31) / 32;
                            worst = std::max(worst, c);
                        }
                    const int n = ntx * nty;
                    if (best < 0 || worst < best || (worst == best && n < bn) ||
                        (worst == best && n == bn && std::abs(tx - ty) < std::abs(btx - bty))) {
                        best = worst;
                        btx = tx;
                        bty = ty;
                        bn = n;
                    }
                }
            }
            if (best >= 0) {
                int wmax = 0;
                int64_t ntiles = 0;
                windows(btx, bty, wmax, ntiles);
                const size_t smem = cgk::tb_smem_bytes(P->nv, P->ns, wmax);
                int occ = 0;
                if (smem + inst_smem <= (size_t)dev_smem) {
                    const cg_status st = occupancy(smem, occ);
                    if (st != CG_OK) return st;
                }
                if (occ >= 1 && ntiles <= (int64_t)occ * P->num_sms) {
                    P->tb_tiles_x = (nx + btx - 1) / btx;
                    P->tb_tiles_y = (ny + bty - 1) / bty;
                    P->tb_nbr = ((P->flags & CG_FLAG_NEIGHBOR_SYNC) && ntiles <= cgk::MAX_FLAG_BLOCKS) ? 1 : 0;
                    return finish(btx, bty, wmax, ntiles, (int)ntiles, smem);
                }
            }
        }
        int ty = s0, tx = ty;
        if (ty > ny) {
            ty = ny;
            tx = (int)((per + ny - 1) / ny);
        }
        tx = std::max(1, std::min(tx, nx));
        for (int attempt = 0; attempt < 4096; ++attempt) {
            int wmax = 0;
            int64_t ntiles = 0;
            windows(tx, ty, wmax, ntiles);
            const size_t smem = cgk::tb_smem_bytes(P->nv, P->ns, wmax);
            if (smem + inst_smem > (size_t)dev_smem)
                return fail(CG_EUNSUPPORTED, "temporal blocking: a tile and its halo (%d steps) need %zu bytes of "
                                             "shared memory, the device has %d", P->tb_k, smem, dev_smem);
            int occ = 0;
            const cg_status st = occupancy(smem, occ);
            if (st != CG_OK) return st;
            if (occ >= 1 && ntiles <= (int64_t)occ * P->num_sms) {
                // CG_FLAG_NEIGHBOR_SYNC: each block waits between passes
                // for the tiles its window covers only (one flag per tile)
                P->tb_tiles_x = (nx + tx - 1) / tx;
                P->tb_tiles_y = (ny + ty - 1) / ty;
                P->tb_nbr = ((P->flags & CG_FLAG_NEIGHBOR_SYNC) && ntiles <= cgk::MAX_FLAG_BLOCKS) ? 1 : 0;
                return finish(tx, ty, wmax, ntiles, (int)ntiles, smem);
            }
            // too many tiles to be resident together: make them larger
            if (tx < nx && (tx <= ty || ty >= ny)) ++tx;
            else if (ty < ny) ++ty;
            else break;
        }
        return fail(CG_EUNSUPPORTED, "temporal blocking: no tile size fits this device");
    }
    int side = (int)std::ceil(std::sqrt((double)per));
    side = std::max(1, std::min(side, std::max(maxnx, maxny)));
    for (;;) {
        const int tx = std::min(side, maxnx), ty = std::min(side, maxny);
        int wmax = 0;
        int64_t ntiles = 0;
        windows(tx, ty, wmax, ntiles);
        const size_t smem = cgk::tb_smem_bytes(P->nv, P->ns, wmax);
        if (smem + inst_smem <= (size_t)dev_smem && ntiles < (int64_t)1 << 30) {
            int occ = 0;
            const cg_status st = occupancy(smem, occ);
            if (st != CG_OK) return st;
            if (occ >= 1) {
                const int64_t resident = (int64_t)occ * P->num_sms;
                return finish(tx, ty, wmax, ntiles, (int)std::min<int64_t>(ntiles, resident), smem);
            }
        }
        if (side == 1)
            return fail(CG_EUNSUPPORTED, "temporal blocking: a 1 x 1 tile and its halo (%d steps) do not fit "
                                         "shared memory", P->tb_k);
        side = std::max(1, side * 7 / 8);
    }
}

cg_status make_plan(const cg_problem *probs, int32_t n_inst, const cg_tuning *tune, cg_plan *out)
{
    if (!out) return fail(CG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!probs || n_inst < 1) return fail(CG_EINVAL, "need at least one problem");
    for (int i = 0; i < n_inst; ++i) {
        cg_status st = validate(&probs[i], i);
        if (st != CG_OK) return st;
        if (i > 0 && !same_config(probs[0], probs[i]))
            return fail(CG_EINVAL, "problem %d: batch instances must share model, stencil, bc, scheme, "
                                   "dt, params and flags", i);
    }
    const cg_problem &p0 = probs[0];
    cg_plan_s *P = new (std::nothrow) cg_plan_s();
    if (!P) return fail(CG_ENOMEM, "plan allocation failed");
    P->model = p0.model;
    // The 9-point operator with alpha_d = 0 is the 5-point one (zero corner
    // weights), and the 9-point kernels need wd != 0 (row-sum form).
    P->stencil = (p0.stencil == CG_STENCIL9 && p0.alpha_d == 0.0) ? CG_STENCIL5 : p0.stencil;
    P->bc = p0.bc;
    P->scheme = p0.scheme;
    P->kmodel = kernel_model(p0.model, p0.flags);
    P->nv = n_fields(p0.model);
    P->ns = n_stages(p0.scheme);
    P->flags = p0.flags;
    P->dt = p0.dt;
    for (int f = 0; f < 4; ++f) P->dxx[f] = p0.Dxx[f];
    const double tmo = p0.barrier_timeout_s > 0 ? p0.barrier_timeout_s : 10.0;
    P->timeout_ns = (uint64_t)(std::min(tmo, 3600.0) * 1e9);

    // launch shape
    int64_t max_n = 0;
    for (int i = 0; i < n_inst; ++i) max_n = std::max<int64_t>(max_n, probs[i].nx);
    P->cx = (max_n >= 64) ? 2 : 1;
    P->rows = 4;
    P->threads = 512;
    P->bpsm = 1;
    P->sched = cgk::SCHED_STATIC;
    if (tune && tune->schedule == cgk::SCHED_TBLOCK) {
        // temporal blocking of cg_run; the plan's other kernels keep the
        // default launch shape
        P->tb_k = tune->rows ? tune->rows : 2;
        P->tb_threads = tune->threads ? tune->threads : 256;
        if (p0.bc == CG_BC_PERIODIC || gate_scheme(p0.scheme)) {
            delete P;
            return fail(CG_EUNSUPPORTED, "temporal blocking needs mirror or clamp ghosts and an explicit Euler, "
                                         "Heun or RK4 scheme");
        }
        if (P->tb_k < 1 || P->tb_k > 64 || P->tb_threads < 64 || P->tb_threads > 512 || (P->tb_threads % 32)) {
            delete P;
            return fail(CG_EINVAL, "temporal blocking: rows (steps per pass) in [1, 64], threads a multiple of "
                                   "32 in [64, 512]");
        }
    } else if (tune) {
        if (tune->cells_x) P->cx = tune->cells_x;
        if (tune->rows) P->rows = tune->rows;
        if (tune->threads) P->threads = tune->threads;
        if (tune->blocks_per_sm) P->bpsm = tune->blocks_per_sm;
        P->sched = tune->schedule;
    }
    if (P->sched != cgk::SCHED_STATIC && P->sched != cgk::SCHED_QUEUE) {
        delete P;
        return fail(CG_EINVAL, "tuning.schedule must be 0 (static), 1 (queue) or 2 (temporal blocking)");
    }
    if ((P->cx != 1 && P->cx != 2) || P->rows < 1 || P->rows > 4096 ||
        P->threads < 64 || P->threads > 512 || (P->threads % 32) != 0 || P->bpsm < 1 || P->bpsm > 8) {
        delete P;
        return fail(CG_EINVAL, "tuning out of range (cells_x 1|2, rows >= 1, threads a multiple of 32 in "
                               "[64, 512], blocks_per_sm 1..8)");
    }
    P->kernel = lookup_kernel(P->kmodel, P->stencil, P->scheme, P->cx);
    if (!P->kernel) {
        delete P;
        return fail(CG_EUNSUPPORTED, "no kernel for this model/stencil/scheme");
    }

    // instances: packed offsets in user order, tiles largest-first
    P->offsets.resize(n_inst + 1);
    P->offsets[0] = 0;
    for (int i = 0; i < n_inst; ++i) {
        int64_t sz = (int64_t)P->nv * probs[i].nx * probs[i].ny;
        P->offsets[i + 1] = P->offsets[i] + sz;
    }
    std::vector<int32_t> ord(n_inst);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        return probs[a].nx * probs[a].ny > probs[b].nx * probs[b].ny;
    });
    P->order.assign(n_inst, 0);
    P->inst.resize(n_inst);
    const int tw = 32 * P->cx;
    int64_t tiles = 0, scratch = 0;
    for (int k = 0; k < n_inst; ++k) {
        const int i = ord[k];
        P->order[i] = k;
        const cg_problem &p = probs[i];
        Inst &I = P->inst[k];
        std::memset(&I, 0, sizeof I);
        I.nx = (int32_t)p.nx;
        I.ny = (int32_t)p.ny;
        I.tiles_x = (int32_t)((p.nx + tw - 1) / tw);
        I.tiles_y = (int32_t)((p.ny + P->rows - 1) / P->rows);
        I.tile_begin = (int32_t)tiles;
        I.off = P->offsets[i];
        I.vec_ok = ((p.nx % 2) == 0 && (I.off % 2) == 0) ? 1 : 0;
        I.ws_off = scratch;
        fold_constants(*P, p, I);
        tiles += (int64_t)I.tiles_x * I.tiles_y;
        int64_t blk = (int64_t)cgk::SCRATCH_PLANES * P->nv * p.nx * p.ny;
        scratch += (blk + 31) / 32 * 32;     // keep blocks 256-byte aligned
    }
    if (tiles > 0x7fffffff) {
        delete P;
        return fail(CG_EINVAL, "too many tiles (%lld)", (long long)tiles);
    }
    P->n_tiles = (int32_t)tiles;
    P->scratch_elems = scratch;

    // Runge-Kutta combine weights (Sect. 3): acc += b_s dt F, Y_{s+1} = z + a dt F
    const double dt = P->dt;
    if (P->scheme == CG_EULER || gate_scheme(P->scheme)) {
        P->cacc[0] = dt;
    } else if (P->scheme == CG_HEUN) {
        P->cacc[0] = dt / 2; P->cacc[1] = dt / 2;
        P->cy[0] = dt;
    } else {
        P->cacc[0] = dt / 6; P->cacc[1] = dt / 3; P->cacc[2] = dt / 3; P->cacc[3] = dt / 6;
        P->cy[0] = dt / 2; P->cy[1] = dt / 2; P->cy[2] = dt;
    }

    // device table and persistent grid
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess && P->model == CG_BOCF)
        e = cgk::bocf_rcp_constants(P->mp[cgk::BP_TS1], P->mp[cgk::BD_DTS], &P->mp[cgk::BD_RS0]);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, P->kernel, P->threads, 0);
    if (e == cudaSuccess && occ < 1) {
        delete P;
        return fail(CG_EUNSUPPORTED, "kernel cannot run with %d threads per block", P->threads);
    }
    if (e == cudaSuccess) {
        P->nblocks = P->num_sms * std::min(P->bpsm, occ);
        std::vector<int32_t> nxs, nys;
        for (const Inst &I : P->inst) { nxs.push_back(I.nx); nys.push_back(I.ny); }
        const std::vector<int64_t> rg = static_ranges(nxs, nys, 32 * P->cx, P->nblocks);
        static_schedule(nxs, nys, P->cx, P->nblocks, P->threads / 32, P->segs, P->warp_seg, rg);
        halo_dependencies(nxs, nys, P->nblocks, rg, P->deps);
        P->sync_mode = (P->sched == cgk::SCHED_STATIC && P->nblocks <= cgk::MAX_FLAG_BLOCKS &&
                        P->bc != CG_BC_PERIODIC &&
                        (P->flags & CG_FLAG_NEIGHBOR_SYNC)) ? cgk::SYNC_NEIGHBOR : cgk::SYNC_GRID;
        if (P->inst.size() == 1 && P->bc == CG_BC_MIRROR && !gate_scheme(P->scheme) &&
            P->sync_mode == cgk::SYNC_GRID) {
            const std::vector<int64_t> cb =
                cost_balanced_ranges(nxs[0], nys[0], 32 * P->cx, P->nblocks, ADJ_BOUNDARY_COST);
            static_schedule(nxs, nys, P->cx, P->nblocks, P->threads / 32, P->segs_adj, P->warp_seg_adj, cb, true);
        }
    }
    if (e == cudaSuccess && P->tb_k > 0) {
        const cg_status st = tb_setup(P);
        if (st != CG_OK) {
            delete P;
            return st;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&P->d_deps, sizeof(int2) * std::max<size_t>(1, P->deps.size()));
    if (e == cudaSuccess && !P->deps.empty())
        e = cudaMemcpy(P->d_deps, P->deps.data(), sizeof(int2) * P->deps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_tab, sizeof(double) * cgk::EXP_TAB);
    if (e == cudaSuccess) {
        double tab[cgk::EXP_TAB];
        cgk::exp_table(tab, cgk::EXP_TAB);
        e = cudaMemcpy(P->d_tab, tab, sizeof tab, cudaMemcpyHostToDevice);
        for (Inst &I : P->inst) I.tab = P->d_tab;
    }
    if (e == cudaSuccess) e = cudaMalloc(&P->d_inst, sizeof(Inst) * n_inst);
    if (e == cudaSuccess)
        e = cudaMemcpy(P->d_inst, P->inst.data(), sizeof(Inst) * n_inst, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_segs, sizeof(cgk::Seg) * std::max<size_t>(1, P->segs.size()));
    if (e == cudaSuccess && !P->segs.empty())
        e = cudaMemcpy(P->d_segs, P->segs.data(), sizeof(cgk::Seg) * P->segs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_warp_seg, sizeof(int32_t) * P->warp_seg.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(P->d_warp_seg, P->warp_seg.data(), sizeof(int32_t) * P->warp_seg.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !P->warp_seg_adj.empty()) {
        e = cudaMalloc(&P->d_segs_adj, sizeof(cgk::Seg) * std::max<size_t>(1, P->segs_adj.size()));
        if (e == cudaSuccess && !P->segs_adj.empty())
            e = cudaMemcpy(P->d_segs_adj, P->segs_adj.data(), sizeof(cgk::Seg) * P->segs_adj.size(),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&P->d_warp_seg_adj, sizeof(int32_t) * P->warp_seg_adj.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(P->d_warp_seg_adj, P->warp_seg_adj.data(), sizeof(int32_t) * P->warp_seg_adj.size(),
                           cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        if (P->d_inst) cudaFree(P->d_inst);
        if (P->d_segs) cudaFree(P->d_segs);
        if (P->d_warp_seg) cudaFree(P->d_warp_seg);
        if (P->d_segs_adj) cudaFree(P->d_segs_adj);
        if (P->d_warp_seg_adj) cudaFree(P->d_warp_seg_adj);
        if (P->d_deps) cudaFree(P->d_deps);
        if (P->d_tab) cudaFree(P->d_tab);
        delete P;
        return cuda_fail(e, "plan creation");
    }
    *out = P;
    g_err.clear();
    return CG_OK;
}

// Run global stages [g0, g1) of a kernel whose first argument is `a`: one
// cooperative persistent launch (grid barriers between stages), or with
// CG_FLAG_PER_STAGE_LAUNCH one ordinary launch of `stage_grid` blocks per
// stage.
cg_status launch_stages(cg_plan P, const void *kernel, void **args, RunArgs &a, int64_t g0, int64_t g1,
                        int stage_grid, cudaStream_t s)
{
    cudaError_t e;
    if (g1 <= g0) return CG_OK;
    if (P->flags & CG_FLAG_PER_STAGE_LAUNCH) {
        a.persistent = 0;
        for (int64_t g = g0; g < g1; ++g) {
            a.g_begin = g;
            a.g_end = g + 1;
            e = cudaLaunchKernel(kernel, dim3(stage_grid), dim3(P->threads), args, 0, s);
            if (e != cudaSuccess) return cuda_fail(e, "stage kernel launch");
        }
        return CG_OK;
    }
    a.persistent = 1;
    a.g_begin = g0;
    a.g_end = g1;
    a.nblocks_expect = (uint32_t)P->nblocks;
    // neighbour waits count stages in 32-bit flags: longer launches take
    // the grid barrier (64-bit arrival counter)
    if (a.sync_mode == cgk::SYNC_NEIGHBOR && g1 - g0 >= ((int64_t)1 << 31)) a.sync_mode = cgk::SYNC_GRID;
    if (a.sync_mode == cgk::SYNC_NEIGHBOR) {
        e = cudaMemsetAsync(a.flags, 0, sizeof(unsigned) * (size_t)P->nblocks, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(flags)");
    } else {
        e = cudaMemsetAsync(a.sync, 0, sizeof(unsigned long long), s);   // grid-barrier arrival counter
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(barrier)");
    }
    a.stuck_barrier = (P->flags & CG_FLAG_TEST_STUCK_BARRIER) ? 1u : 0u;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3(P->nblocks);
    cfg.blockDim = dim3(P->threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, kernel, args);
    if (e != cudaSuccess) return cuda_fail(e, "persistent kernel launch");
    return CG_OK;
}

// Co-residency of a secondary kernel (tangent / adjoint) on the plan's grid.
cg_status check_coresident(cg_plan P, const void *kernel)
{
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, P->threads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (occ * P->num_sms < P->nblocks)
        return fail(CG_EUNSUPPORTED, "kernel fits %d blocks per SM; the plan's grid needs %d", occ,
                    (P->nblocks + P->num_sms - 1) / P->num_sms);
    return CG_OK;
}

int64_t round32(int64_t n) { return (n + 31) / 32 * 32; }

cg_status check_plan_device(cg_plan P)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != P->device) return fail(CG_EINVAL, "plan was made on device %d, current device is %d", P->device, dev);
    return CG_OK;
}

}  // namespace

// ------------------------------------------------------------------ ABI

CG_API cg_status cg_plan_create(const cg_problem *prob, cg_plan *out)
{
    return make_plan(prob, 1, nullptr, out);
}

CG_API cg_status cg_plan_create_tuned(const cg_problem *prob, const cg_tuning *tuning, cg_plan *out)
{
    cgk::NvtxRange nvtx_range("cg_plan_create");
    return make_plan(prob, 1, tuning, out);
}

CG_API cg_status cg_batch_create(const cg_problem *probs, int32_t n_inst, const cg_tuning *tuning,
                                 cg_plan *out)
{
    cgk::NvtxRange nvtx_range("cg_batch_create");
    return make_plan(probs, n_inst, tuning, out);
}

CG_API cg_status cg_batch_offsets(cg_plan plan, int64_t *offsets)
{
    if (!plan || !offsets) return fail(CG_EINVAL, "NULL argument");
    std::copy(plan->offsets.begin(), plan->offsets.end(), offsets);
    return CG_OK;
}

CG_API int32_t cg_plan_n_instances(cg_plan plan)
{
    return plan ? (int32_t)plan->inst.size() : 0;
}

CG_API cg_status cg_plan_destroy(cg_plan plan)
{
    if (!plan) return CG_OK;
    if (plan->d_inst) cudaFree(plan->d_inst);
    if (plan->d_segs) cudaFree(plan->d_segs);
    if (plan->d_warp_seg) cudaFree(plan->d_warp_seg);
    if (plan->d_segs_adj) cudaFree(plan->d_segs_adj);
    if (plan->d_warp_seg_adj) cudaFree(plan->d_warp_seg_adj);
    if (plan->d_deps) cudaFree(plan->d_deps);
    if (plan->d_tab) cudaFree(plan->d_tab);
    delete plan;
    return CG_OK;
}

// Bytes of the per-instance pointer tables of cg_batch_run at the end of
// the workspace (input then output pointers, plan order).
static size_t ptr_table_bytes(cg_plan plan)
{
    return (2 * plan->inst.size() * sizeof(void *) + 255) / 256 * 256;
}

static size_t ptr_table_offset(cg_plan plan)
{
    return (cgk::WS_HEADER + (size_t)plan->scratch_elems * sizeof(double) + 255) / 256 * 256;
}

CG_API cg_status cg_workspace_size(cg_plan plan, size_t *bytes)
{
    if (!plan || !bytes) return fail(CG_EINVAL, "NULL argument");
    *bytes = ptr_table_offset(plan) + ptr_table_bytes(plan);
    return CG_OK;
}

namespace {

// Up to 120 pointers written into a device table by one launch (the values
// travel in the kernel's parameters, so the call can be graph-captured).
struct PtrChunk {
    const double *p[120];
    int32_t n, base;
};

__global__ void k_set_ptrs(const double **dst, PtrChunk c)
{
    const int i = threadIdx.x;
    if (i < c.n) dst[c.base + i] = c.p[i];
}

// Shared body of cg_run (packed state: z_in, z_out) and cg_batch_run
// (per-instance buffers in user order: zin_u, zout_u).
cg_status run_impl(cg_plan plan, const double *z_in, double *z_out, const double *const *zin_u,
                   double *const *zout_u, int64_t n_steps, void *workspace, void *stream)
{
    const bool tab = (zin_u != nullptr);
    const size_t n_inst = plan->inst.size();
    cg_status st = check_plan_device(plan);
    if (st != CG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    // per-instance buffers in plan order, and whether any is stepped in place
    std::vector<const double *> pin(n_inst);
    std::vector<double *> pout(n_inst);
    bool any_alias = false;
    for (size_t i = 0; i < n_inst; ++i) {
        const size_t k = (size_t)plan->order[i];
        pin[k] = tab ? zin_u[i] : z_in + plan->inst[k].off;
        pout[k] = tab ? zout_u[i] : z_out + plan->inst[k].off;
        any_alias |= (pin[k] == pout[k]);
    }
    note_run(plan, ws, s);
    cudaError_t e = cudaMemsetAsync(ws, 0, cgk::WS_HEADER, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
    auto inst_bytes = [&](size_t k) {
        const Inst &I = plan->inst[k];
        return sizeof(double) * (size_t)plan->nv * I.nx * I.ny;
    };
    if (n_steps == 0) {
        for (size_t k = 0; k < n_inst; ++k) {
            if (pin[k] == pout[k]) continue;
            e = cudaMemcpyAsync(pout[k], pin[k], inst_bytes(k), cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        }
        return CG_OK;
    }

    RunArgs a;
    std::memset(&a, 0, sizeof a);
    a.inst = plan->d_inst;
    a.segs = plan->d_segs;
    a.warp_seg = plan->d_warp_seg;
    a.sched = plan->sched;
    const cg_plan_s *P = plan;
    a.n_inst = (int32_t)n_inst;
    a.n_tiles = plan->n_tiles;
    a.bc = plan->bc;
    a.rows = plan->rows;
    a.z_in = z_in;
    a.z_out = z_out;
    if (tab) {
        double **t = reinterpret_cast<double **>(ws + ptr_table_offset(plan));
        for (size_t b0 = 0; b0 < 2 * n_inst; b0 += 120) {
            PtrChunk c;
            std::memset(&c, 0, sizeof c);
            c.base = (int32_t)b0;
            c.n = (int32_t)std::min<size_t>(120, 2 * n_inst - b0);
            for (int j = 0; j < c.n; ++j) {
                const size_t q = b0 + j;
                c.p[j] = q < n_inst ? pin[q] : pout[q - n_inst];
            }
            k_set_ptrs<<<1, 128, 0, s>>>(const_cast<const double **>(t), c);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "pointer table");
        }
        a.zin_tab = t;
        a.zout_tab = t + n_inst;
    }
    a.ws = reinterpret_cast<double *>(ws + cgk::WS_HEADER);
    a.sync = reinterpret_cast<unsigned *>(ws + cgk::WS_SYNC_OFF);
    a.status = reinterpret_cast<uint32_t *>(ws + cgk::WS_STATUS_OFF);
    a.flags = reinterpret_cast<unsigned *>(ws + cgk::WS_FLAGS_OFF);
    a.deps = P->d_deps;
    a.sync_mode = P->sync_mode;
    // one-stage steps in place would overwrite their own input: alternate
    // through the scratch copy, starting there (parity 1)
    const bool alias_single_stage = (plan->ns == 1) && any_alias;
    a.parity = alias_single_stage ? 1 : (int32_t)((n_steps - 1) & 1);
    a.timeout_ns = plan->timeout_ns;
    std::memcpy(a.cacc, plan->cacc, sizeof a.cacc);
    std::memcpy(a.cy, plan->cy, sizeof a.cy);
    std::memcpy(a.mp, plan->mp, sizeof a.mp);
    const int64_t G = n_steps * plan->ns;
    void *args[] = {&a};

    if (plan->tb_k > 0) {
        // temporally blocked: one cooperative launch, one grid barrier per
        // tb_k steps (cg_tblock.cuh)
        cgk::TbArgs t;
        std::memset(&t, 0, sizeof t);
        t.tx = plan->tb_tx;
        t.ty = plan->tb_ty;
        t.n_tiles = plan->tb_tiles;
        t.k = plan->tb_k;
        t.wmax = plan->tb_wmax;
        t.n_steps = n_steps;
        const int64_t n_pass = (n_steps + plan->tb_k - 1) / plan->tb_k;
        // pass counts are 32-bit flags: longer runs take the grid barrier
        t.nbr = (plan->tb_nbr && n_pass < ((int64_t)1 << 31)) ? 1 : 0;
        t.tiles_x = plan->tb_tiles_x;
        t.tiles_y = plan->tb_tiles_y;
        {
            const int H = plan->tb_k * plan->ns;
            t.rx = (H + plan->tb_tx - 1) / plan->tb_tx;
            t.ry = (H + plan->tb_ty - 1) / plan->tb_ty;
        }
        a.persistent = 1;
        a.nblocks_expect = (uint32_t)plan->tb_blocks;
        a.stuck_barrier = (plan->flags & CG_FLAG_TEST_STUCK_BARRIER) ? 1u : 0u;
        if (t.nbr)
            e = cudaMemsetAsync(a.flags, 0, sizeof(unsigned) * (size_t)plan->tb_blocks, s);
        else
            e = cudaMemsetAsync(a.sync, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(pass synchronisation)");
        void *targs[] = {&a, &t};
        cudaLaunchConfig_t cfg;
        std::memset(&cfg, 0, sizeof cfg);
        cfg.gridDim = dim3(plan->tb_blocks);
        cfg.blockDim = dim3(plan->tb_threads);
        cfg.dynamicSmemBytes = plan->tb_smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelExC(&cfg, plan->tb_kernel, targs);
        if (e != cudaSuccess) return cuda_fail(e, "temporally blocked kernel launch");
        const int64_t passes = (n_steps + plan->tb_k - 1) / plan->tb_k;
        if (any_alias && ((passes - 1) & 1) == 0) {
            // in place with an odd number of passes: the result of each
            // in-place instance is in its scratch copy
            for (size_t k = 0; k < n_inst; ++k) {
                if (pin[k] != pout[k]) continue;
                e = cudaMemcpyAsync(pout[k], a.ws + plan->inst[k].ws_off, inst_bytes(k), cudaMemcpyDeviceToDevice,
                                    s);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(final)");
            }
        }
        return CG_OK;
    }
    const int wpb = plan->threads / 32;
    const int qgrid = (plan->sched == cgk::SCHED_STATIC) ? plan->nblocks : (plan->n_tiles + wpb - 1) / wpb;
    st = launch_stages(plan, plan->kernel, args, a, 0, G, qgrid, s);
    if (st != CG_OK) return st;
    if (alias_single_stage && (n_steps & 1)) {
        // odd number of single-stage steps: the last result sits in the
        // scratch copy of each instance
        for (size_t k = 0; k < n_inst; ++k) {
            e = cudaMemcpyAsync(pout[k], a.ws + plan->inst[k].ws_off, inst_bytes(k), cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(final)");
        }
    }
    return CG_OK;
}

}  // namespace

CG_API cg_status cg_run(cg_plan plan, const double *z_in, double *z_out, int64_t n_steps, void *workspace,
                        void *stream)
{
    cgk::NvtxRange nvtx_range("cg_run");
    if (!plan) return fail(CG_EINVAL, "plan is NULL");
    if (!z_in || !z_out || !workspace) return fail(CG_EINVAL, "NULL buffer");
    if (n_steps < 0 || n_steps > MAX_STEPS) return fail(CG_EINVAL, "n_steps out of range");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return fail(CG_EINVAL, "workspace must be 256-byte aligned");
    if ((reinterpret_cast<uintptr_t>(z_in) & 7) || (reinterpret_cast<uintptr_t>(z_out) & 7))
        return fail(CG_EINVAL, "state buffers must be 8-byte aligned");
    const int64_t total = plan->offsets.back();
    const size_t nbytes = (size_t)total * sizeof(double);
    if (z_in != z_out) {
        const char *a0 = reinterpret_cast<const char *>(z_in), *b0 = reinterpret_cast<const char *>(z_out);
        if (a0 < b0 + nbytes && b0 < a0 + nbytes) return fail(CG_EINVAL, "z_in and z_out partially overlap");
    }
    return run_impl(plan, z_in, z_out, nullptr, nullptr, n_steps, workspace, stream);
}

CG_API cg_status cg_batch_run(cg_plan plan, const double *const *z_in, double *const *z_out, int64_t n_steps,
                              void *workspace, void *stream)
{
    cgk::NvtxRange nvtx_range("cg_batch_run");
    if (!plan) return fail(CG_EINVAL, "plan is NULL");
    if (!z_in || !z_out || !workspace) return fail(CG_EINVAL, "NULL buffer");
    if (n_steps < 0 || n_steps > MAX_STEPS) return fail(CG_EINVAL, "n_steps out of range");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return fail(CG_EINVAL, "workspace must be 256-byte aligned");
    for (size_t i = 0; i < plan->inst.size(); ++i) {
        if (!z_in[i] || !z_out[i]) return fail(CG_EINVAL, "instance %zu: NULL buffer", i);
        if ((reinterpret_cast<uintptr_t>(z_in[i]) & 7) || (reinterpret_cast<uintptr_t>(z_out[i]) & 7))
            return fail(CG_EINVAL, "instance %zu: state buffers must be 8-byte aligned", i);
        const size_t nb = (size_t)(plan->offsets[i + 1] - plan->offsets[i]) * sizeof(double);
        const char *a0 = reinterpret_cast<const char *>(z_in[i]), *b0 = reinterpret_cast<const char *>(z_out[i]);
        if (a0 != b0 && a0 < b0 + nb && b0 < a0 + nb)
            return fail(CG_EINVAL, "instance %zu: z_in and z_out partially overlap", i);
    }
    return run_impl(plan, nullptr, nullptr, z_in, z_out, n_steps, workspace, stream);
}

CG_API cg_status cg_rhs(cg_plan plan, const double *z, double *f, void *workspace, void *stream)
{
    cgk::NvtxRange nvtx_range("cg_rhs");
    if (!plan) return fail(CG_EINVAL, "plan is NULL");
    if (!z || !f || !workspace) return fail(CG_EINVAL, "NULL buffer");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return fail(CG_EINVAL, "workspace must be 256-byte aligned");
    if ((reinterpret_cast<uintptr_t>(z) & 7) || (reinterpret_cast<uintptr_t>(f) & 7))
        return fail(CG_EINVAL, "state buffers must be 8-byte aligned");
    const size_t nbytes = (size_t)plan->offsets.back() * sizeof(double);
    const char *a0 = reinterpret_cast<const char *>(z), *b0 = reinterpret_cast<const char *>(f);
    if (a0 < b0 + nbytes && b0 < a0 + nbytes) return fail(CG_EINVAL, "z and f overlap");
    cg_status st = check_plan_device(plan);
    if (st != CG_OK) return st;
    // the one-stage (explicit Euler) kernel of the plan's model, stencil and
    // tile width, writing F itself
    const void *k = lookup_kernel(plan->kmodel, plan->stencil, CG_EULER, plan->cx);
    if (!k) return fail(CG_EUNSUPPORTED, "no kernel for this model/stencil");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    note_run(plan, ws, s);
    cudaError_t e = cudaMemsetAsync(ws, 0, cgk::WS_HEADER, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
    RunArgs a;
    std::memset(&a, 0, sizeof a);
    a.inst = plan->d_inst;
    a.segs = plan->d_segs;
    a.warp_seg = plan->d_warp_seg;
    a.sched = plan->sched;
    a.n_inst = (int32_t)plan->inst.size();
    a.n_tiles = plan->n_tiles;
    a.bc = plan->bc;
    a.rows = plan->rows;
    a.z_in = z;
    a.z_out = f;
    a.ws = reinterpret_cast<double *>(ws + cgk::WS_HEADER);
    a.sync = reinterpret_cast<unsigned *>(ws + cgk::WS_SYNC_OFF);
    a.status = reinterpret_cast<uint32_t *>(ws + cgk::WS_STATUS_OFF);
    a.flags = reinterpret_cast<unsigned *>(ws + cgk::WS_FLAGS_OFF);
    a.deps = plan->d_deps;
    a.timeout_ns = plan->timeout_ns;
    a.rhs_only = 1;
    a.persistent = 0;
    a.g_begin = 0;
    a.g_end = 1;
    a.cacc[0] = 1.0;
    std::memcpy(a.mp, plan->mp, sizeof a.mp);
    void *args[] = {&a};
    const int wpb = plan->threads / 32;
    const int grid = (plan->sched == cgk::SCHED_STATIC) ? plan->nblocks : (plan->n_tiles + wpb - 1) / wpb;
    e = cudaLaunchKernel(k, dim3(grid), dim3(plan->threads), args, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "rhs kernel launch");
    return CG_OK;
}

// Device state copies of cg_run_host sit after the cg_run workspace.
static size_t host_state_offset(cg_plan plan)
{
    size_t ws = 0;
    cg_workspace_size(plan, &ws);
    return (ws + 255) / 256 * 256;
}

CG_API cg_status cg_host_workspace_size(cg_plan plan, size_t *bytes)
{
    if (!plan || !bytes) return fail(CG_EINVAL, "bad argument");
    const size_t state = ((size_t)plan->offsets.back() * sizeof(double) + 255) / 256 * 256;
    *bytes = host_state_offset(plan) + 2 * state;
    return CG_OK;
}

CG_API cg_status cg_run_host(cg_plan plan, const double *z_in_host, double *z_out_host, int64_t n_steps,
                             void *workspace, void *stream)
{
    cgk::NvtxRange nvtx_range("cg_run_host");
    if (!plan) return fail(CG_EINVAL, "plan is NULL");
    if (!z_in_host || !z_out_host || !workspace) return fail(CG_EINVAL, "NULL buffer");
    if (n_steps < 0 || n_steps > MAX_STEPS) return fail(CG_EINVAL, "n_steps out of range");
    const size_t nbytes = (size_t)plan->offsets.back() * sizeof(double);
    char *ws = reinterpret_cast<char *>(workspace);
    double *d_in = reinterpret_cast<double *>(ws + host_state_offset(plan));
    double *d_out = reinterpret_cast<double *>(ws + host_state_offset(plan) + (nbytes + 255) / 256 * 256);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(d_in, z_in_host, nbytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(host to device)");
    cg_status st = cg_run(plan, d_in, d_out, n_steps, workspace, stream);
    if (st != CG_OK) return st;
    e = cudaMemcpyAsync(z_out_host, d_out, nbytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(device to host)");
    uint32_t flags = 0;
    return cg_read_status(plan, workspace, stream, &flags);
}

CG_API cg_status cg_get_device_status(cg_plan plan, uint32_t *flags)
{
    if (!plan || !flags) return fail(CG_EINVAL, "NULL argument");
    const void *ws;
    void *stream;
    {
        std::lock_guard<std::mutex> g(plan->last_mu);
        ws = plan->last_ws;
        stream = plan->last_stream;
    }
    if (!ws) {
        *flags = 0;
        return CG_OK;
    }
    return cg_read_status(plan, ws, stream, flags);
}

CG_API cg_status cg_read_status(cg_plan plan, const void *workspace, void *stream, uint32_t *flags)
{
    if (!plan || !workspace || !flags) return fail(CG_EINVAL, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    uint32_t v = 0;
    e = cudaMemcpy(&v, reinterpret_cast<const char *>(workspace) + cgk::WS_STATUS_OFF, sizeof v,
                   cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
    *flags = v;
    if (v & CG_DEV_BOUNDS) return fail(CG_EBOUNDS, "a device-side index check failed (status 0x%x)", v);
    if (v & CG_DEV_TIMEOUT) return fail(CG_ETIMEOUT, "a device-side wait gave up (status 0x%x)", v);
    if (v & CG_DEV_NONFINITE) return fail(CG_ENAN, "a non-finite value was written (status 0x%x)", v);
    return CG_OK;
}

// ----------------------------------------------------------- tangent-linear

namespace {

const void *lookup_tlm_kernel(int kmodel, int stencil, int scheme, int cx)
{
    switch (kmodel) {
    case cgk::MODEL_BOCFH: return cgk::tlm_kernel_bocfh(stencil, scheme, cx);
    case CG_FHN: return cgk::tlm_kernel_fhn(stencil, scheme, cx);
    case CG_BOCF: return cgk::tlm_kernel_bocf(stencil, scheme, cx);
    case CG_DIFFUSION: return cgk::tlm_kernel_diff(stencil, scheme, cx);
    case CG_KARMA: return cgk::tlm_kernel_karma(stencil, scheme, cx);
    default: return nullptr;
    }
}

// Stored Jacobian entries per cell of a kernel family (the models' own NJ;
// 0 for the linear model).
int model_nj(int kmodel)
{
    switch (kmodel) {
    case CG_FHN: return cgk::Model<cgk::MODEL_FHN>::NJ;
    case CG_BOCF: return cgk::Model<cgk::MODEL_BOCF>::NJ;
    case cgk::MODEL_BOCFH: return cgk::Model<cgk::MODEL_BOCFH>::NJ;
    case CG_KARMA: return cgk::Model<cgk::MODEL_KARMA>::NJ;
    case CG_DIFFUSION: return cgk::Model<cgk::MODEL_DIFF>::NJ;
    default: return 0;
    }
}

struct TlmLayout {
    size_t jbuf_off, tan_off, total;
    int64_t tstride, tblk, jstride;
    bool ok;               // false: the byte count does not fit (reported as CG_EINVAL)
};

// Workspace byte counts are formed in size_t; the same sum in double (exact
// to far better than the margin) tells whether it stayed below 2^62 bytes.
constexpr double WS_LIMIT = 4611686018427387904.0;   // 2^62

// Workspace of the tangent-linear runs: header | primal scratch | stage
// Jacobians (one stage, or n_jstages when linearized) | tangent scratch.
TlmLayout tlm_layout(cg_plan P, int32_t n_tan, int64_t n_jstages = 1)
{
    const Inst &I = P->inst[0];
    const int64_t plane = (int64_t)I.nx * I.ny;
    TlmLayout L;
    L.tstride = (int64_t)P->nv * plane;
    L.tblk = round32((int64_t)cgk::SCRATCH_PLANES * P->nv * plane);
    L.jstride = round32(std::max(1, model_nj(P->kmodel)) * plane);
    L.jbuf_off = cgk::WS_HEADER + (size_t)P->scratch_elems * sizeof(double);
    L.tan_off = L.jbuf_off + (size_t)std::max<int64_t>(1, n_jstages) * (size_t)L.jstride * sizeof(double);
    L.total = L.tan_off + (size_t)n_tan * (size_t)L.tblk * sizeof(double);
    const double est = (double)L.jbuf_off + (double)std::max<int64_t>(1, n_jstages) * (double)L.jstride * 8.0 +
                       (double)n_tan * (double)L.tblk * 8.0;
    L.ok = est < WS_LIMIT;
    return L;
}

bool overlaps(const void *a, const void *b, size_t n)
{
    const char *x = reinterpret_cast<const char *>(a), *y = reinterpret_cast<const char *>(b);
    return x != y && x < y + n && y < x + n;
}

// Fill the fields of RunArgs shared by every single-instance launch.
void base_args(cg_plan P, RunArgs &a, const double *z_in, double *z_out, char *ws)
{
    std::memset(&a, 0, sizeof a);
    a.inst = P->d_inst;
    a.segs = P->d_segs;
    a.warp_seg = P->d_warp_seg;
    a.sched = cgk::SCHED_STATIC;
    a.n_inst = (int32_t)P->inst.size();
    a.n_tiles = P->n_tiles;
    a.bc = P->bc;
    a.rows = P->rows;
    a.z_in = z_in;
    a.z_out = z_out;
    a.ws = reinterpret_cast<double *>(ws + cgk::WS_HEADER);
    a.sync = reinterpret_cast<unsigned *>(ws + cgk::WS_SYNC_OFF);
    a.status = reinterpret_cast<uint32_t *>(ws + cgk::WS_STATUS_OFF);
    a.flags = reinterpret_cast<unsigned *>(ws + cgk::WS_FLAGS_OFF);
    a.deps = P->d_deps;
    a.sync_mode = P->sync_mode;
    a.timeout_ns = P->timeout_ns;
    std::memcpy(a.cacc, P->cacc, sizeof a.cacc);
    std::memcpy(a.cy, P->cy, sizeof a.cy);
    std::memcpy(a.mp, P->mp, sizeof a.mp);
}

}  // namespace

CG_API cg_status cg_tlm_workspace_size(cg_plan plan, int32_t n_tangents, size_t *bytes)
{
    if (!plan || !bytes || n_tangents < 0) return fail(CG_EINVAL, "bad argument");
    if (plan->inst.size() != 1) return fail(CG_EUNSUPPORTED, "tangent-linear runs need a single-instance plan");
    if (gate_scheme(plan->scheme))
        return fail(CG_EUNSUPPORTED, "no tangent-linear model of the gate integrators");
    const TlmLayout L = tlm_layout(plan, n_tangents);
    if (!L.ok) return fail(CG_EINVAL, "workspace size overflows");
    *bytes = L.total;
    return CG_OK;
}

CG_API cg_status cg_tlm_run(cg_plan plan, const double *z0, const double *dz0, double *zT, double *dzT,
                            int32_t n_tangents, int64_t n_steps, void *workspace, void *stream)
{
    cgk::NvtxRange nvtx_range("cg_tlm_run");
    if (!plan) return fail(CG_EINVAL, "plan is NULL");
    if (plan->inst.size() != 1) return fail(CG_EUNSUPPORTED, "tangent-linear runs need a single-instance plan");
    if (gate_scheme(plan->scheme))
        return fail(CG_EUNSUPPORTED, "no tangent-linear model of the gate integrators");
    if (!z0 || !zT || !workspace || n_tangents < 0 || n_steps < 0 || n_steps > MAX_STEPS)
        return fail(CG_EINVAL, "bad argument");
    if (n_tangents > 0 && (!dz0 || !dzT)) return fail(CG_EINVAL, "NULL tangent buffer");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return fail(CG_EINVAL, "workspace must be 256-byte aligned");
    const TlmLayout L = tlm_layout(plan, n_tangents);
    if (!L.ok) return fail(CG_EINVAL, "workspace size overflows");
    const size_t sbytes = (size_t)L.tstride * sizeof(double);
    const size_t tbytes = sbytes * (size_t)n_tangents;
    if (overlaps(z0, zT, sbytes) || (n_tangents && overlaps(dz0, dzT, tbytes)))
        return fail(CG_EINVAL, "input and output partially overlap");
    if (plan->ns == 1 && n_steps > 0 && (z0 == zT || (n_tangents && dz0 == dzT)))
        return fail(CG_EINVAL, "in-place tangent-linear runs need a multi-stage scheme");
    cg_status st = check_plan_device(plan);
    if (st != CG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    note_run(plan, ws, s);
    cudaError_t e = cudaMemsetAsync(ws, 0, cgk::WS_HEADER, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
    if (n_steps == 0) {
        if (z0 != zT) e = cudaMemcpyAsync(zT, z0, sbytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && n_tangents && dz0 != dzT)
            e = cudaMemcpyAsync(dzT, dz0, tbytes, cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? CG_OK : cuda_fail(e, "cudaMemcpyAsync");
    }
    const void *k = lookup_tlm_kernel(plan->kmodel, plan->stencil, plan->scheme, plan->cx);
    if (!k) return fail(CG_EUNSUPPORTED, "no tangent-linear kernel for this problem");
    st = check_coresident(plan, k);
    if (st != CG_OK) return st;
    RunArgs a;
    base_args(plan, a, z0, zT, ws);
    a.parity = (int32_t)((n_steps - 1) & 1);
    cgk::TlmArgs t;
    std::memset(&t, 0, sizeof t);
    t.dz_in = dz0;
    t.dz_out = dzT;
    t.jbuf = reinterpret_cast<double *>(ws + L.jbuf_off);
    t.tws = reinterpret_cast<double *>(ws + L.tan_off);
    t.n_tan = n_tangents;
    t.tstride = L.tstride;
    t.tblk = L.tblk;
    void *args[] = {&a, &t};
    return launch_stages(plan, k, args, a, 0, n_steps * plan->ns, plan->nblocks, s);
}

CG_API cg_status cg_tlm_linearized_workspace_size(cg_plan plan, int32_t n_tangents, int64_t n_steps, size_t *bytes)
{
    if (!plan || !bytes || n_tangents < 0 || n_steps < 0 || n_steps > MAX_STEPS)
        return fail(CG_EINVAL, "bad argument");
    if (plan->inst.size() != 1) return fail(CG_EUNSUPPORTED, "tangent-linear runs need a single-instance plan");
    if (gate_scheme(plan->scheme))
        return fail(CG_EUNSUPPORTED, "no tangent-linear model of the gate integrators");
    const TlmLayout L = tlm_layout(plan, n_tangents, n_steps * plan->ns);
    if (!L.ok) return fail(CG_EINVAL, "workspace size overflows");
    *bytes = L.total;
    return CG_OK;
}

// Shared body of cg_tlm_linearize (primal, every stage's Jacobian kept) and
// cg_tlm_apply (tangents only, with those Jacobians).
static cg_status tlm_linearized(cg_plan plan, const double *z0, double *zT, const double *dz0, double *dzT,
                                int32_t n_tangents, int64_t n_steps, bool apply, void *workspace, void *stream)
{
    if (!plan) return fail(CG_EINVAL, "plan is NULL");
    if (plan->inst.size() != 1) return fail(CG_EUNSUPPORTED, "tangent-linear runs need a single-instance plan");
    if (gate_scheme(plan->scheme))
        return fail(CG_EUNSUPPORTED, "no tangent-linear model of the gate integrators");
    if (!workspace || n_tangents < 0 || n_steps < 0 || n_steps > MAX_STEPS)
        return fail(CG_EINVAL, "bad argument");
    if (apply ? (n_tangents > 0 && (!dz0 || !dzT)) : (!z0 || !zT)) return fail(CG_EINVAL, "NULL buffer");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return fail(CG_EINVAL, "workspace must be 256-byte aligned");
    const TlmLayout L = tlm_layout(plan, n_tangents, n_steps * plan->ns);
    if (!L.ok) return fail(CG_EINVAL, "workspace size overflows");
    const size_t sbytes = (size_t)L.tstride * sizeof(double);
    const size_t tbytes = sbytes * (size_t)n_tangents;
    if (!apply && overlaps(z0, zT, sbytes)) return fail(CG_EINVAL, "input and output partially overlap");
    if (apply && n_tangents && overlaps(dz0, dzT, tbytes)) return fail(CG_EINVAL, "input and output partially overlap");
    if (plan->ns == 1 && n_steps > 0 && (apply ? (n_tangents && dz0 == dzT) : (z0 == zT)))
        return fail(CG_EINVAL, "in-place tangent-linear runs need a multi-stage scheme");
    {
        std::lock_guard<std::mutex> g(plan->last_mu);
        auto &lin = plan->linearized;
        auto it = std::find_if(lin.begin(), lin.end(), [&](const auto &r) { return r.first == workspace; });
        if (apply) {
            if (it == lin.end() || it->second != n_steps)
                return fail(CG_EINVAL, "this workspace was not linearized with this plan over %lld steps",
                            (long long)n_steps);
        } else {
            if (it != lin.end()) lin.erase(it);
            if (lin.size() >= 16) lin.erase(lin.begin());
            lin.emplace_back(workspace, n_steps);
        }
    }
    cg_status st = check_plan_device(plan);
    if (st != CG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    note_run(plan, ws, s);
    cudaError_t e = cudaMemsetAsync(ws, 0, cgk::WS_HEADER, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
    if (n_steps == 0) {
        if (!apply && z0 != zT) e = cudaMemcpyAsync(zT, z0, sbytes, cudaMemcpyDeviceToDevice, s);
        if (apply && n_tangents && dz0 != dzT) e = cudaMemcpyAsync(dzT, dz0, tbytes, cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? CG_OK : cuda_fail(e, "cudaMemcpyAsync");
    }
    if (apply && n_tangents == 0) return CG_OK;
    const void *k = lookup_tlm_kernel(plan->kmodel, plan->stencil, plan->scheme, plan->cx);
    if (!k) return fail(CG_EUNSUPPORTED, "no tangent-linear kernel for this problem");
    st = check_coresident(plan, k);
    if (st != CG_OK) return st;
    RunArgs a;
    base_args(plan, a, apply ? nullptr : z0, apply ? nullptr : zT, ws);
    a.parity = (int32_t)((n_steps - 1) & 1);
    cgk::TlmArgs t;
    std::memset(&t, 0, sizeof t);
    t.dz_in = apply ? dz0 : nullptr;
    t.dz_out = apply ? dzT : nullptr;
    t.jbuf = reinterpret_cast<double *>(ws + L.jbuf_off);
    t.tws = reinterpret_cast<double *>(ws + L.tan_off);
    t.n_tan = apply ? n_tangents : 0;
    t.skip_primal = apply ? 1 : 0;
    t.tstride = L.tstride;
    t.tblk = L.tblk;
    t.jstride = L.jstride;
    void *args[] = {&a, &t};
    return launch_stages(plan, k, args, a, 0, n_steps * plan->ns, plan->nblocks, s);
}

CG_API cg_status cg_tlm_linearize(cg_plan plan, const double *z0, double *zT, int64_t n_steps, void *workspace,
                                  void *stream)
{
    cgk::NvtxRange nvtx_range("cg_tlm_linearize");
    return tlm_linearized(plan, z0, zT, nullptr, nullptr, 0, n_steps, false, workspace, stream);
}

CG_API cg_status cg_tlm_apply(cg_plan plan, const double *dz0, double *dzT, int32_t n_tangents, int64_t n_steps,
                              void *workspace, void *stream)
{
    cgk::NvtxRange nvtx_range("cg_tlm_apply");
    return tlm_linearized(plan, nullptr, nullptr, dz0, dzT, n_tangents, n_steps, true, workspace, stream);
}

// ------------------------------------------------------------------ adjoint

namespace {

const void *lookup_adj_kernel(int kmodel, int stencil, int scheme, int cx)
{
    switch (kmodel) {
    case cgk::MODEL_BOCFH: return cgk::adj_kernel_bocfh(stencil, scheme, cx);
    case CG_FHN: return cgk::adj_kernel_fhn(stencil, scheme, cx);
    case CG_BOCF: return cgk::adj_kernel_bocf(stencil, scheme, cx);
    case CG_DIFFUSION: return cgk::adj_kernel_diff(stencil, scheme, cx);
    case CG_KARMA: return cgk::adj_kernel_karma(stencil, scheme, cx);
    default: return nullptr;
    }
}

// Workspace of cg_adjoint_run: header | primal scratch | checkpoints |
// segment store | kb0 kb1 lam lacc | per-warp dL/dD partials.
struct AdjLayout {
    int64_t c, nseg, S;
    size_t cp_off, store_off, kb_off, part_off, total;
    bool ok;               // false: the byte count does not fit (reported as CG_EINVAL)
};

AdjLayout adj_layout(cg_plan P, int64_t n_steps, int32_t every)
{
    AdjLayout L;
    const Inst &I = P->inst[0];
    L.S = round32((int64_t)P->nv * I.nx * I.ny);
    L.c = every > 0 ? every : std::max<int64_t>(1, (int64_t)std::ceil(std::sqrt((double)std::max<int64_t>(1, n_steps))));
    L.c = std::min<int64_t>(L.c, std::max<int64_t>(1, n_steps));   // a segment never exceeds the horizon
    L.nseg = std::max<int64_t>(1, (n_steps + L.c - 1) / L.c);
    const size_t d = sizeof(double);
    L.cp_off = cgk::WS_HEADER + (size_t)P->scratch_elems * d;
    L.store_off = L.cp_off + (size_t)L.nseg * L.S * d;
    L.kb_off = L.store_off + (size_t)(L.c * P->ns + 1) * L.S * d;
    L.part_off = L.kb_off + (size_t)4 * L.S * d;
    const int nd = P->model == CG_FHN ? 2 : 1;
    L.total = L.part_off + (size_t)round32((int64_t)P->nblocks * (P->threads / 32) * nd) * d;
    const double dS = (double)L.S * 8.0;
    const double est = (double)L.cp_off + (double)L.nseg * dS + ((double)L.c * P->ns + 1.0) * dS + 4.0 * dS +
                       8.0 * (double)round32((int64_t)P->nblocks * (P->threads / 32) * nd);
    L.ok = est < WS_LIMIT;
    return L;
}

}  // namespace

CG_API cg_status cg_adjoint_workspace_size(cg_plan plan, int64_t n_steps, int32_t checkpoint_every, size_t *bytes)
{
    if (!plan || !bytes || n_steps < 0 || n_steps > MAX_STEPS || checkpoint_every < 0)
        return fail(CG_EINVAL, "bad argument");
    if (plan->inst.size() != 1) return fail(CG_EUNSUPPORTED, "adjoint runs need a single-instance plan");
    if (gate_scheme(plan->scheme)) return fail(CG_EUNSUPPORTED, "no adjoint of the gate integrators");
    const AdjLayout L = adj_layout(plan, n_steps, checkpoint_every);
    if (!L.ok) return fail(CG_EINVAL, "workspace size overflows");
    *bytes = L.total;
    return CG_OK;
}

namespace {

// Common argument checks of the adjoint calls; fills L.
cg_status adjoint_checks(cg_plan plan, int64_t n_steps, int32_t checkpoint_every, const void *workspace,
                         AdjLayout &L)
{
    if (!plan) return fail(CG_EINVAL, "plan is NULL");
    if (plan->inst.size() != 1) return fail(CG_EUNSUPPORTED, "adjoint runs need a single-instance plan");
    if (gate_scheme(plan->scheme)) return fail(CG_EUNSUPPORTED, "no adjoint of the gate integrators");
    if (!workspace || n_steps < 0 || n_steps > MAX_STEPS || checkpoint_every < 0)
        return fail(CG_EINVAL, "bad argument");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return fail(CG_EINVAL, "workspace must be 256-byte aligned");
    L = adj_layout(plan, n_steps, checkpoint_every);
    if (!L.ok) return fail(CG_EINVAL, "workspace size overflows");
    return CG_OK;
}

// Forward segments j = 1 .. j_end - 1 of the checkpoint sweep: cp[j] is
// c steps after cp[j-1] (cp[0] already holds z0).
cg_status checkpoint_sweep(cg_plan plan, const AdjLayout &L, double *cp, int64_t j_end, char *ws, cudaStream_t s)
{
    RunArgs a;
    for (int64_t j = 1; j < j_end; ++j) {
        base_args(plan, a, cp + (j - 1) * L.S, cp + j * L.S, ws);
        a.parity = (int32_t)((L.c - 1) & 1);
        void *args[] = {&a};
        const cg_status st = launch_stages(plan, plan->kernel, args, a, 0, L.c * plan->ns, plan->nblocks, s);
        if (st != CG_OK) return st;
    }
    return CG_OK;
}

// The adjoint stage kernel of the plan, checked to fit the persistent grid.
cg_status adjoint_kernel(cg_plan plan, const void *&ka)
{
    ka = lookup_adj_kernel(plan->kmodel, plan->stencil, plan->scheme, plan->cx);
    if (!ka) return fail(CG_EUNSUPPORTED, "no adjoint kernel for this problem");
    return check_coresident(plan, ka);
}

// The reverse part of the adjoint: given the checkpoints cp[0 .. nseg-1] of
// z0's trajectory (c steps apart), every segment in reverse is recomputed
// with its stage inputs kept and swept back.  The workspace's header has
// been cleared and dLdD / the partial sums zeroed by the caller.
cg_status adjoint_sweep_back(cg_plan plan, const AdjLayout &L, const double *cp, const double *lamT, double *lam0,
                             double *dLdD, int64_t n_steps, char *ws, cudaStream_t s)
{
    const Inst &I = plan->inst[0];
    const size_t sbytes = (size_t)plan->nv * I.nx * I.ny * sizeof(double);
    const int nd = plan->model == CG_FHN ? 2 : 1;
    double *store = reinterpret_cast<double *>(ws + L.store_off);
    double *kb = reinterpret_cast<double *>(ws + L.kb_off);
    double *part = reinterpret_cast<double *>(ws + L.part_off);
    const int nwarps = plan->nblocks * (plan->threads / 32);
    const void *ka = nullptr;
    cg_status st = adjoint_kernel(plan, ka);
    if (st != CG_OK) return st;
    // lam = lamT, kh = kbar / (dt b_last) = lamT
    double *lam = kb + 2 * L.S, *lacc = kb + 3 * L.S;
    cudaError_t e = cudaMemcpyAsync(lam, lamT, sbytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(kb, lamT, sbytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(lam)");
    // segments in reverse: recompute with every stage kept, then sweep back
    RunArgs a;
    int64_t r = 0;
    for (int64_t j = L.nseg - 1; j >= 0; --j) {
        const int64_t m = std::min<int64_t>(L.c, n_steps - j * L.c);
        // the segment's first state is the first stage input the sweep revisits
        e = cudaMemcpyAsync(store, cp + j * L.S, sbytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(segment start)");
        base_args(plan, a, cp + j * L.S, store + m * plan->ns * L.S, ws);
        a.store = store;
        void *fargs[] = {&a};
        st = launch_stages(plan, plan->kernel, fargs, a, 0, m * plan->ns, plan->nblocks, s);
        if (st != CG_OK) return st;
        base_args(plan, a, cp + j * L.S, nullptr, ws);
        if (plan->d_warp_seg_adj) {
            a.segs = plan->d_segs_adj;
            a.warp_seg = plan->d_warp_seg_adj;
        }
        cgk::AdjArgs b;
        std::memset(&b, 0, sizeof b);
        for (int q = 1; q < plan->ns; ++q) b.chat[q] = plan->cy[q - 1] * plan->cacc[q] / plan->cacc[q - 1];
        b.store = store;
        b.kb0 = kb;
        b.kb1 = kb + L.S;
        b.lam = lam;
        b.lacc = lacc;
        b.partial = part;
        b.want_dd = dLdD != nullptr;
        b.m = m;
        b.r0 = r;
        void *aargs[] = {&a, &b};
        st = launch_stages(plan, ka, aargs, a, 0, m * plan->ns, plan->nblocks, s);
        if (st != CG_OK) return st;
        r += m * plan->ns;
    }
    // outputs
    e = cudaMemcpyAsync(lam0, lam, sbytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(lam0)");
    if (!dLdD) return CG_OK;
    cgk::Inv4 inv;
    for (int f = 0; f < 4; ++f) inv.v[f] = plan->dxx[f] != 0.0 ? 1.0 / plan->dxx[f] : 0.0;
    cgk::k_reduce_partials<<<1, 32, 0, s>>>(part, nwarps, nd, inv, dLdD);
    e = cudaGetLastError();
    return e == cudaSuccess ? CG_OK : cuda_fail(e, "reduce kernel");
}

// Clear the status header and, with dLdD, the partial sums and dLdD.
cg_status adjoint_clear(cg_plan plan, const AdjLayout &L, double *dLdD, char *ws, cudaStream_t s)
{
    const int nd = plan->model == CG_FHN ? 2 : 1;
    const int nwarps = plan->nblocks * (plan->threads / 32);
    cudaError_t e = cudaMemsetAsync(ws, 0, cgk::WS_HEADER, s);
    if (dLdD) {
        if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.part_off, 0, sizeof(double) * (size_t)nwarps * nd, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dLdD, 0, sizeof(double) * nd, s);
    }
    return e == cudaSuccess ? CG_OK : cuda_fail(e, "cudaMemsetAsync");
}

}  // namespace

CG_API cg_status cg_adjoint_run(cg_plan plan, const double *z0, const double *lamT, double *lam0, double *dLdD,
                                int64_t n_steps, int32_t checkpoint_every, void *workspace, void *stream)
{
    cgk::NvtxRange nvtx_range("cg_adjoint_run");
    AdjLayout L;
    cg_status st = adjoint_checks(plan, n_steps, checkpoint_every, workspace, L);
    if (st != CG_OK) return st;
    if (!z0 || !lamT || !lam0) return fail(CG_EINVAL, "bad argument");
    st = check_plan_device(plan);
    if (st != CG_OK) return st;
    const Inst &I = plan->inst[0];
    const size_t sbytes = (size_t)plan->nv * I.nx * I.ny * sizeof(double);
    if (overlaps(lamT, lam0, sbytes)) return fail(CG_EINVAL, "lamT and lam0 partially overlap");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    double *cp = reinterpret_cast<double *>(ws + L.cp_off);
    note_run(plan, ws, s);
    st = adjoint_clear(plan, L, dLdD, ws, s);
    if (st != CG_OK) return st;
    cudaError_t e;
    if (n_steps == 0) {
        e = lam0 != lamT ? cudaMemcpyAsync(lam0, lamT, sbytes, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
        return e == cudaSuccess ? CG_OK : cuda_fail(e, "cudaMemcpyAsync");
    }
    const void *ka = nullptr;
    st = adjoint_kernel(plan, ka);
    if (st != CG_OK) return st;
    // forward sweep keeping a checkpoint every c steps, then the sweep back
    e = cudaMemcpyAsync(cp, z0, sbytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(checkpoint)");
    st = checkpoint_sweep(plan, L, cp, L.nseg, ws, s);
    if (st != CG_OK) return st;
    return adjoint_sweep_back(plan, L, cp, lamT, lam0, dLdD, n_steps, ws, s);
}

CG_API cg_status cg_adjoint_checkpoint_size(cg_plan plan, int64_t n_steps, int32_t checkpoint_every, size_t *bytes)
{
    if (!plan || !bytes || n_steps < 0 || n_steps > MAX_STEPS || checkpoint_every < 0)
        return fail(CG_EINVAL, "bad argument");
    if (plan->inst.size() != 1) return fail(CG_EUNSUPPORTED, "adjoint runs need a single-instance plan");
    if (gate_scheme(plan->scheme)) return fail(CG_EUNSUPPORTED, "no adjoint of the gate integrators");
    const AdjLayout L = adj_layout(plan, n_steps, checkpoint_every);
    if (!L.ok) return fail(CG_EINVAL, "workspace size overflows");
    *bytes = (size_t)L.nseg * L.S * sizeof(double);
    return CG_OK;
}

CG_API cg_status cg_adjoint_forward(cg_plan plan, const double *z0, double *zT, int64_t n_steps,
                                    int32_t checkpoint_every, double *checkpoints, void *workspace, void *stream)
{
    cgk::NvtxRange nvtx_range("cg_adjoint_forward");
    AdjLayout L;
    cg_status st = adjoint_checks(plan, n_steps, checkpoint_every, workspace, L);
    if (st != CG_OK) return st;
    if (!z0 || !zT || !checkpoints) return fail(CG_EINVAL, "bad argument");
    if ((reinterpret_cast<uintptr_t>(checkpoints) & 255) != 0)
        return fail(CG_EINVAL, "the checkpoint buffer must be 256-byte aligned");
    const Inst &I = plan->inst[0];
    const size_t sbytes = (size_t)plan->nv * I.nx * I.ny * sizeof(double);
    const size_t cbytes = (size_t)L.nseg * L.S * sizeof(double);
    auto range_overlap = [](const void *p, size_t n, const void *q, size_t m) {
        const char *x = reinterpret_cast<const char *>(p), *y = reinterpret_cast<const char *>(q);
        return x < y + m && y < x + n;
    };
    if (overlaps(z0, zT, sbytes)) return fail(CG_EINVAL, "z0 and zT partially overlap");
    if (range_overlap(zT, sbytes, checkpoints, cbytes) || range_overlap(z0, sbytes, checkpoints, cbytes))
        return fail(CG_EINVAL, "z0 or zT overlaps the checkpoint buffer");
    st = check_plan_device(plan);
    if (st != CG_OK) return st;
    const void *ka = nullptr;
    st = adjoint_kernel(plan, ka);       // the reverse sweep must be able to run
    if (st != CG_OK) return st;
    {
        std::lock_guard<std::mutex> g(plan->last_mu);
        auto &reg = plan->checkpointed;
        auto it = std::find_if(reg.begin(), reg.end(), [&](const auto &r) { return r.buf == checkpoints; });
        if (it != reg.end()) reg.erase(it);
        if (reg.size() >= 16) reg.erase(reg.begin());
        reg.push_back({checkpoints, n_steps, L.c});
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    note_run(plan, ws, s);
    cudaError_t e = cudaMemsetAsync(ws, 0, cgk::WS_HEADER, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(checkpoints, z0, sbytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(checkpoint)");
    if (n_steps == 0) {
        e = zT != z0 ? cudaMemcpyAsync(zT, z0, sbytes, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
        return e == cudaSuccess ? CG_OK : cuda_fail(e, "cudaMemcpyAsync");
    }
    st = checkpoint_sweep(plan, L, checkpoints, L.nseg, ws, s);
    if (st != CG_OK) return st;
    // the last segment ends at zT
    const int64_t m = n_steps - (L.nseg - 1) * L.c;
    RunArgs a;
    base_args(plan, a, checkpoints + (L.nseg - 1) * L.S, zT, ws);
    a.parity = (int32_t)((m - 1) & 1);
    void *args[] = {&a};
    return launch_stages(plan, plan->kernel, args, a, 0, m * plan->ns, plan->nblocks, s);
}

CG_API cg_status cg_adjoint_reverse(cg_plan plan, const double *checkpoints, const double *lamT, double *lam0,
                                    double *dLdD, int64_t n_steps, int32_t checkpoint_every, void *workspace,
                                    void *stream)
{
    cgk::NvtxRange nvtx_range("cg_adjoint_reverse");
    AdjLayout L;
    cg_status st = adjoint_checks(plan, n_steps, checkpoint_every, workspace, L);
    if (st != CG_OK) return st;
    if (!checkpoints || !lamT || !lam0) return fail(CG_EINVAL, "bad argument");
    const Inst &I = plan->inst[0];
    const size_t sbytes = (size_t)plan->nv * I.nx * I.ny * sizeof(double);
    const size_t cbytes = (size_t)L.nseg * L.S * sizeof(double);
    if (overlaps(lamT, lam0, sbytes)) return fail(CG_EINVAL, "lamT and lam0 partially overlap");
    {
        const char *x = reinterpret_cast<const char *>(lam0), *y = reinterpret_cast<const char *>(checkpoints);
        if (x < y + cbytes && y < x + sbytes) return fail(CG_EINVAL, "lam0 overlaps the checkpoint buffer");
    }
    {
        std::lock_guard<std::mutex> g(plan->last_mu);
        const auto &reg = plan->checkpointed;
        auto it = std::find_if(reg.begin(), reg.end(), [&](const auto &r) { return r.buf == checkpoints; });
        if (it == reg.end() || it->n_steps != n_steps || it->c != L.c)
            return fail(CG_EINVAL, "this buffer holds no checkpoints of this plan over %lld steps, %lld apart",
                        (long long)n_steps, (long long)L.c);
    }
    st = check_plan_device(plan);
    if (st != CG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    note_run(plan, ws, s);
    st = adjoint_clear(plan, L, dLdD, ws, s);
    if (st != CG_OK) return st;
    if (n_steps == 0) {
        const cudaError_t e =
            lam0 != lamT ? cudaMemcpyAsync(lam0, lamT, sbytes, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
        return e == cudaSuccess ? CG_OK : cuda_fail(e, "cudaMemcpyAsync");
    }
    return adjoint_sweep_back(plan, L, checkpoints, lamT, lam0, dLdD, n_steps, ws, s);
}

cg_status cgk::set_last_error(cg_status st, const char *msg)
{
    g_err = msg;
    return st;
}

CG_API const char *cg_last_error(void)
{
    return g_err.c_str();
}

CG_API int32_t cg_n_fields(int32_t model)
{
    return n_fields(model);
}

CG_API int32_t cg_n_params(int32_t model)
{
    return n_params(model);
}

CG_API cg_status cg_default_params(int32_t model, double *out)
{
    if (!out) return fail(CG_EINVAL, "out is NULL");
    if (n_params(model) < 0) return fail(CG_EINVAL, "unknown model %d", model);
    default_params(model, out);
    return CG_OK;
}

namespace {

cg_status schedule_preview(const int32_t *nx, const int32_t *ny, int32_t n_inst, int32_t cells_x, int32_t n_blocks,
                           int32_t warps_per_block, int32_t *segs_out, int64_t segs_cap, int32_t *warp_seg_out,
                           int64_t *n_segs, int32_t *deps_out, bool adjoint)
{
    if (!nx || !ny || n_inst < 1 || (cells_x != 1 && cells_x != 2) || n_blocks < 1 || warps_per_block < 1 ||
        !warp_seg_out || !n_segs)
        return fail(CG_EINVAL, "bad schedule request");
    std::vector<int32_t> nxs(nx, nx + n_inst), nys(ny, ny + n_inst);
    for (int i = 0; i < n_inst; ++i)
        if (nxs[i] < 1 || nys[i] < 1) return fail(CG_EINVAL, "instance %d has an empty grid", i);
    std::vector<cgk::Seg> segs;
    std::vector<int32_t> ws;
    std::vector<int64_t> cb;
    if (adjoint) {
        if (n_inst != 1) return fail(CG_EINVAL, "the adjoint schedule is for one instance");
        cb = cost_balanced_ranges(nxs[0], nys[0], 32 * cells_x, n_blocks, ADJ_BOUNDARY_COST);
    } else {
        cb = static_ranges(nxs, nys, 32 * cells_x, n_blocks);
    }
    static_schedule(nxs, nys, cells_x, n_blocks, warps_per_block, segs, ws, cb, adjoint);
    *n_segs = (int64_t)segs.size();
    std::copy(ws.begin(), ws.end(), warp_seg_out);
    if (deps_out) {
        std::vector<int2> deps;
        halo_dependencies(nxs, nys, n_blocks, cb, deps);
        for (int b = 0; b < n_blocks; ++b) {
            deps_out[2 * b] = deps[b].x;
            deps_out[2 * b + 1] = deps[b].y;
        }
    }
    if (segs_out) {
        if ((int64_t)segs.size() > segs_cap) return fail(CG_EINVAL, "segs_cap too small (%lld needed)",
                                                         (long long)segs.size());
        std::memcpy(segs_out, segs.data(), sizeof(cgk::Seg) * segs.size());
    }
    return CG_OK;
}

}  // namespace

CG_API cg_status cg_static_schedule(const int32_t *nx, const int32_t *ny, int32_t n_inst, int32_t cells_x,
                                    int32_t n_blocks, int32_t warps_per_block, int32_t *segs_out,
                                    int64_t segs_cap, int32_t *warp_seg_out, int64_t *n_segs, int32_t *deps_out)
{
    return schedule_preview(nx, ny, n_inst, cells_x, n_blocks, warps_per_block, segs_out, segs_cap, warp_seg_out,
                            n_segs, deps_out, false);
}

CG_API cg_status cg_adjoint_schedule(int32_t nx, int32_t ny, int32_t cells_x, int32_t n_blocks,
                                     int32_t warps_per_block, int32_t *segs_out, int64_t segs_cap,
                                     int32_t *warp_seg_out, int64_t *n_segs)
{
    return schedule_preview(&nx, &ny, 1, cells_x, n_blocks, warps_per_block, segs_out, segs_cap, warp_seg_out,
                            n_segs, nullptr, true);
}

CG_API int32_t cg_abi_version(void)
{
    return CG_ABI_VERSION;
}

CG_API int32_t cg_bounds_checked(void)
{
    return cgk::BOUNDS_CHECK ? 1 : 0;
}
