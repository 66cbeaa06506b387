// Fused explicit stage kernel for dz/dt = D L z + N[z] (Eq. rdeqn, Sect. 2-3).
//
// One warp owns a tile of 32*CX columns x `rows` rows of one instance.  It
// sweeps the rows from bottom to top keeping a three-row register window of
// every diffusive field; west/east neighbours come from the neighbouring
// lanes by warp shuffles, the two columns just outside the tile are loaded by
// lanes 0 and 31.  Ghost points (Fig. 1) are resolved in the load indices:
// column -1 reads column 1 (MIRROR), 0 (CLAMP) or nx-1 (PERIODIC), column nx
// reads nx-2, nx-1 or 0, and likewise for rows, so no branch touches the
// arithmetic.
//
// Each cell of each stage costs one FMA chain: the model's local terms with
// the stencil's centre weight folded in, then the off-centre stencil sums,
// then the Runge-Kutta combine (two FMAs per field, one in the last stage).
// The FP64 pipe is the binding resource on GB300, so every non-FP64 piece of
// work (index arithmetic, clamps of the smoothed steps, NaN checks) is done
// with integer instructions.
//
// Work assignment: a static schedule computed on the host (equal cells per
// block, equal strip-rows per warp) or an atomic tile queue per stage.
// Launch modes: persistent (one cooperative launch runs all stages of all
// steps, separated by a bounded grid barrier or by bounded waits on the
// blocks that own a block's halo) or one launch per stage (no waiting).
#pragma once

#include "cg_fastmath.cuh"
#include "cg_internal.h"

namespace cgk {

#define CG_FULL 0xffffffffu

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t nonfinite_bit(double v)
{
    return (uint32_t)((((unsigned long long)__double_as_longlong(v)) >> 52 & 0x7ffull) == 0x7ffull);
}

// Order-preserving integer key of a double (x < y iff key(x) < key(y) for
// non-NaN values; -0 sorts just below +0): integer-pipe comparisons.
__device__ __forceinline__ long long order_key(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}

// Clamp to [0, 1] on the integer pipe: non-negative doubles order like their
// bit patterns, and every negative double has the sign bit set.
__device__ __forceinline__ double clamp01_int(double t)
{
    long long b = __double_as_longlong(t);
    b = b < 0 ? 0 : b;
    b = b > 0x3FF0000000000000ll ? 0x3FF0000000000000ll : b;
    return __longlong_as_double(b);
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Bounded grid barrier on a monotonic 64-bit arrival counter that the host
// zeroes before each persistent launch.  Barrier k of a launch is passed
// once the counter reaches (k + 1) x blocks: thread 0 of each block adds 1
// (a release) and polls the counter (acquires) until it gets there.  One
// round trip to the counter per block and no reset or generation word, so
// the last block's arrival is seen directly by every waiting block (1.2 us
// per barrier for 152 blocks on GB300, against 2.0 us for an arrival counter
// with a separate generation word).  On
// expiry of the time limit the block records CG_DEV_TIMEOUT and every thread
// of the block returns false.
static __device__ __noinline__ bool grid_barrier(unsigned long long *count, uint32_t *status, uint64_t timeout_ns,
                                                 unsigned long long target)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        // The release is cumulative: the block's writes, ordered before it by
        // __syncthreads, become visible with it at GPU scope.
        red_release_add_u64(count, 1ull);
        int ok = 1;
        const uint64_t t0 = global_timer_ns();
        const uint64_t max_iter = (timeout_ns >> 4) + (1ull << 20);
        uint64_t it = 0;
        while (ld_acquire_u64(count) < target) {
            if ((++it & 63) == 0 && (global_timer_ns() - t0 > timeout_ns || it > max_iter)) {
                ok = 0;
                atomicOr(status, CG_DEV_TIMEOUT);
                break;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Neighbour synchronisation between stages (static schedule).  A stage of
// block b only reads its own cells and a one-cell halo, which blocks
// deps[b].x .. deps[b].y own; and it only overwrites buffers that those same
// blocks read in the stage before.  So block b publishes how many stages it
// has finished and, before the next one, waits (bounded) until every block
// of its range has finished as many.  No grid-wide barrier: blocks drift by
// at most one stage against their neighbours and stage tails overlap.
static __device__ __noinline__ bool neighbor_sync(unsigned *flags, const int2 *deps, uint32_t *status,
                                                  uint64_t timeout_ns, unsigned done, unsigned extra)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release_u32(flags + blockIdx.x, done);
        const int2 d = deps[blockIdx.x];
        const unsigned need = done + extra;
        int ok = 1;
        const uint64_t t0 = global_timer_ns();
        const uint64_t max_iter = (timeout_ns >> 5) + (1ull << 20);
        uint64_t it = 0;
        for (int q = d.x; q <= d.y && ok; ++q) {
            while (ld_acquire_u32(flags + q) < need) {
                __nanosleep(32);
                if ((++it & 63) == 0 && (global_timer_ns() - t0 > timeout_ns || it > max_iter)) {
                    ok = 0;
                    atomicOr(status, CG_DEV_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Synchronise after global stage g of a persistent launch (g_begin <= g).
__device__ __forceinline__ bool stage_sync(const RunArgs &a, int64_t g, bool first)
{
    const unsigned extra = (first && a.stuck_barrier) ? 1u : 0u;
    if (a.sync_mode == SYNC_NEIGHBOR)
        return neighbor_sync(a.flags, a.deps, a.status, a.timeout_ns, (unsigned)(g - a.g_begin + 1), extra);
    const unsigned long long target = (unsigned long long)(g - a.g_begin + 1) * a.nblocks_expect + extra;
    return grid_barrier(reinterpret_cast<unsigned long long *>(a.sync), a.status, a.timeout_ns, target);
}

// ----------------------------------------------------------- checked build
// Compiled with -DCG_BOUNDS_CHECK (libcardiac_gb300_checked.so), every stage
// worker checks the indices it is about to use before the first access of a
// segment (each lane's columns and halo column, the vector-access
// conditions, the buffer pointers) and before each new row; a failed check
// skips the rest of the segment and sets CG_DEV_BOUNDS in the status word.
// Only integer compares are added, so results equal the plain build's bit
// for bit.  It stands in for a memory checker, which is not available here.
#ifdef CG_BOUNDS_CHECK
constexpr bool BOUNDS_CHECK = true;
#else
constexpr bool BOUNDS_CHECK = false;
#endif

// Warp-uniform: some lane's column or halo column lies outside [0, nx), or a
// 16-byte access would not cover two adjacent cells starting at an even one.
template <int CX>
__device__ __forceinline__ bool cols_out_of_grid(const int (&cx)[CX], int hx, bool want_halo, int x0, int nx,
                                                 bool vec_row)
{
    bool b = x0 < 0;
#pragma unroll
    for (int c = 0; c < CX; ++c) b |= (cx[c] < 0) || (cx[c] >= nx);
    b |= want_halo && ((hx < 0) || (hx >= nx));
    if (CX == 2 && vec_row) b |= ((cx[0] & 1) != 0) || (cx[CX - 1] != cx[0] + 1) || (x0 + CX > nx);
    return __any_sync(CG_FULL, b);
}

__device__ __forceinline__ bool row_out_of_grid(int y, int ny) { return y < 0 || y >= ny; }

__device__ __forceinline__ bool bad_ptr(const void *p)
{
    return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 7) != 0;
}

// ------------------------------------------------------------------ models

template <int M> struct Model;

// FitzHugh-Nagumo, Eq. (fhn): both fields diffusive.
//   F_u = (1 + wc_u) u - v - u^3 + stencil_u
//   F_v = eps u + (wc_v - eps a1) v - eps a0 + stencil_v
template <> struct Model<MODEL_FHN> {
    static constexpr int NV = 2, ND = 2;
    // Jacobian entries stored per cell: J0 = d t_u / d u = (1 + wc_u) - 3 u^2
    // (the other entries, -1, eps and wc_v - eps a1, are constants).
    static constexpr int NJ = 1;
    struct Coef { double A_u, B_v; };
    __device__ static Coef coef(const Inst &I) { return Coef{I.mi[0], I.mi[1]}; }
    // mp[0] = eps, mp[1] = -eps a0 ; Coef holds instance-dependent folds.
    __device__ static void local(const Coef &c, const double *mp, const double (&z)[NV], double (&t)[NV])
    {
        const double u = z[0], v = z[1];
        const double p = u * u;
        t[0] = fma(-p, u, fma(c.A_u, u, -v));
        t[1] = fma(mp[0], u, fma(c.B_v, v, mp[1]));
    }
    __device__ static void local_jac(const Coef &c, const double *mp, const double (&z)[NV], double (&t)[NV],
                                     double (&J)[NJ])
    {
        const double u = z[0], v = z[1];
        const double p = u * u;
        t[0] = fma(-p, u, fma(c.A_u, u, -v));
        t[1] = fma(mp[0], u, fma(c.B_v, v, mp[1]));
        J[0] = fma(-3.0, p, c.A_u);
    }
    // tangent: J d with the centre weights folded in
    __device__ static void tan_local(const Coef &c, const double *mp, const double (&J)[NJ],
                                     const double (&d)[NV], double (&t)[NV])
    {
        t[0] = fma(J[0], d[0], -d[1]);
        t[1] = fma(mp[0], d[0], c.B_v * d[1]);
    }
    // adjoint: J^T k with the centre weights folded in
    __device__ static void adj_local(const Coef &c, const double *mp, const double (&J)[NJ],
                                     const double (&k)[NV], double (&t)[NV])
    {
        t[0] = fma(J[0], k[0], mp[0] * k[1]);
        t[1] = fma(c.B_v, k[1], -k[0]);
    }
};

// Pure diffusion (N = 0), one field: F = wc u + stencil.
template <> struct Model<MODEL_DIFF> {
    static constexpr int NV = 1, ND = 1, NJ = 0;
    struct Coef { double wc; };
    __device__ static Coef coef(const Inst &I) { return Coef{I.mi[0]}; }
    __device__ static void local(const Coef &c, const double *, const double (&z)[NV], double (&t)[NV])
    {
        t[0] = c.wc * z[0];
    }
    __device__ static void local_jac(const Coef &c, const double *, const double (&z)[NV], double (&t)[NV],
                                     double (&)[1])
    {
        t[0] = c.wc * z[0];
    }
    __device__ static void tan_local(const Coef &c, const double *, const double (&)[1], const double (&d)[NV],
                                     double (&t)[NV])
    {
        t[0] = c.wc * d[0];
    }
    __device__ static void adj_local(const Coef &c, const double *, const double (&)[1], const double (&k)[NV],
                                     double (&t)[NV])
    {
        t[0] = c.wc * k[0];
    }
};

// Two-variable Karma model, Eq. (karma); only u diffuses (gamma = D_u).
// With sig = (1 - tanh(u - u_h))/2 = sigmoid(2 (u_h - u)) and g = u* - v^M:
//   t_u = wc_u u + (u^2 sig g - u)/tau_u     (u^2/2 (1 - tanh) = u^2 sig)
//   t_v = (a H_k(u - u_v) - v)/tau_v         (H_k(u_v - u) = 1 - H_k(u - u_v)
//                                             for the cubic step), a = 1/(1 - e^-Re)
// Under the tanh variant of Sect. 6 (tanh x -> 2 H_{1/3}(x) - 1), sig is
// H_{1/3}(u_h - u).  An integer M takes v^M by repeated squaring (the
// integer power Sect. 6 recommends), any other M by pow().
// Constant layout of mp (filled by the host):
enum {
    KP_ITU,     // 1/tau_u
    KP_ITV,     // 1/tau_v
    KP_USTAR,   // u*
    KP_SA,      // 2 u_h: sig = sigmoid(2 u_h - 2 u)
    KP_HA,      // 1/2 + u_h/3: variant sig = H(t), t = 1/2 + (u_h - u)/3
    KP_AITV,    // a/tau_v
    KP_K,       // k of H_k
    KP_CV,      // 1/2 - k u_v
    KP_6KA,     // 6 k a/tau_v: d t_v/du = KP_6KA t (1 - t)
    KP_M,       // M
    KP_MI,      // bits of an int64: M if it is an integer in [0, 64], else -1
    KP_TH,      // 1.0: tanh variant (tested by its bits, on the integer pipe)
    KP_N
};

// v^m for an integer m >= 1 by repeated squaring (M = 6: v^2, v^4, v^2 v^4).
__device__ __forceinline__ double int_pow(double v, int m)
{
    while (!(m & 1)) {
        v *= v;
        m >>= 1;
    }
    double r = v;
    m >>= 1;
    while (m) {
        v *= v;
        if (m & 1) r *= v;
        m >>= 1;
    }
    return r;
}

template <> struct Model<MODEL_KARMA> {
    static constexpr int NV = 2, ND = 1;
    // Stored Jacobian entries: [d t_u/du (wc_u folded in), d t_u/dv,
    // d t_v/du]; d t_v/dv = -1/tau_v is a constant.
    static constexpr int NJ = 3;
    struct Coef { double A_u; const double *tab; };    // A_u = wc_u - 1/tau_u
    __device__ static Coef coef(const Inst &I) { return Coef{I.mi[0], I.tab}; }

    // v^M and, when JAC, M v^(M-1) (M = 0: 1 and 0).  v^M is computed the
    // same way with and without JAC, so both give the same values.
    template <bool JAC>
    __device__ __forceinline__ static double vpow(const double *mp, double v, double &dvm)
    {
        const int mi = (int)__double_as_longlong(mp[KP_MI]);
        if (mi >= 1) {
            if constexpr (JAC) dvm = (mi >= 2) ? mp[KP_M] * int_pow(v, mi - 1) : 1.0;
            return int_pow(v, mi);
        }
        if (mi == 0) {
            if constexpr (JAC) dvm = 0.0;
            return 1.0;
        }
        if constexpr (JAC) dvm = mp[KP_M] * pow(v, mp[KP_M] - 1.0);
        return pow(v, mp[KP_M]);
    }

    template <bool JAC>
    __device__ __forceinline__ static void eval(const Coef &c, const double *mp, const double (&z)[NV],
                                                double (&t)[NV], double *J)
    {
        const double u = z[0], v = z[1];
        double sig, dsig = 0.0;
        if (__double_as_longlong(mp[KP_TH]) != 0) {
            const double th = clamp01_int(fma(-1.0 / 3.0, u, mp[KP_HA]));
            sig = (th * th) * fma(-2.0, th, 3.0);
            if constexpr (JAC) dsig = -2.0 * (th * (1.0 - th));
        } else if constexpr (JAC) {
            double ds;
            sig = sigmoid(fma(-2.0, u, mp[KP_SA]), c.tab, ds);
            dsig = -2.0 * ds;
        } else {
            sig = sigmoid(fma(-2.0, u, mp[KP_SA]), c.tab);
        }
        double dvm = 0.0;
        const double g = mp[KP_USTAR] - vpow<JAC>(mp, v, dvm);
        const double uu = u * u;
        const double q = uu * sig;
        t[0] = fma(q * g, mp[KP_ITU], c.A_u * u);
        const double tv = clamp01_int(fma(mp[KP_K], u, mp[KP_CV]));
        const double H = (tv * tv) * fma(-2.0, tv, 3.0);
        t[1] = fma(mp[KP_AITV], H, -(v * mp[KP_ITV]));
        if constexpr (JAC) {
            // d/du (u^2 sig g)/tau_u = (2 u sig + u^2 dsig) g / tau_u
            J[0] = fma(fma(2.0 * u, sig, uu * dsig) * g, mp[KP_ITU], c.A_u);
            J[1] = -(q * dvm) * mp[KP_ITU];
            J[2] = mp[KP_6KA] * (tv * (1.0 - tv));
        }
    }
    __device__ static void local(const Coef &c, const double *mp, const double (&z)[NV], double (&t)[NV])
    {
        eval<false>(c, mp, z, t, nullptr);
    }
    __device__ static void local_jac(const Coef &c, const double *mp, const double (&z)[NV], double (&t)[NV],
                                     double (&J)[NJ])
    {
        eval<true>(c, mp, z, t, J);
    }
    __device__ static void tan_local(const Coef &, const double *mp, const double (&J)[NJ], const double (&d)[NV],
                                     double (&t)[NV])
    {
        t[0] = fma(J[0], d[0], J[1] * d[1]);
        t[1] = fma(J[2], d[0], -(mp[KP_ITV] * d[1]));
    }
    __device__ static void adj_local(const Coef &, const double *mp, const double (&J)[NJ], const double (&k)[NV],
                                     double (&t)[NV])
    {
        t[0] = fma(J[0], k[0], J[2] * k[1]);
        t[1] = fma(J[1], k[0], -(mp[KP_ITV] * k[1]));
    }
};

// Bueno-Orovio-Cherry-Fenton, Eq. (bochfe) with the currents J_fi, J_so,
// J_si, the alpha/beta gate form and the u-dependent time constants of the
// cited minimal model; every step is the cubic H_k.  Only u diffuses.
// Constant layout of mp (filled by the host):
enum {
    BP_UO, BP_UU, BP_THV, BP_THW, BP_THVM, BP_THO,
    BP_TV1M, BP_TV2M, BP_TVP, BP_TW1M, BP_TW2M, BP_KWM, BP_UWM, BP_TWP,
    BP_TFI, BP_TO1, BP_TO2, BP_TSO1, BP_TSO2, BP_KSO, BP_USO,
    BP_TS1, BP_TS2, BP_KS, BP_US, BP_TSI, BP_TWINF, BP_WINFSTAR, BP_K,
    BP_NRAW,
    // derived on the host
    BD_CV = BP_NRAW,   // 1/2 - k thv
    BD_CW,             // 1/2 - k thw
    BD_CVM,            // 1/2 - k thvm
    BD_CO,             // 1/2 - k tho
    BD_DTV,            // tv2m - tv1m
    BD_DTO,            // to2 - to1
    BD_DTS,            // ts2 - ts1
    BD_IFI,            // 1/tfi
    BD_ISI,            // 1/tsi
    BD_IVP,            // 1/tvp
    BD_IWP,            // 1/twp
    BD_IWINF,          // 1/twinf
    BD_AW2,            // -2 kwm uwm
    BD_KW2,            // 2 kwm
    BD_ASO2,           // -2 kso uso
    BD_KSO2,           // 2 kso
    BD_AS2,            // -2 ks us
    BD_KS2,            // 2 ks
    BD_DTW,            // tw2m - tw1m
    BD_DTSO,           // tso2 - tso1
    BD_6K,             // 6 k
    BD_KWH,            // kwm / 3        (tanh variant: H_{k/3} in place of (1 + tanh)/2)
    BD_AWH,            // 1/2 - kwm uwm / 3
    BD_KSOH,           // kso / 3
    BD_ASOH,           // 1/2 - kso uso / 3
    BD_KSH,            // ks / 3
    BD_ASH,            // 1/2 - ks us / 3
    BD_RS0,            // 1/ts1 by fast_rcp on the device (the s-gate rate where H_w = 0)
    BD_RS1,            // 1/(ts1 + (ts2 - ts1)) likewise (H_w = 1)
    BD_KREST,          // order key (bits) of the largest u with H_v = H_w = 0 (host, exact)
    BD_KEXC,           // order key (bits) of the smallest u with all four switches at 1
    BD_FLAGS,          // bit pattern: BF_SAME_VMO (set at plan time)
    BD_N
};
// Plan-time fact of the four-field constants that saves FP64 work, exactly:
// the v^- and o switches share their threshold (both 0.006 in the
// epicardial set), so H_k is evaluated once for both (4 FP64 instructions
// fewer per cell and stage on the resting and general paths).
enum : long long { BF_SAME_VMO = 1 };

// TH selects the model variant of Sect. 6 in which each (1 + tanh(kk x))/2
// becomes the smoothed step H_{kk/3}(x) (same value and slope at x = 0).
template <bool TH> struct BocfModel {
    static constexpr int NV = 4, ND = 1;
    // Stored Jacobian entries (wc_u folded into J_uu):
    // [J_uu, J_uv, J_uw, J_us, J_vu, J_vv, J_wu, J_ww, J_su, J_ss]
    static constexpr int NJ = 10;
    struct Coef { double wc_u; const double *tab; };
    __device__ static Coef coef(const Inst &I) { return Coef{I.mi[0], I.tab}; }

    // (1 + tanh(kk (u - cc)))/2: the sigmoid of 2 kk (u - cc) (constants
    // ik = 2 kk, ia = -2 kk cc), or H_{kk/3}(u - cc) in the variant
    // (ihk = kk/3, iha = 1/2 - kk cc/3).  ds times 2 kk is the u-derivative.
    template <int IA, int IK, int IHA, int IHK>
    __device__ __forceinline__ static double half_tanh(const double *mp, double u, const double *tab, double &ds)
    {
        if constexpr (TH) {
            const double t = clamp01_int(fma(mp[IHK], u, mp[IHA]));
            ds = t * (1.0 - t);
            return (t * t) * fma(-2.0, t, 3.0);
        } else {
            return sigmoid(fma(mp[IK], u, mp[IA]), tab, ds);
        }
    }
    template <int IA, int IK, int IHA, int IHK>
    __device__ __forceinline__ static double half_tanh(const double *mp, double u, const double *tab)
    {
        if constexpr (TH) {
            const double t = clamp01_int(fma(mp[IHK], u, mp[IHA]));
            return (t * t) * fma(-2.0, t, 3.0);
        } else {
            return sigmoid(fma(mp[IK], u, mp[IA]), tab);
        }
    }
    // 1 / (tau1 + dtau (1 + tanh(kk (u - cc)))/2), the rates of the
    // u-dependent time constants tau_w^- and tau_so (tau2 = tau1 + dtau).
    // In the sigmoid form s = 1/(1 + e) (a >= 0) or e/(1 + e) (a < 0),
    // e = e^-|a|, so (tau1 + dtau s)(1 + e) is tau2 + tau1 e or
    // tau1 + tau2 e: one FMA with its operands chosen by the sign of a (on
    // the integer pipe), and one reciprocal, 1/(tau1 + dtau s) =
    // (1 + e)/fma(.).  With DS, ds = s (1 - s) as in half_tanh.
    template <int IA, int IK, int IHA, int IHK, bool DS>
    __device__ __forceinline__ static double rcp_tau(const double *mp, double u, const double *tab, double tau1,
                                                     double dtau, double tau2, double &ds)
    {
        if constexpr (TH) {
            const double t = clamp01_int(fma(mp[IHK], u, mp[IHA]));
            if constexpr (DS) ds = t * (1.0 - t);
            return fast_rcp(fma(dtau, (t * t) * fma(-2.0, t, 3.0), tau1));
        } else {
            const double a = fma(mp[IK], u, mp[IA]);
            const double e = exp_neg(a, tab);
            const double ope = 1.0 + e;
            const bool pos = __double_as_longlong(a) >= 0;
            const double ca = pos ? tau1 : tau2, cb = pos ? tau2 : tau1;
            if constexpr (DS) {
                const double r1 = fast_rcp(ope);
                ds = (e * r1) * r1;
            }
            return ope * fast_rcp(fma(ca, e, cb));
        }
    }
#define CG_SW BD_AW2, BD_KW2, BD_AWH, BD_KWH
#define CG_SSO BD_ASO2, BD_KSO2, BD_ASOH, BD_KSOH
#define CG_SS BD_AS2, BD_KS2, BD_ASH, BD_KSH

    // Shared body: right-hand side t and, when JAC, the Jacobian entries.
    // The three (1 + tanh(k (u - c)))/2 terms are sigmoids of 2 k (u - c)
    // (cg_fastmath.cuh); time constants enter through fast reciprocals.
    template <bool JAC>
    __device__ __forceinline__ static void eval(const Coef &c, const double *mp, const double (&z)[NV],
                                                double (&t)[NV], double *J)
    {
        const double u = z[0], v = z[1], w = z[2], s = z[3];
        const double k = mp[BP_K];
        if constexpr (!JAC) {
            // Warp-uniform shortcuts where the v and w switches are saturated
            // for every lane.  Terms multiplied by an exact 0 are dropped and
            // terms multiplied by an exact 1 kept, so the values equal the
            // general path's.  The switch t_x = clamp(k u + c_x) is 0 exactly
            // when u is at most the largest double with fma(k, u, c_x) <= 0,
            // and 1 from the smallest with fma(k, u, c_x) >= 1 on (fma is
            // monotone in u); the plan holds those bounds, so the decision
            // takes one integer compare and no switch is evaluated first.
            const long long ku = order_key(u);
            if (__all_sync(CG_FULL, ku <= __double_as_longlong(mp[BD_KREST]))) {
                // resting tissue: H_v = H_w = 0 (only the u-dependent steady
                // states and time constants near u = 0 remain)
                const long long fl = __double_as_longlong(mp[BD_FLAGS]);
                const double tvm = clamp01_int(fma(k, u, mp[BD_CVM]));
                const double Hvm = (tvm * tvm) * fma(-2.0, tvm, 3.0);
                double Ho = Hvm;
                if (!(fl & BF_SAME_VMO)) {
                    const double to = clamp01_int(fma(k, u, mp[BD_CO]));
                    Ho = (to * to) * fma(-2.0, to, 3.0);
                }
                const double r_vm = fast_rcp(fma(Hvm, mp[BD_DTV], mp[BP_TV1M]));
                const double v_inf = 1.0 - Hvm;
                double unused;
                const double r_wm = rcp_tau<CG_SW, false>(mp, u, c.tab, mp[BP_TW1M], mp[BD_DTW], mp[BP_TW2M], unused);
                const double q = fma(-u, mp[BD_IWINF], 1.0);
                const double w_inf = fma(Ho, mp[BP_WINFSTAR] - q, q);
                const double r_o = fast_rcp(fma(Ho, mp[BD_DTO], mp[BP_TO1]));
                const double r_s = mp[BD_RS0];
                const double s_inf = half_tanh<CG_SS>(mp, u, c.tab);
                const double uo = u - mp[BP_UO];
                t[0] = fma(c.wc_u, u, -(uo * r_o));
                t[1] = (v_inf - v) * r_vm;
                t[2] = (w_inf - w) * r_wm;
                t[3] = (s_inf - s) * r_s;
                return;
            }
            if (__all_sync(CG_FULL, ku >= __double_as_longlong(mp[BD_KEXC]))) {
                // excited tissue: every switch is 1
                double unused;
                const double r_so = rcp_tau<CG_SSO, false>(mp, u, c.tab, mp[BP_TSO1], mp[BD_DTSO], mp[BP_TSO2], unused);
                const double r_s = mp[BD_RS1];
                const double s_inf = half_tanh<CG_SS>(mp, u, c.tab);
                const double ua = u - mp[BP_THV], ub = mp[BP_UU] - u;
                const double J_fi = -v * (ua * ub) * mp[BD_IFI];
                const double J_si = -w * (s * mp[BD_ISI]);
                t[0] = fma(c.wc_u, u, -((J_fi + r_so) + J_si));
                t[1] = -v * mp[BD_IVP];
                t[2] = -w * mp[BD_IWP];
                t[3] = (s_inf - s) * r_s;
                return;
            }
        }
        const long long fl = __double_as_longlong(mp[BD_FLAGS]);
        const double tv = clamp01_int(fma(k, u, mp[BD_CV]));
        const double tw = clamp01_int(fma(k, u, mp[BD_CW]));
        const double tvm = clamp01_int(fma(k, u, mp[BD_CVM]));
        const double Hv = (tv * tv) * fma(-2.0, tv, 3.0);
        const double Hw = (tw * tw) * fma(-2.0, tw, 3.0);
        const double Hvm = (tvm * tvm) * fma(-2.0, tvm, 3.0);
        double to = tvm, Ho = Hvm;
        if (!(fl & BF_SAME_VMO)) {
            to = clamp01_int(fma(k, u, mp[BD_CO]));
            Ho = (to * to) * fma(-2.0, to, 3.0);
        }
        const double tau_vm = fma(Hvm, mp[BD_DTV], mp[BP_TV1M]);
        const double r_vm = fast_rcp(tau_vm);
        const double v_inf = 1.0 - Hvm;
        double dsw = 0.0, dsso = 0.0, dss;
        const double r_wm = rcp_tau<CG_SW, JAC>(mp, u, c.tab, mp[BP_TW1M], mp[BD_DTW], mp[BP_TW2M], dsw);
        const double q = fma(-u, mp[BD_IWINF], 1.0);
        const double w_inf = fma(Ho, mp[BP_WINFSTAR] - q, q);
        const double r_o = fast_rcp(fma(Ho, mp[BD_DTO], mp[BP_TO1]));
        const double r_so = rcp_tau<CG_SSO, JAC>(mp, u, c.tab, mp[BP_TSO1], mp[BD_DTSO], mp[BP_TSO2], dsso);
        const double r_s = fast_rcp(fma(Hw, mp[BD_DTS], mp[BP_TS1]));
        const double s_inf = half_tanh<CG_SS>(mp, u, c.tab, dss);
        const double ua = u - mp[BP_THV], ub = mp[BP_UU] - u, uo = u - mp[BP_UO];
        const double omHv = 1.0 - Hv, omHw = 1.0 - Hw;
        const double vinf_v = v_inf - v, winf_w = w_inf - w, sinf_s = s_inf - s;
        const double J_fi = -(v * Hv) * (ua * ub) * mp[BD_IFI];
        const double J_so = fma(uo * omHw, r_o, Hw * r_so);
        const double J_si = -(Hw * w) * (s * mp[BD_ISI]);
        t[0] = fma(c.wc_u, u, -(J_fi + J_so + J_si));
        t[1] = fma(omHv * vinf_v, r_vm, -(Hv * v) * mp[BD_IVP]);
        t[2] = fma(omHw * winf_w, r_wm, -(Hw * w) * mp[BD_IWP]);
        t[3] = sinf_s * r_s;
        if constexpr (JAC) {
            const double k6 = mp[BD_6K];
            const double dHv = k6 * (tv * (1.0 - tv));
            const double dHw = k6 * (tw * (1.0 - tw));
            const double dHvm = k6 * (tvm * (1.0 - tvm));
            const double dHo = (fl & BF_SAME_VMO) ? dHvm : k6 * (to * (1.0 - to));
            const double dtau_vm = dHvm * mp[BD_DTV];
            const double dtau_wm = mp[BD_DTW] * mp[BD_KW2] * dsw;
            const double dtau_o = dHo * mp[BD_DTO];
            const double dtau_so = mp[BD_DTSO] * mp[BD_KSO2] * dsso;
            const double dtau_s = dHw * mp[BD_DTS];
            const double dw_inf = fma(dHo, mp[BP_WINFSTAR] - q, -(1.0 - Ho) * mp[BD_IWINF]);
            const double ds_inf = mp[BD_KS2] * dss;
            const double dJfi_du = -(v * mp[BD_IFI]) * fma(dHv, ua * ub, Hv * (ub - ua));
            const double dJfi_dv = -Hv * (ua * ub) * mp[BD_IFI];
            const double dJso_du = omHw * r_o - uo * dHw * r_o - uo * omHw * dtau_o * (r_o * r_o)
                                   + dHw * r_so - Hw * dtau_so * (r_so * r_so);
            const double dJsi_du = -dHw * (w * s) * mp[BD_ISI];
            J[0] = c.wc_u - (dJfi_du + dJso_du + dJsi_du);
            J[1] = -dJfi_dv;
            J[2] = Hw * s * mp[BD_ISI];
            J[3] = Hw * w * mp[BD_ISI];
            J[4] = -dHv * vinf_v * r_vm + omHv * (-dHvm * r_vm - vinf_v * dtau_vm * (r_vm * r_vm))
                   - dHv * v * mp[BD_IVP];
            J[5] = -omHv * r_vm - Hv * mp[BD_IVP];
            J[6] = -dHw * winf_w * r_wm + omHw * (dw_inf * r_wm - winf_w * dtau_wm * (r_wm * r_wm))
                   - dHw * w * mp[BD_IWP];
            J[7] = -omHw * r_wm - Hw * mp[BD_IWP];
            J[8] = ds_inf * r_s - sinf_s * dtau_s * (r_s * r_s);
            J[9] = -r_s;
        }
    }
    __device__ static void local(const Coef &c, const double *mp, const double (&z)[NV], double (&t)[NV])
    {
        eval<false>(c, mp, z, t, nullptr);
    }
    __device__ static void local_jac(const Coef &c, const double *mp, const double (&z)[NV], double (&t)[NV],
                                     double (&J)[NJ])
    {
        eval<true>(c, mp, z, t, J);
    }
    __device__ static void tan_local(const Coef &, const double *, const double (&J)[NJ], const double (&d)[NV],
                                     double (&t)[NV])
    {
        t[0] = fma(J[0], d[0], fma(J[1], d[1], fma(J[2], d[2], J[3] * d[3])));
        t[1] = fma(J[4], d[0], J[5] * d[1]);
        t[2] = fma(J[6], d[0], J[7] * d[2]);
        t[3] = fma(J[8], d[0], J[9] * d[3]);
    }
    __device__ static void adj_local(const Coef &, const double *, const double (&J)[NJ], const double (&k)[NV],
                                     double (&t)[NV])
    {
        t[0] = fma(J[0], k[0], fma(J[4], k[1], fma(J[6], k[2], J[8] * k[3])));
        t[1] = fma(J[1], k[0], J[5] * k[1]);
        t[2] = fma(J[2], k[0], J[7] * k[2]);
        t[3] = fma(J[3], k[0], J[9] * k[3]);
    }

    // For the gate integrators (Rush-Larsen, implicit Euler): t[0] as in
    // eval and the coefficients of dx/dt = al x + be for x = v, w, s.
    __device__ static void local_gates(const Coef &c, const double *mp, const double (&z)[NV], double (&t)[NV],
                                       double (&al)[3], double (&be)[3])
    {
        const double u = z[0], v = z[1], w = z[2], s = z[3];
        const double k = mp[BP_K];
        const double tv = clamp01_int(fma(k, u, mp[BD_CV]));
        const double tw = clamp01_int(fma(k, u, mp[BD_CW]));
        const double tvm = clamp01_int(fma(k, u, mp[BD_CVM]));
        const double to = clamp01_int(fma(k, u, mp[BD_CO]));
        const double Hv = (tv * tv) * fma(-2.0, tv, 3.0);
        const double Hw = (tw * tw) * fma(-2.0, tw, 3.0);
        const double Hvm = (tvm * tvm) * fma(-2.0, tvm, 3.0);
        const double Ho = (to * to) * fma(-2.0, to, 3.0);
        const double r_vm = fast_rcp(fma(Hvm, mp[BD_DTV], mp[BP_TV1M]));
        const double v_inf = 1.0 - Hvm;
        double unused;
        const double r_wm = rcp_tau<CG_SW, false>(mp, u, c.tab, mp[BP_TW1M], mp[BD_DTW], mp[BP_TW2M], unused);
        const double q = fma(-u, mp[BD_IWINF], 1.0);
        const double w_inf = fma(Ho, mp[BP_WINFSTAR] - q, q);
        const double r_o = fast_rcp(fma(Ho, mp[BD_DTO], mp[BP_TO1]));
        const double r_so = rcp_tau<CG_SSO, false>(mp, u, c.tab, mp[BP_TSO1], mp[BD_DTSO], mp[BP_TSO2], unused);
        const double r_s = fast_rcp(fma(Hw, mp[BD_DTS], mp[BP_TS1]));
        const double s_inf = half_tanh<CG_SS>(mp, u, c.tab);
        const double ua = u - mp[BP_THV], ub = mp[BP_UU] - u, uo = u - mp[BP_UO];
        const double omHv = 1.0 - Hv, omHw = 1.0 - Hw;
        const double J_fi = -(v * Hv) * (ua * ub) * mp[BD_IFI];
        const double J_so = fma(uo * omHw, r_o, Hw * r_so);
        const double J_si = -(Hw * w) * (s * mp[BD_ISI]);
        t[0] = fma(c.wc_u, u, -(J_fi + J_so + J_si));
        t[1] = t[2] = t[3] = 0.0;
        const double rv = omHv * r_vm, rw = omHw * r_wm;
        al[0] = -fma(Hv, mp[BD_IVP], rv);
        be[0] = rv * v_inf;
        al[1] = -fma(Hw, mp[BD_IWP], rw);
        be[1] = rw * w_inf;
        al[2] = -r_s;
        be[2] = s_inf * r_s;
    }
};
#undef CG_SW
#undef CG_SSO
#undef CG_SS

template <> struct Model<MODEL_BOCF> : BocfModel<false> {};
template <> struct Model<MODEL_BOCFH> : BocfModel<true> {};

// ------------------------------------------------------------- index maps

// Column/row index with ghost resolution: i == -1 and i == n are the ghost
// points of Fig. 1 (MIRROR: 1 and n-2, CLAMP: 0 and n-1, PERIODIC: the
// opposite edge, n-1 and 0); i > n is outside every stored cell's stencil
// and is clamped only to stay in bounds.
__device__ __forceinline__ int map_idx(int i, int n, int bc)
{
    if (i < 0) return bc == CG_BC_MIRROR ? 1 : (bc == CG_BC_PERIODIC ? n - 1 : 0);
    if (i == n) return bc == CG_BC_MIRROR ? n - 2 : (bc == CG_BC_PERIODIC ? 0 : n - 1);
    return i < n ? i : n - 1;
}

// ------------------------------------------------------- stencil helpers

// F[c] += wd (V(x-1) + V(x+1)) + wy V(x) + wx (W + E) for the CX cells of a
// lane, V = N + S (the vertical pair sum), from a three-row window (lo, mid,
// hi) and the halo column held by lanes 0 (west) and 31 (east).  V(x) is
// formed once per column and shared with the neighbouring columns, so the
// 9-point stencil costs three additions and three FMAs per cell.
template <int ST, int CX>
__device__ __forceinline__ void add_offcentre(int lane, const double (&lo)[CX], const double (&mid)[CX],
                                              const double (&hi)[CX], double hlo, double hmid, double hhi,
                                              double wx, double wy, double wd, double (&F)[CX])
{
    double up = __shfl_up_sync(CG_FULL, mid[CX - 1], 1);
    double dn = __shfl_down_sync(CG_FULL, mid[0], 1);
    if (lane == 0) up = hmid;
    if (lane == 31) dn = hmid;
    double V[CX];
#pragma unroll
    for (int c = 0; c < CX; ++c) V[c] = lo[c] + hi[c];
    double Vl = 0.0, Vr = 0.0;
    if (ST == CG_STENCIL9) {
        const double Vh = hlo + hhi;
        Vl = __shfl_up_sync(CG_FULL, V[CX - 1], 1);
        Vr = __shfl_down_sync(CG_FULL, V[0], 1);
        if (lane == 0) Vl = Vh;
        if (lane == 31) Vr = Vh;
    }
#pragma unroll
    for (int c = 0; c < CX; ++c) {
        const double W = (c == 0) ? up : mid[c - 1];
        const double E = (c == CX - 1) ? dn : mid[c + 1];
        double acc_f = F[c];
        if (ST == CG_STENCIL9) {
            const double VW = (c == 0) ? Vl : V[c - 1];
            const double VE = (c == CX - 1) ? Vr : V[c + 1];
            acc_f = fma(wd, VW + VE, acc_f);
        }
        acc_f = fma(wy, V[c], acc_f);
        acc_f = fma(wx, W + E, acc_f);
        F[c] = acc_f;
    }
}

// Row sums for the 9-point stencil in row-sum form: for one row of CX cells
// per lane, R = W + E (the horizontal pair) and T = R + ct C with
// ct = wy / wd.  Then wd (T(y-1) + T(y+1)) + wx R(y) is the off-centre part
// wd (NW + NE + SW + SE) + wy (N + S) + wx (W + E) at row y, and R and T of a
// row are formed once and used by the rows above and below: five FP64
// instructions per cell and field instead of six, and two shuffles per row.
template <int CX>
__device__ __forceinline__ void row_sums(int lane, const double (&v)[CX], double h, double ct, double (&R)[CX],
                                         double (&T)[CX])
{
    double up = __shfl_up_sync(CG_FULL, v[CX - 1], 1);
    double dn = __shfl_down_sync(CG_FULL, v[0], 1);
    if (lane == 0) up = h;
    if (lane == 31) dn = h;
#pragma unroll
    for (int c = 0; c < CX; ++c) {
        const double W = (c == 0) ? up : v[c - 1];
        const double E = (c == CX - 1) ? dn : v[c + 1];
        R[c] = W + E;
        T[c] = fma(ct, v[c], R[c]);
    }
}

// ------------------------------------------------------------ tile worker

// Buffers of one state being advanced: input, output, and its scratch block
// (zb | acc | Ya | Yb).
// With `store` set, every stage input of every step is kept instead: step k
// reads its state from store[k*NS] and its stage inputs from store[k*NS + s]
// and writes store[(k+1)*NS] (states of NV planes each), so that the
// adjoint sweep can revisit them.
// (no default member initializers: the type also lives in shared memory)
struct Bufs {
    const double *zin;
    double *zout;
    double *blk;
    double *store;
};

// Buffers of instance i (plan order): its slice of the packed state, or the
// caller's own per-instance buffers when the launch carries pointer tables.
__device__ __forceinline__ Bufs inst_bufs(const RunArgs &a, const Inst &I, int i)
{
    if (a.zin_tab != nullptr) return Bufs{a.zin_tab[i], a.zout_tab[i], a.ws + I.ws_off, a.store};
    return Bufs{a.z_in + I.off, a.z_out + I.off, a.ws + I.ws_off, a.store};
}

// What a sweep computes: the model's right-hand side (PRIMAL), the same plus
// the local Jacobian dN/dz written to jbuf (PRIMAL_J), or the tangent-linear
// right-hand side D L dz + J dz with J read from jbuf (TANGENT).
enum { KIND_PRIMAL = 0, KIND_PRIMAL_J = 1, KIND_TANGENT = 2 };

// How the non-diffusive gates advance in a one-stage step: with the explicit
// Euler combine like u, or (Sect. 3, Table 2; four-field model only) by
// Rush-Larsen, x_inf + (x - x_inf) e^(al dt), or implicit Euler,
// (x + dt be) / (1 - dt al), from the coefficients of dx/dt = al x + be at
// the step's starting state.
enum { GATE_EXPLICIT = 0, GATE_RUSH_LARSEN = 1, GATE_IMPLICIT_EULER = 2 };

template <int M, int ST, int NS, int CX, int KIND = KIND_PRIMAL, int GT = GATE_EXPLICIT>
struct Stepper {
    using MD = Model<M>;
    static constexpr int NV = MD::NV, ND = MD::ND, NJ = MD::NJ;

    __device__ static inline void load_row(const double *plane, int nx, int yrow, const int (&cx)[CX],
                                           int hx, bool vec, bool want_halo, double (&v)[CX], double &h)
    {
        const double *rp = plane + (int64_t)yrow * nx;
        if (CX == 2 && vec) {
            const double2 d = __ldcg(reinterpret_cast<const double2 *>(rp + cx[0]));
            v[0] = d.x;
            v[CX - 1] = d.y;
        } else {
#pragma unroll
            for (int c = 0; c < CX; ++c) v[c] = __ldcg(rp + cx[c]);
        }
        if (want_halo) h = __ldcg(rp + hx);
    }

    // Store CX values of one row; `own` has bit c set for every stored cell.
    __device__ static inline void store_row(double *rp, int x0, bool vec, unsigned own, const double (&v)[CX])
    {
        if (CX == 2 && vec && own == 3u) {
            __stcg(reinterpret_cast<double2 *>(rp + x0), make_double2(v[0], v[CX - 1]));
        } else {
#pragma unroll
            for (int c = 0; c < CX; ++c)
                if (own & (1u << c)) __stcg(rp + x0 + c, v[c]);
        }
    }

    // Stage s of step `step` on columns [xt, xt + 32 CX) x rows y0..y1 of
    // instance I.  Row mrow_a stores only columns [ma0, ma1), row mrow_b only
    // [mb0, mb1).
    __device__ __forceinline__ static uint32_t seg(const RunArgs &a, const Inst &I, const double *mp,
                                                   const Bufs &B, double *jbuf, int xt, int y0, int y1,
                                                   int mrow_a, int ma0, int ma1, int mrow_b, int mb0, int mb1,
                                                   int s, int64_t step, int lane)
    {
        const int nx = I.nx, ny = I.ny, bc = a.bc;
        const int64_t plane = (int64_t)nx * ny;

        double *blk = B.blk;
        double *zb = blk;
        double *acc = blk + NV * plane;
        double *Ya = blk + 2 * NV * plane;
        double *Yb = blk + 3 * NV * plane;
        const double *zin = B.zin;
        double *zout = B.zout;
        const double *src = (step == 0) ? zin : ((((step - 1) + a.parity) & 1) == 0 ? zout : zb);
        double *dst = (((step + a.parity) & 1) == 0) ? zout : zb;
        const double *Yin = (s == 0) ? src : ((s & 1) ? Ya : Yb);
        double *Ynext = (s & 1) ? Yb : Ya;
        if (B.store != nullptr) {
            const int64_t S = NV * plane;
            src = B.store + step * NS * S;
            dst = B.store + (step + 1) * NS * S;
            Yin = B.store + (step * NS + s) * S;
            Ynext = B.store + (step * NS + s + 1) * S;
        }
        const bool last = (s == NS - 1);
        const double ca = a.cacc[s];
        const double cyv = last ? 0.0 : a.cy[s];

        // columns of this lane's cells and of the tile's halo columns
        const int x0 = xt + CX * lane;
        int cx[CX];
#pragma unroll
        for (int c = 0; c < CX; ++c) cx[c] = map_idx(x0 + c, nx, bc);
        const bool want_halo = (lane == 0) || (lane == 31);
        const int hx = map_idx(lane == 0 ? xt - 1 : xt + 32 * CX, nx, bc);
        const bool full = (x0 + CX - 1) < nx;     // every cell of this lane is inside the grid
        unsigned in_grid = 0;
#pragma unroll
        for (int c = 0; c < CX; ++c) in_grid |= (x0 + c < nx) ? (1u << c) : 0u;
        unsigned own_a = 0, own_b = 0;
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            own_a |= (x0 + c >= ma0 && x0 + c < ma1) ? (1u << c) : 0u;
            own_b |= (x0 + c >= mb0 && x0 + c < mb1) ? (1u << c) : 0u;
        }
        own_a &= in_grid;
        own_b &= in_grid;
        const bool aligned_base = I.vec_ok != 0;
        auto vec_for = [&](const void *p) {
            return CX == 2 && aligned_base && full && ((reinterpret_cast<uintptr_t>(p) & 15) == 0);
        };
        const bool vin = vec_for(Yin), vsrc = vec_for(src), vacc = vec_for(acc);
        const bool vdst = vec_for(dst), vyn = vec_for(Ynext);
        if constexpr (BOUNDS_CHECK) {
            const bool vec_row = aligned_base && full;
            bool rows = row_out_of_grid(y0, ny) || row_out_of_grid(y1, ny) || y1 < y0 ||
                        row_out_of_grid(map_idx(y0 - 1, ny, bc), ny);
            rows = rows || bad_ptr(Yin) || bad_ptr(src) || bad_ptr(dst) || bad_ptr(acc) || bad_ptr(Ynext);
            if constexpr (KIND != KIND_PRIMAL) rows = rows || bad_ptr(jbuf);
            if (cols_out_of_grid<CX>(cx, hx, want_halo, x0, nx, vec_row) || rows) return CG_DEV_BOUNDS;
        }

        // stencil weights of the diffusive fields
        double wx[ND], wy[ND], wd[ND], wt[ND];
#pragma unroll
        for (int f = 0; f < ND; ++f) {
            wx[f] = I.wx[f];
            wy[f] = I.wy[f];
            wd[f] = I.wd[f];
            wt[f] = I.wt[f];
        }
        const typename MD::Coef coef = MD::coef(I);

        // 5-point: three-row window lo/mid/hi.  9-point (row-sum form, see
        // row_sums): the centre row's values and R, and T of the rows below
        // (Tl) and at the centre (Tm).
        constexpr bool RS = (ST == CG_STENCIL9);
        double lo[ND][CX], mid[ND][CX], hi[ND][CX];
        double hlo[ND], hmid[ND], hhi[ND];
        double Rm[ND][CX], Tl[ND][CX], Tm[ND][CX];
#pragma unroll
        for (int f = 0; f < ND; ++f) {
            hlo[f] = hmid[f] = hhi[f] = 0.0;
            load_row(Yin + f * plane, nx, map_idx(y0 - 1, ny, bc), cx, hx, vin, want_halo, lo[f], hlo[f]);
            load_row(Yin + f * plane, nx, y0, cx, hx, vin, want_halo, mid[f], hmid[f]);
            if constexpr (RS) {
                double Rl[CX];
                row_sums<CX>(lane, lo[f], hlo[f], wt[f], Rl, Tl[f]);
                row_sums<CX>(lane, mid[f], hmid[f], wt[f], Rm[f], Tm[f]);
            }
        }

        uint32_t bad = 0;
        for (int y = y0; y <= y1; ++y) {
            const int yn = map_idx(y + 1, ny, bc);
            if constexpr (BOUNDS_CHECK) {
                if (row_out_of_grid(yn, ny)) return bad | CG_DEV_BOUNDS;
            }
#pragma unroll
            for (int f = 0; f < ND; ++f)
                load_row(Yin + f * plane, nx, yn, cx, hx, vin, want_halo, hi[f], hhi[f]);
            const unsigned own = (y == mrow_a) ? own_a : ((y == mrow_b) ? own_b : in_grid);

            // centre values of every field
            double zc[CX][NV];
#pragma unroll
            for (int f = 0; f < NV; ++f) {
                if (f < ND) {
#pragma unroll
                    for (int c = 0; c < CX; ++c) zc[c][f] = mid[f < ND ? f : 0][c];
                } else {
                    double v[CX], dummy;
                    load_row(Yin + f * plane, nx, y, cx, hx, vin, false, v, dummy);
#pragma unroll
                    for (int c = 0; c < CX; ++c) zc[c][f] = v[c];
                }
            }

            // local terms (centre weight folded in)
            double F[CX][NV];
            double gal[CX][3], gbe[CX][3];       // gate coefficients (GT != GATE_EXPLICIT)
            const int64_t ro_j = (int64_t)y * nx;
            if constexpr (KIND == KIND_PRIMAL && GT != GATE_EXPLICIT) {
                static_assert(NS == 1 && NV == 4 && ND == 1, "gate integrators: one stage, four-field model");
#pragma unroll
                for (int c = 0; c < CX; ++c) {
                    double t[NV];
                    MD::local_gates(coef, mp, zc[c], t, gal[c], gbe[c]);
#pragma unroll
                    for (int f = 0; f < NV; ++f) F[c][f] = t[f];
                }
            } else if constexpr (KIND == KIND_PRIMAL) {
#pragma unroll
                for (int c = 0; c < CX; ++c) {
                    double t[NV];
                    MD::local(coef, mp, zc[c], t);
#pragma unroll
                    for (int f = 0; f < NV; ++f) F[c][f] = t[f];
                }
            } else if constexpr (KIND == KIND_PRIMAL_J) {
                double Jv[NJ > 0 ? NJ : 1][CX];
#pragma unroll
                for (int c = 0; c < CX; ++c) {
                    double t[NV], J[NJ > 0 ? NJ : 1];
                    MD::local_jac(coef, mp, zc[c], t, J);
#pragma unroll
                    for (int f = 0; f < NV; ++f) F[c][f] = t[f];
#pragma unroll
                    for (int j = 0; j < NJ; ++j) Jv[j][c] = J[j];
                }
#pragma unroll
                for (int j = 0; j < NJ; ++j) store_row(jbuf + j * plane + ro_j, x0, vin, in_grid, Jv[j]);
            } else {
                double Jv[NJ > 0 ? NJ : 1][CX];
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    double dummy;
                    load_row(jbuf + j * plane, nx, y, cx, hx, vin, false, Jv[j], dummy);
                }
#pragma unroll
                for (int c = 0; c < CX; ++c) {
                    double t[NV], J[NJ > 0 ? NJ : 1];
#pragma unroll
                    for (int j = 0; j < NJ; ++j) J[j] = Jv[j][c];
                    MD::tan_local(coef, mp, J, zc[c], t);
#pragma unroll
                    for (int f = 0; f < NV; ++f) F[c][f] = t[f];
                }
            }

            // off-centre stencil sums of the diffusive fields
            double Rh[ND][CX], Th[ND][CX];
#pragma unroll
            for (int f = 0; f < ND; ++f) {
                if constexpr (RS) {
                    row_sums<CX>(lane, hi[f], hhi[f], wt[f], Rh[f], Th[f]);
#pragma unroll
                    for (int c = 0; c < CX; ++c) {
                        const double acc_f = fma(wd[f], Tl[f][c] + Th[f][c], F[c][f]);
                        F[c][f] = fma(wx[f], Rm[f][c], acc_f);
                    }
                } else {
                    double Ff[CX];
#pragma unroll
                    for (int c = 0; c < CX; ++c) Ff[c] = F[c][f];
                    add_offcentre<ST, CX>(lane, lo[f], mid[f], hi[f], hlo[f], hmid[f], hhi[f], wx[f], wy[f], wd[f],
                                          Ff);
#pragma unroll
                    for (int c = 0; c < CX; ++c) F[c][f] = Ff[c];
                }
            }

            // Runge-Kutta combine and stores
            const int64_t ro = (int64_t)y * nx;
#pragma unroll
            for (int f = 0; f < NV; ++f) {
                double base[CX];
                if (s == 0) {
#pragma unroll
                    for (int c = 0; c < CX; ++c) base[c] = zc[c][f];
                } else {
                    double dummy;
                    load_row(acc + f * plane, nx, y, cx, hx, vacc, false, base, dummy);
                }
                double outv[CX];
#pragma unroll
                for (int c = 0; c < CX; ++c) outv[c] = a.rhs_only ? F[c][f] : fma(ca, F[c][f], base[c]);
                if constexpr (GT != GATE_EXPLICIT) {
                    if (f >= ND) {
#pragma unroll
                        for (int c = 0; c < CX; ++c) {
                            const double al = gal[c][f - ND], be = gbe[c][f - ND], x = base[c];
                            if constexpr (GT == GATE_RUSH_LARSEN) {
                                const double x_inf = be * fast_rcp(-al);      // al < 0
                                outv[c] = fma(x - x_inf, exp_neg(al * ca, coef.tab), x_inf);
                            } else {
                                outv[c] = fma(ca, be, x) * fast_rcp(fma(-ca, al, 1.0));
                            }
                        }
                    }
                }
                store_row((last ? dst : acc) + f * plane + ro, x0, last ? vdst : vacc, own, outv);
                if (last) {
#pragma unroll
                    for (int c = 0; c < CX; ++c)
                        if (own & (1u << c)) bad |= nonfinite_bit(outv[c]);
                } else {
                    double zz[CX];
                    if (s == 0) {
#pragma unroll
                        for (int c = 0; c < CX; ++c) zz[c] = zc[c][f];
                    } else {
                        double dummy;
                        load_row(src + f * plane, nx, y, cx, hx, vsrc, false, zz, dummy);
                    }
                    double yv[CX];
#pragma unroll
                    for (int c = 0; c < CX; ++c) yv[c] = fma(cyv, F[c][f], zz[c]);
                    store_row(Ynext + f * plane + ro, x0, vyn, own, yv);
                }
            }

            // slide the window
#pragma unroll
            for (int f = 0; f < ND; ++f) {
#pragma unroll
                for (int c = 0; c < CX; ++c) {
                    lo[f][c] = mid[f][c];
                    mid[f][c] = hi[f][c];
                    if constexpr (RS) {
                        Tl[f][c] = Tm[f][c];
                        Tm[f][c] = Th[f][c];
                        Rm[f][c] = Rh[f][c];
                    }
                }
                hlo[f] = hmid[f];
                hmid[f] = hhi[f];
            }
        }
        return bad;
    }

    // Queue tile lt of instance I: rows [ty*rows, ...) x columns of tile tx.
    __device__ __forceinline__ static uint32_t tile(const RunArgs &a, const Inst &I, int i, const double *mp,
                                                    int lt, int s, int64_t step, int lane)
    {
        const int tx = lt % I.tiles_x, ty = lt / I.tiles_x;
        const int y0 = ty * a.rows;
        const int y1 = min(y0 + a.rows, I.ny) - 1;
        const Bufs B = inst_bufs(a, I, i);
        return seg(a, I, mp, B, nullptr, tx * 32 * CX, y0, y1, -1, 0, 0, -1, 0, 0, s, step, lane);
    }
};

// Shared-memory copies of a warp's first static-schedule segments and of
// their instance records.  They never change during a launch, but a global
// load after each grid-barrier acquire misses L1, and the segment, its
// instance record and then the state rows would be three dependent L2 round
// trips at the start of every stage.
constexpr int SEG_CACHE = 4;
constexpr int MAX_WARPS = 16;          // 512 threads per block at most
struct SegCache {
    Seg seg[SEG_CACHE];
    Inst inst[SEG_CACHE];
    Bufs bufs[SEG_CACHE];
};

__device__ __forceinline__ void fill_seg_cache(SegCache &c, const RunArgs &a, int sbeg, int send, int lane)
{
    const int n = min(send - sbeg, SEG_CACHE);
    if (lane < n) {
        c.seg[lane] = a.segs[sbeg + lane];
        c.inst[lane] = a.inst[c.seg[lane].inst];
        c.bufs[lane] = inst_bufs(a, c.inst[lane], c.seg[lane].inst);
    }
    __syncwarp();
}

template <int M, int ST, int NS, int CX, int GT = GATE_EXPLICIT>
__global__ void __launch_bounds__(512, 1) k_stage(const RunArgs a)
{
    using S = Stepper<M, ST, NS, CX, KIND_PRIMAL, GT>;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const double *mp = a.mp;
    uint32_t bad = 0;

    auto find_inst = [&](int t) -> int {
        int lo = 0, hi = a.n_inst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.inst[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    // static schedule: this warp's segments
    const int gw = blockIdx.x * nwarps + warp;
    const int sbeg = (a.sched == SCHED_STATIC) ? a.warp_seg[gw] : 0;
    const int send = (a.sched == SCHED_STATIC) ? a.warp_seg[gw + 1] : 0;
    __shared__ SegCache s_cache[MAX_WARPS];
    SegCache &cache = s_cache[warp];
    fill_seg_cache(cache, a, sbeg, send, lane);
    auto run_static = [&](int s, int64_t step) {
        for (int k = sbeg; k < send; ++k) {
            const bool cached = (k - sbeg) < SEG_CACHE;
            const Seg sg = cached ? cache.seg[k - sbeg] : a.segs[k];
            const Inst &I = cached ? cache.inst[k - sbeg] : a.inst[sg.inst];
            const Bufs B = cached ? cache.bufs[k - sbeg] : inst_bufs(a, I, sg.inst);
            bad |= S::seg(a, I, mp, B, nullptr, sg.x0, sg.y0, sg.y1, sg.mrow_a, sg.ma0, sg.ma1, sg.mrow_b,
                          sg.mb0, sg.mb1,
                          s, step, lane);
        }
    };

    if (!a.persistent) {
        const int64_t g = a.g_begin;
        const int s = (int)(g % NS);
        const int64_t step = g / NS;
        if (a.sched == SCHED_STATIC) {
            run_static(s, step);
        } else {
            for (int t = blockIdx.x * nwarps + warp; t < a.n_tiles; t += gridDim.x * nwarps) {
                const int i = find_inst(t);
                const Inst &I = a.inst[i];
                bad |= S::tile(a, I, i, mp, t - I.tile_begin, s, step, lane);
            }
        }
    } else {
        bool first_barrier = true;
        for (int64_t g = a.g_begin; g < a.g_end; ++g) {
            const int s = (int)(g % NS);
            const int64_t step = g / NS;
            if (a.sched == SCHED_STATIC) {
                run_static(s, step);
            } else {
                unsigned *q = a.sync + 2 + (int)(g % 3);
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(a.sync + 2 + (int)((g + 1) % 3), 0u);
                int t = 0;
                if (lane == 0) t = (int)atomicAdd(q, 1u);
                t = __shfl_sync(CG_FULL, t, 0);
                while (t < a.n_tiles) {
                    int tn = 0;
                    if (lane == 0) tn = (int)atomicAdd(q, 1u);
                    const int i = find_inst(t);
                    const Inst &I = a.inst[i];
                    bad |= S::tile(a, I, i, mp, t - I.tile_begin, s, step, lane);
                    t = __shfl_sync(CG_FULL, tn, 0);
                }
            }
            if (g + 1 < a.g_end) {
                const bool ok = stage_sync(a, g, first_barrier);
                first_barrier = false;
                if (!ok) return;
            }
        }
    }
    bad = __reduce_or_sync(CG_FULL, bad);
    if (lane == 0 && bad) atomicOr(a.status, bad);
}

// Kernel table for one model: [stencil][scheme][cx-1].
template <int M>
inline const void *pick_fwd_kernel(int stencil, int scheme, int cx)
{
    if (cx != 1 && cx != 2) return nullptr;
    constexpr bool gates = (M == MODEL_BOCF || M == MODEL_BOCFH);
#define CG_K(ST, NS, CXV) reinterpret_cast<const void *>(&k_stage<M, ST, NS, CXV>)
#define CG_KG(ST, CXV, GT) reinterpret_cast<const void *>(&k_stage<M, ST, 1, CXV, gates ? GT : GATE_EXPLICIT>)
#define CG_SCH(ST, CXV)                                                    \
    switch (scheme) {                                                      \
    case CG_EULER: return CG_K(ST, 1, CXV);                               \
    case CG_HEUN: return CG_K(ST, 2, CXV);                                \
    case CG_RK4: return CG_K(ST, 4, CXV);                                 \
    case CG_RUSH_LARSEN: return gates ? CG_KG(ST, CXV, GATE_RUSH_LARSEN) : nullptr;        \
    case CG_IMPLICIT_EULER: return gates ? CG_KG(ST, CXV, GATE_IMPLICIT_EULER) : nullptr;  \
    default: return nullptr;                                               \
    }
    if (stencil == CG_STENCIL5) {
        if (cx == 1) { CG_SCH(CG_STENCIL5, 1) } else { CG_SCH(CG_STENCIL5, 2) }
    } else if (stencil == CG_STENCIL9) {
        if (cx == 1) { CG_SCH(CG_STENCIL9, 1) } else { CG_SCH(CG_STENCIL9, 2) }
    }
#undef CG_SCH
#undef CG_KG
#undef CG_K
    return nullptr;
}

}  // namespace cgk
