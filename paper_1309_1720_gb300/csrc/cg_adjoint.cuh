// Discrete adjoint of the explicit scheme (Sect. 3): the transpose of the
// Jacobian of one step, applied stage by stage in reverse.
//
// Forward stage s of step k: Y_s = z + dt a_s k_{s-1}, k_s = F(Y_s),
// z' = z + dt sum_s b_s k_s.  Reverse, with lam = dL/dz':
//   kb_{NS-1} = dt b_{NS-1} lam
//   Yb_s      = (D L)^T kb_s + (dN/dz(Y_s))^T kb_s
//   kb_{s-1}  = dt b_{s-1} lam + dt a_s Yb_s
//   dL/dz     = lam + sum_s Yb_s
//   dL/dD_f  += <kb_s,f , (D L Y_s)_f> / Dxx_f   (= <(D L)^T kb_s,f , Y_s,f> / Dxx_f)
// The kernel carries kh_s = kb_s / (dt b_s) instead of kb_s (every
// explicit scheme here has b_s != 0).  With G_s = (D L)^T kh_s +
// (dN/dz(Y_s))^T kh_s, so that Yb_s = dt b_s G_s:
//   kh_{NS-1} = lam
//   kh_{s-1}  = lam + (dt a_s b_s / b_{s-1}) G_s
//   dL/dz     = lam + sum_s dt b_s G_s
//   dL/dD_f  += dt b_s <(D L)^T kh_s,f , Y_s,f> / Dxx_f
// which takes one multiply per field and stage fewer than the kb form (and
// two fewer at s = 0, where kh_{NS-1} of the step before is dL/dz itself);
// the dt b_s of dL/dD is applied once per warp and stage to the warp's
// partial sum of that stage.
//
// (D L)^T under the MIRROR ghosts: L is not symmetric there, but W L is,
// with W the trapezoid weights (1/2 on each boundary line), so
// L^T k = W L (W^-1 k).  The kernel doubles every loaded value that lies on
// a boundary row or column, applies the forward stencil, and halves the
// off-centre sum of boundary cells; all factors are powers of two, hence
// exact.  Under CLAMP and PERIODIC ghosts L is symmetric and no scaling is
// applied.
//
// dL/dD partial sums live in one slot per warp of the static schedule and
// are summed in a fixed order at the end, so gradients are bitwise
// reproducible.
#pragma once

#include "cg_stepper.cuh"

namespace cgk {

struct AdjArgs {
    const double *store;   // the segment's stage inputs, (m NS + 1) states
    double *kb0, *kb1;     // kh = kbar / (dt b) ping-pong
    double chat[4];        // [s] = dt a_s b_s / b_{s-1} (s >= 1)
    double *lam;           // lambda: in dL/dz_{k+1}, out dL/dz_k
    double *lacc;          // running sum lam + sum Yb_s
    double *partial;       // [warps][ND] dL/dD partial sums (accumulated over launches)
    int32_t want_dd;       // nonzero: accumulate dL/dD (else partial is not touched)
    int64_t m;             // steps of this segment
    int64_t r0;            // reverse stage counter at this segment's first reverse stage
};

template <int M, int ST, int NS, int CX>
struct Adjoint {
    using MD = Model<M>;
    using SP = Stepper<M, ST, NS, CX>;
    static constexpr int NV = MD::NV, ND = MD::ND, NJ = MD::NJ;

    // Load one row of a kbar plane scaled by W^-1 (MIRROR; BND segments only).
    template <bool BND>
    __device__ static inline void load_scaled(const double *plane, int nx, int ny, int yrow, const int (&cx)[CX],
                                              int hx, bool vec, bool want_halo, bool mirror, bool xedge,
                                              const double (&fx)[CX], double fh, double (&v)[CX], double &h)
    {
        SP::load_row(plane, nx, yrow, cx, hx, vec, want_halo, v, h);
        if (BND && mirror) {
            if (yrow == 0 || yrow == ny - 1) {
#pragma unroll
                for (int c = 0; c < CX; ++c) v[c] *= 2.0;
                h *= 2.0;
            }
            if (xedge) {
#pragma unroll
                for (int c = 0; c < CX; ++c) v[c] *= fx[c];
                h *= fh;
            }
        }
    }

    // A segment is a BND segment when it may load or own a cell of a
    // boundary row or column (mirror ghosts only): only those carry the
    // W^-1 / W scaling, so the interior's code has none of it.
    __device__ __forceinline__ static bool bnd_segment(const RunArgs &a, const Inst &I, const Seg &sg)
    {
        return a.bc == CG_BC_MIRROR && (sg.x0 <= 1 || sg.x0 + 32 * CX >= I.nx - 1 || sg.y0 <= 1 ||
                                        sg.y1 >= I.ny - 2);
    }

    template <bool BND>
    __device__ __forceinline__ static uint32_t seg(const RunArgs &a, const AdjArgs &b, const Inst &I,
                                                   const double *mp, const Seg &sg, int64_t k, int s, int64_t r,
                                                   int lane, double dtb, double ch, double (&dd)[ND > 0 ? ND : 1])
    {
        const int nx = I.nx, ny = I.ny, bc = a.bc;
        const bool mirror = (bc == CG_BC_MIRROR);
        const int64_t plane = (int64_t)nx * ny;
        const int64_t S = NV * plane;
        const double *Y = b.store + (k * NS + s) * S;
        const double *Kin = (r & 1) ? b.kb1 : b.kb0;
        double *Kout = (r & 1) ? b.kb0 : b.kb1;
        double *lam = b.lam;
        double *lacc = b.lacc;

        const int xt = sg.x0;
        const int x0 = xt + CX * lane;
        int cx[CX];
#pragma unroll
        for (int c = 0; c < CX; ++c) cx[c] = map_idx(x0 + c, nx, bc);
        const bool want_halo = (lane == 0) || (lane == 31);
        const int hx = map_idx(lane == 0 ? xt - 1 : xt + 32 * CX, nx, bc);
        const bool full = (x0 + CX - 1) < nx;
        unsigned in_grid = 0, own_a = 0, own_b = 0;
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            in_grid |= (x0 + c < nx) ? (1u << c) : 0u;
            own_a |= (x0 + c >= sg.ma0 && x0 + c < sg.ma1) ? (1u << c) : 0u;
            own_b |= (x0 + c >= sg.mb0 && x0 + c < sg.mb1) ? (1u << c) : 0u;
        }
        own_a &= in_grid;
        own_b &= in_grid;
        auto vec_for = [&](const void *p) {
            return CX == 2 && I.vec_ok != 0 && full && ((reinterpret_cast<uintptr_t>(p) & 15) == 0);
        };
        const bool vk = vec_for(Kin) && vec_for(Kout), vy = vec_for(Y), vl = vec_for(lam) && vec_for(lacc);
        if constexpr (BOUNDS_CHECK) {
            const bool rows = row_out_of_grid(sg.y0, ny) || row_out_of_grid(sg.y1, ny) || sg.y1 < sg.y0 ||
                              row_out_of_grid(map_idx(sg.y0 - 1, ny, bc), ny) || bad_ptr(Y) || bad_ptr(Kin) ||
                              bad_ptr(Kout) || bad_ptr(lam) || bad_ptr(lacc);
            if (cols_out_of_grid<CX>(cx, hx, want_halo, x0, nx, I.vec_ok != 0 && full) || rows)
                return CG_DEV_BOUNDS;
        }

        // W^-1 factors of this lane's columns and halo column; W of its cells
        double fx[CX], wcol[CX];
        bool edge_lane = false;
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            const bool e = (cx[c] == 0 || cx[c] == nx - 1);
            fx[c] = e ? 2.0 : 1.0;
            const bool ecell = (x0 + c == 0 || x0 + c == nx - 1);
            wcol[c] = ecell ? 0.5 : 1.0;
            edge_lane |= e || ecell;
        }
        const double fh = (hx == 0 || hx == nx - 1) ? 2.0 : 1.0;
        if (want_halo && fh != 1.0) edge_lane = true;
        const bool xedge = BND && mirror && __any_sync(CG_FULL, edge_lane);

        double wx[ND], wy[ND], wd[ND], wcf[ND];
#pragma unroll
        for (int f = 0; f < ND; ++f) {
            wx[f] = I.wx[f];
            wy[f] = I.wy[f];
            wd[f] = I.wd[f];
            wcf[f] = I.wc[f];
        }
        const typename MD::Coef coef = MD::coef(I);

        double lo[ND][CX], mid[ND][CX], hi[ND][CX];
        double hlo[ND], hmid[ND], hhi[ND];
#pragma unroll
        for (int f = 0; f < ND; ++f) {
            hlo[f] = hmid[f] = hhi[f] = 0.0;
            load_scaled<BND>(Kin + f * plane, nx, ny, map_idx(sg.y0 - 1, ny, bc), cx, hx, vk, want_halo, mirror, xedge,
                        fx, fh, lo[f], hlo[f]);
            load_scaled<BND>(Kin + f * plane, nx, ny, sg.y0, cx, hx, vk, want_halo, mirror, xedge, fx, fh, mid[f],
                        hmid[f]);
        }

        uint32_t bad = 0;
        for (int y = sg.y0; y <= sg.y1; ++y) {
            const int yn = map_idx(y + 1, ny, bc);
            if constexpr (BOUNDS_CHECK) {
                if (row_out_of_grid(yn, ny)) return bad | CG_DEV_BOUNDS;
            }
#pragma unroll
            for (int f = 0; f < ND; ++f)
                load_scaled<BND>(Kin + f * plane, nx, ny, yn, cx, hx, vk, want_halo, mirror, xedge, fx, fh, hi[f],
                            hhi[f]);
            const unsigned own = (y == sg.mrow_a) ? own_a : ((y == sg.mrow_b) ? own_b : in_grid);
            const bool yedge = BND && mirror && (y == 0 || y == ny - 1);
            const bool bnd = yedge || xedge;      // warp-uniform: some cell of this row may sit on the boundary
            double wcell[CX];
#pragma unroll
            for (int c = 0; c < CX; ++c) wcell[c] = 1.0;
            if (bnd) {
#pragma unroll
                for (int c = 0; c < CX; ++c) wcell[c] = (yedge ? 0.5 : 1.0) * (mirror ? wcol[c] : 1.0);
            }

            // primal stage input and kbar at the cells
            double yc[CX][NV], kc[CX][NV];
#pragma unroll
            for (int f = 0; f < NV; ++f) {
                double v[CX], dummy;
                SP::load_row(Y + f * plane, nx, y, cx, hx, vy, false, v, dummy);
#pragma unroll
                for (int c = 0; c < CX; ++c) yc[c][f] = v[c];
                if (f < ND) {
                    // boundary rows/columns only (warp-uniform branch, so the
                    // interior does not pay for the multiplies)
#pragma unroll
                    for (int c = 0; c < CX; ++c) kc[c][f] = mid[f < ND ? f : 0][c];
                    if (bnd) {
#pragma unroll
                        for (int c = 0; c < CX; ++c) kc[c][f] *= wcell[c];
                    }
                } else {
                    SP::load_row(Kin + f * plane, nx, y, cx, hx, vk, false, v, dummy);
#pragma unroll
                    for (int c = 0; c < CX; ++c) kc[c][f] = v[c];
                }
            }

            // local part J^T kbar (centre weight folded in)
            double F[CX][NV];
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                double t[NV], J[NJ > 0 ? NJ : 1], tf[NV];
                MD::local_jac(coef, mp, yc[c], tf, J);
                MD::adj_local(coef, mp, J, kc[c], t);
#pragma unroll
                for (int f = 0; f < NV; ++f) F[c][f] = t[f];
            }

            // transposed off-centre part W (L_off (W^-1 kbar)) and the dL/dD dot
#pragma unroll
            for (int f = 0; f < ND; ++f) {
                double So[CX];
#pragma unroll
                for (int c = 0; c < CX; ++c) So[c] = 0.0;
                add_offcentre<ST, CX>(lane, lo[f], mid[f], hi[f], hlo[f], hmid[f], hhi[f], wx[f], wy[f], wd[f], So);
                if (bnd) {
#pragma unroll
                    for (int c = 0; c < CX; ++c) So[c] *= wcell[c];
                }
#pragma unroll
                for (int c = 0; c < CX; ++c) {
                    const double Sw = So[c];
                    F[c][f] += Sw;
                    if (b.want_dd) {                                    // kernel argument: warp-uniform
                        const double lt = fma(wcf[f], kc[c][f], Sw);    // ((D L)^T kbar)_f at the cell
                        if (own & (1u << c)) dd[f] = fma(yc[c][f], lt, dd[f]);
                    }
                }
            }

            // reverse combine (F holds G_s)
            const int64_t ro = (int64_t)y * nx;
#pragma unroll
            for (int f = 0; f < NV; ++f) {
                double lv[CX], dummy;
                SP::load_row(lam + f * plane, nx, y, cx, hx, vl, false, lv, dummy);
                double base[CX];
                if (s == NS - 1) {
#pragma unroll
                    for (int c = 0; c < CX; ++c) base[c] = lv[c];
                } else {
                    SP::load_row(lacc + f * plane, nx, y, cx, hx, vl, false, base, dummy);
                }
                double na[CX];
#pragma unroll
                for (int c = 0; c < CX; ++c) na[c] = fma(dtb, F[c][f], base[c]);
                if (s > 0) {
                    double ko[CX];
#pragma unroll
                    for (int c = 0; c < CX; ++c) ko[c] = fma(ch, F[c][f], lv[c]);
                    SP::store_row(lacc + f * plane + ro, x0, vl, own, na);
                    SP::store_row(Kout + f * plane + ro, x0, vk, own, ko);
                } else {
#pragma unroll
                    for (int c = 0; c < CX; ++c)
                        if (own & (1u << c)) bad |= nonfinite_bit(na[c]);
                    SP::store_row(lam + f * plane + ro, x0, vl, own, na);
                    SP::store_row(Kout + f * plane + ro, x0, vk, own, na);
                }
            }

#pragma unroll
            for (int f = 0; f < ND; ++f) {
#pragma unroll
                for (int c = 0; c < CX; ++c) {
                    lo[f][c] = mid[f][c];
                    mid[f][c] = hi[f][c];
                }
                hlo[f] = hmid[f];
                hmid[f] = hhi[f];
            }
        }
        return bad;
    }
};

template <int M, int ST, int NS, int CX>
__global__ void __launch_bounds__(512, 1) k_adj(const RunArgs a, const AdjArgs b)
{
    using AD = Adjoint<M, ST, NS, CX>;
    constexpr int ND = AD::ND;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const double *mp = a.mp;
    const int gw = blockIdx.x * nwarps + warp;
    const int sbeg = a.warp_seg[gw], send = a.warp_seg[gw + 1];
    __shared__ SegCache s_cache[MAX_WARPS];
    SegCache &cache = s_cache[warp];
    fill_seg_cache(cache, a, sbeg, send, lane);
    __shared__ Inst s_inst;                  // the single instance (see SegCache)
    if (threadIdx.x == 0) s_inst = a.inst[0];
    __syncthreads();
    const Inst &I = s_inst;
    uint32_t bad = 0;
    // dL/dD: dds sums one stage's <(D L)^T kh, Y> over the lane's cells,
    // s_dd (shared memory: touched once per stage, so it takes no registers
    // from the stage worker) the stages' sums weighted by dt b_s
    double dds[ND > 0 ? ND : 1];
    __shared__ double s_dd[ND > 0 ? ND : 1][512];
#pragma unroll
    for (int f = 0; f < ND; ++f) s_dd[f][threadIdx.x] = 0.0;

    auto stage = [&](int64_t g) {
        const int64_t k = b.m - 1 - g / NS;
        const int s = NS - 1 - (int)(g % NS);
        // dt b_s and dt a_s b_s / b_{s-1} of this stage (constant indices
        // only, so the argument blocks stay in the parameter bank)
        double dtb = a.cacc[0], ch = 0.0;
#pragma unroll
        for (int q = 1; q < NS; ++q) {
            if (s == q) {
                dtb = a.cacc[q];
                ch = b.chat[q];
            }
        }
#pragma unroll
        for (int f = 0; f < ND; ++f) dds[f] = 0.0;
        for (int q = sbeg; q < send; ++q) {
            const Seg sg = (q - sbeg) < SEG_CACHE ? cache.seg[q - sbeg] : a.segs[q];
            if (AD::bnd_segment(a, I, sg))
                bad |= AD::template seg<true>(a, b, I, mp, sg, k, s, b.r0 + g, lane, dtb, ch, dds);
            else
                bad |= AD::template seg<false>(a, b, I, mp, sg, k, s, b.r0 + g, lane, dtb, ch, dds);
        }
        if (b.want_dd) {
#pragma unroll
            for (int f = 0; f < ND; ++f) s_dd[f][threadIdx.x] = fma(dtb, dds[f], s_dd[f][threadIdx.x]);
        }
    };

    bool ok = true;
    if (!a.persistent) {
        stage(a.g_begin);
    } else {
        for (int64_t g = a.g_begin; g < a.g_end; ++g) {
            stage(g);
            if (g + 1 < a.g_end && !stage_sync(a, g, g == a.g_begin)) {
                ok = false;
                break;
            }
        }
    }
    if (!ok) return;
    // fixed-order warp reduction of the dL/dD partials, one slot per warp
    if (b.want_dd) {
#pragma unroll
        for (int f = 0; f < ND; ++f) {
            double v = s_dd[f][threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(CG_FULL, v, o);
            if (lane == 0) b.partial[(int64_t)gw * ND + f] += v;
        }
    }
    bad = __reduce_or_sync(CG_FULL, bad);
    if (lane == 0 && bad) atomicOr(a.status, bad);
}

struct Inv4 { double v[4]; };
// out[f] = (sum over w of partial[w*nd + f]) * inv.v[f], summed in index order.
__global__ void k_reduce_partials(const double *partial, int nw, int nd, Inv4 inv, double *out);

template <int M>
inline const void *pick_adj_kernel(int stencil, int scheme, int cx)
{
    if (cx != 1 && cx != 2) return nullptr;
#define CG_K(ST, NS, CXV) reinterpret_cast<const void *>(&k_adj<M, ST, NS, CXV>)
#define CG_SCH(ST, CXV)                                  \
    switch (scheme) {                                    \
    case CG_EULER: return CG_K(ST, 1, CXV);             \
    case CG_HEUN: return CG_K(ST, 2, CXV);              \
    case CG_RK4: return CG_K(ST, 4, CXV);               \
    default: return nullptr;                             \
    }
    if (stencil == CG_STENCIL5) {
        if (cx == 1) { CG_SCH(CG_STENCIL5, 1) } else { CG_SCH(CG_STENCIL5, 2) }
    } else if (stencil == CG_STENCIL9) {
        if (cx == 1) { CG_SCH(CG_STENCIL9, 1) } else { CG_SCH(CG_STENCIL9, 2) }
    }
#undef CG_SCH
#undef CG_K
    return nullptr;
}

}  // namespace cgk
