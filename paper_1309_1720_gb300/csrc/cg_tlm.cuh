// Tangent-linear stepping: exact Jacobian-vector products of the discrete
// flow map of the explicit scheme (Sect. 3) for a batch of tangents that
// share one primal trajectory.
//
// For every RK stage each warp first advances the primal state on its static
// segment and stores the local Jacobian dN/dz of that stage at its own cells
// (KIND_PRIMAL_J); it then advances every tangent on the same cells with
// dF = D L dY + J dY (KIND_TANGENT), reading J back from its own stores, so
// the primal and all tangents of a stage need one grid barrier, not two.
//
// Linearized mode: a first run keeps every stage's Jacobian (jstride > 0)
// and later runs advance tangents only (skip_primal), reading them back, for
// repeated Jacobian-vector products at one base point.
#pragma once

#include "cg_stepper.cuh"

namespace cgk {

struct TlmArgs {
    const double *dz_in;   // n_tan tangent states, each n_v planes
    double *dz_out;
    double *tws;           // n_tan scratch blocks of tblk doubles
    double *jbuf;          // NJ planes of stage Jacobian entries (per stage when jstride > 0)
    int32_t n_tan;
    int32_t skip_primal;   // 1: tangents only, with the Jacobians a linearizing run stored
    int64_t tstride;       // doubles per tangent state
    int64_t tblk;          // doubles per tangent scratch block
    int64_t jstride;       // 0: one stage buffer reused; else doubles between stages' Jacobians
};

template <int M, int ST, int NS, int CX>
__global__ void __launch_bounds__(512, 1) k_tlm(const RunArgs a, const TlmArgs t)
{
    using SP = Stepper<M, ST, NS, CX, KIND_PRIMAL_J>;
    using STn = Stepper<M, ST, NS, CX, KIND_TANGENT>;
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
    auto seg_k = [&](int k) { return (k - sbeg) < SEG_CACHE ? cache.seg[k - sbeg] : a.segs[k]; };

    auto stage = [&](int64_t g) {
        const int s = (int)(g % NS);
        const int64_t step = g / NS;
        double *jb = t.jbuf + g * t.jstride;
        if (!t.skip_primal) {
            const Bufs Bp{a.z_in + I.off, a.z_out + I.off, a.ws + I.ws_off, nullptr};
            for (int k = sbeg; k < send; ++k) {
                const Seg sg = seg_k(k);
                bad |= SP::seg(a, I, mp, Bp, jb, sg.x0, sg.y0, sg.y1, sg.mrow_a, sg.ma0, sg.ma1, sg.mrow_b,
                               sg.mb0, sg.mb1, s, step, lane);
            }
        }
        for (int q = 0; q < t.n_tan; ++q) {
            const Bufs Bt{t.dz_in + q * t.tstride, t.dz_out + q * t.tstride, t.tws + q * t.tblk, nullptr};
            for (int k = sbeg; k < send; ++k) {
                const Seg sg = seg_k(k);
                bad |= STn::seg(a, I, mp, Bt, jb, sg.x0, sg.y0, sg.y1, sg.mrow_a, sg.ma0, sg.ma1,
                                sg.mrow_b, sg.mb0, sg.mb1, s, step, lane);
            }
        }
    };

    if (!a.persistent) {
        stage(a.g_begin);
    } else {
        for (int64_t g = a.g_begin; g < a.g_end; ++g) {
            stage(g);
            if (g + 1 < a.g_end && !stage_sync(a, g, g == a.g_begin)) return;
        }
    }
    bad = __reduce_or_sync(CG_FULL, bad);
    if (lane == 0 && bad) atomicOr(a.status, bad);
}

template <int M>
inline const void *pick_tlm_kernel(int stencil, int scheme, int cx)
{
    if (cx != 1 && cx != 2) return nullptr;
#define CG_K(ST, NS, CXV) reinterpret_cast<const void *>(&k_tlm<M, ST, NS, CXV>)
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
