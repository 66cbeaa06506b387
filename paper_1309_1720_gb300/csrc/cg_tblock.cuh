// Temporally blocked stepping for small grids (one instance or a batch,
// mirror or clamp ghosts).
//
// On a small grid every stage of the persistent stage kernel costs about one
// grid barrier plus one L2 round trip, far more than its arithmetic.  Here
// the instances are cut into rectangular tiles (a single instance: one per
// block; a batch: the blocks loop over them).  A tile is loaded with a halo
// of H = K n_s cells (K steps of n_s stages), advanced through all H stages
// in shared memory, the region it updates shrinking by one cell per stage (a
// stage reads one ring of neighbours), and written back: one grid barrier
// per K steps instead of one per stage, at the price of recomputing the halo.
// Ghost points (Fig. 1) at the domain's edges are loaded from the cells
// they mirror (or repeat), and at each stage a region that reaches an edge
// also computes its ghost ring, every ghost evaluated as its source cell
// (same inputs, hence the same value): the shrinking region never needs
// values from another tile between barriers, and no stage needs a separate
// ghost refill.
//
// Between passes the blocks synchronise either with the grid barrier or,
// for a single instance, with neighbour waits: a block publishes how many
// passes it has finished and, before the next one, waits only for the tiles
// whose cells its window covers (they write what it reads next, and read
// what it overwrites next), so blocks drift against distant tiles and no
// grid-wide round trip is paid.
//
// Each cell's arithmetic is the stage kernel's: the model's local terms with
// the centre weight folded in, the off-centre sums in the same order (5-point:
// wy (S + N) then wx (W + E); 9-point: row sums R = W + E and
// T = R + (wy/wd) C, then wd (T_south + T_north) and wx R), and the same
// Runge-Kutta combine, so results equal cg_run's other launch shapes bit for
// bit (the row sums are formed per cell here instead of once per row).
#pragma once

#include "cg_stepper.cuh"

namespace cgk {

struct TbArgs {
    int32_t tx, ty;          // tile size (cells)
    int32_t n_tiles;         // tiles of all instances (instance i owns [tb_tile_begin, + tb_tiles))
    int32_t k;               // steps per pass
    int32_t wmax;            // shared window capacity in cells (per array)
    int32_t nbr;             // 1: neighbour waits between passes (single instance, one tile per block)
    int32_t tiles_x, tiles_y;   // tile grid of the single instance (neighbour waits)
    int32_t rx, ry;          // a window covers tiles within rx columns and ry rows of its own
    int64_t n_steps;
};

// Neighbour synchronisation between passes (single instance, tile b on
// block b): publish `done` passes, then wait (bounded) until every tile
// within rx columns and ry rows has published `need`.  The lanes of warp 0
// poll up to 32 flags at once.  On expiry the block records CG_DEV_TIMEOUT
// and every thread returns false.
static __device__ __noinline__ bool tb_neighbor_sync(unsigned *flags, uint32_t *status, uint64_t timeout_ns,
                                                     unsigned done, unsigned need, const TbArgs &t)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0) {
            // the block's stores of this pass, ordered before by
            // __syncthreads, become visible with the release
            __threadfence();
            st_release_u32(flags + blockIdx.x, done);
        }
        __syncwarp();
        const int bx = (int)blockIdx.x % t.tiles_x, by = (int)blockIdx.x / t.tiles_x;
        const int x0 = max(bx - t.rx, 0), x1 = min(bx + t.rx, t.tiles_x - 1);
        const int y0 = max(by - t.ry, 0), y1 = min(by + t.ry, t.tiles_y - 1);
        const int w = x1 - x0 + 1, cnt = w * (y1 - y0 + 1);
        int ok = 1;
        const uint64_t t0 = global_timer_ns();
        const uint64_t max_iter = (timeout_ns >> 5) + (1ull << 20);
        uint64_t it = 0;
        for (int base = 0; base < cnt && ok; base += 32) {
            const int j = base + lane;
            const unsigned *f = flags + ((j < cnt) ? (y0 + j / w) * t.tiles_x + (x0 + j % w) : (int)blockIdx.x);
            for (;;) {
                const bool ready = ld_acquire_u32(f) >= need;
                if (__all_sync(CG_FULL, ready)) break;
                __nanosleep(32);
                const bool expired = (++it & 63) == 0 && (global_timer_ns() - t0 > timeout_ns || it > max_iter);
                if (__any_sync(CG_FULL, expired)) {
                    ok = 0;
                    if (lane == 0) atomicOr(status, CG_DEV_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
        if (lane == 0) s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Output buffer of an instance in pass p of P: the last pass writes its
// output, except in place (input == output) where the first pass must not
// overwrite its input; the other passes alternate with the instance's
// scratch copy.
__device__ __forceinline__ double *tb_dst(double *out, double *scr, bool alias, int64_t p, int64_t P)
{
    if (alias) return (p & 1) ? out : scr;
    return (((P - 1 - p) & 1) == 0) ? out : scr;
}

// Window [w0, w1) along one axis for the tile [t0, t1) of an axis of n
// cells and a halo of h: the halo, except that on a side where it reaches
// the domain's edge the window stops at the ghost point (-1 or n) so that
// the ghosts always have a slot.  Used on the host too.
__host__ __device__ inline void tb_window(int t0, int t1, int n, int h, int &w0, int &w1)
{
    w0 = (t0 - h <= 0) ? -1 : t0 - h;
    w1 = (t1 + h >= n) ? n + 1 : t1 + h;
}

template <int M, int ST, int NS>
__global__ void __launch_bounds__(512, 1) k_tblock(const RunArgs a, const TbArgs t)
{
    using MD = Model<M>;
    constexpr int NV = MD::NV, ND = MD::ND;
    extern __shared__ double sm[];
    __shared__ Inst s_inst;
    int cur = -1;                            // instance held in s_inst (the same in every thread)
    const int bc = a.bc;
    const int Hmax = t.k * NS;
    const int WS = t.wmax;
    // arrays (each NV planes of WS): NS == 1: YA, YB; else Z, ACC, YA, YB
    double *Z = sm;
    double *ACC = Z + (NS > 1 ? NV * WS : 0);
    double *YA = ACC + (NS > 1 ? NV * WS : 0);
    double *YB = YA + NV * WS;
    if (NS == 1) Z = YA;
    const double *mp = a.mp;
    uint32_t bad = 0;

    // Per-tile constants (one tile of one instance).
    struct TbCtx {
        int i, nx, ny, x0, y0, x1, y1, gx0, gx1, gy0, gy1, WX;
        double wx[ND > 0 ? ND : 1], wy[ND > 0 ? ND : 1], wd[ND > 0 ? ND : 1], wt[ND > 0 ? ND : 1];
        typename MD::Coef coef;
        const double *zin;
        double *zout, *scr;
    };
    // The tile's instance (every thread finds the same one; a single
    // instance needs no search) is staged in shared memory when it changes.
    auto make_ctx = [&](int tile) {
        int i = 0;
        if (a.n_inst > 1) {
            int hi = a.n_inst - 1;
            while (i < hi) {
                const int mid = (i + hi + 1) >> 1;
                if (a.inst[mid].tb_tile_begin <= tile) i = mid; else hi = mid - 1;
            }
        }
        if (i != cur) {
            __syncthreads();
            if (threadIdx.x == 0) s_inst = a.inst[i];
            __syncthreads();
            cur = i;
        }
        const Inst &I = s_inst;
        TbCtx c;
        c.i = i;
        c.nx = I.nx;
        c.ny = I.ny;
        const int lt = tile - I.tb_tile_begin;
        c.x0 = (lt % I.tb_tiles_x) * t.tx;
        c.y0 = (lt / I.tb_tiles_x) * t.ty;
        c.x1 = min(c.x0 + t.tx, c.nx);
        c.y1 = min(c.y0 + t.ty, c.ny);
        // window: the tile with Hmax cells of halo; where that reaches the
        // domain's edge it ends at the ghost layer instead (tb_window)
        tb_window(c.x0, c.x1, c.nx, Hmax, c.gx0, c.gx1);
        tb_window(c.y0, c.y1, c.ny, Hmax, c.gy0, c.gy1);
        c.WX = c.gx1 - c.gx0;
#pragma unroll
        for (int f = 0; f < ND; ++f) {
            c.wx[f] = I.wx[f];
            c.wy[f] = I.wy[f];
            c.wd[f] = I.wd[f];
            c.wt[f] = I.wt[f];
        }
        c.coef = MD::coef(I);
        c.zin = a.zin_tab ? a.zin_tab[i] : a.z_in + I.off;
        c.zout = a.zout_tab ? a.zout_tab[i] : a.z_out + I.off;
        c.scr = a.ws + I.ws_off;
        return c;
    };

    const int64_t P = (t.n_steps + t.k - 1) / t.k;
    // Pass p (H stages) of one tile: load the window, advance it, write the
    // tile back.
    auto run_tile = [&](const TbCtx &c, int64_t p, int H) {
        const int nx = c.nx, ny = c.ny;
        const int x0 = c.x0, y0 = c.y0, x1 = c.x1, y1 = c.y1;
        const int gx0 = c.gx0, gx1 = c.gx1, gy0 = c.gy0, gy1 = c.gy1, WX = c.WX;
        auto at = [&](int gx, int gy) { return (gy - gy0) * WX + (gx - gx0); };
        // checked build: (gx, gy) is a window cell and the window fits the arrays
        const bool win_fits = WX * (gy1 - gy0) <= WS;
        auto in_window = [&](int gx, int gy) {
            return win_fits && gx >= gx0 && gx < gx1 && gy >= gy0 && gy < gy1;
        };
        double wx[ND > 0 ? ND : 1], wy[ND > 0 ? ND : 1], wd[ND > 0 ? ND : 1], wt[ND > 0 ? ND : 1];
#pragma unroll
        for (int f = 0; f < ND; ++f) {
            wx[f] = c.wx[f];
            wy[f] = c.wy[f];
            wd[f] = c.wd[f];
            wt[f] = c.wt[f];
        }
        const typename MD::Coef coef = c.coef;
        const int64_t plane = (int64_t)nx * ny;
        const bool alias = (c.zin == c.zout);
        const double *src = (p == 0) ? c.zin : tb_dst(c.zout, c.scr, alias, p - 1, P);
        double *dst = tb_dst(c.zout, c.scr, alias, p, P);

        // checked build: a window that does not fit its arrays skips every
        // access of this tile (the block still joins the grid barriers)
        const bool tb_ok = !BOUNDS_CHECK || (win_fits && WX >= 3 && gy1 - gy0 >= 3);
        if (!tb_ok) {
            bad |= CG_DEV_BOUNDS;
            return;
        }
        // load the window: the tile plus H cells of halo and, where that
        // reaches the domain's edge, the ghost points (read from the cells
        // they mirror or repeat)
        {
            const int xl = max(x0 - H, 0), xh = min(x1 + H, nx), yl = max(y0 - H, 0), yh = min(y1 + H, ny);
            const int exl = xl - (xl == 0), exh = xh + (xh == nx), eyl = yl - (yl == 0), eyh = yh + (yh == ny);
            const int w = exh - exl, n = w * (eyh - eyl);
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                const int gx = exl + c % w, gy = eyl + c / w;
                const int sx = map_idx(gx, nx, bc), sy = map_idx(gy, ny, bc);
                if constexpr (BOUNDS_CHECK) {
                    if (!in_window(gx, gy) || sx < 0 || sx >= nx || sy < 0 || sy >= ny || bad_ptr(src)) {
                        bad |= CG_DEV_BOUNDS;
                        continue;
                    }
                }
#pragma unroll
                for (int f = 0; f < NV; ++f)
                    Z[f * WS + at(gx, gy)] = __ldcg(src + f * plane + (int64_t)sy * nx + sx);
            }
            __syncthreads();
        }
        double *Yin = Z;
        for (int g = 1; g <= H; ++g) {
            const int s = (g - 1) % NS;
            const bool last = (s == NS - 1);
            const int rad = H - g;
            const int xl = max(x0 - rad, 0), xh = min(x1 + rad, nx), yl = max(y0 - rad, 0), yh = min(y1 + rad, ny);
            // Where the region reaches the domain's edge it takes in the
            // ghost ring, each ghost computed as the cell it mirrors (same
            // inputs, same value), so no refill is needed; not at the pass's
            // last stage, which nothing reads.  A ghost's source is at most
            // two cells in, inside the previous stage's region.
            const bool gr = g < H;
            const int exl = xl - (gr && xl == 0), exh = xh + (gr && xh == nx);
            const int eyl = yl - (gr && yl == 0), eyh = yh + (gr && yh == ny);
            const int w = exh - exl, n = w * (eyh - eyl);
            double *Yout = (NS == 1) ? ((Yin == YA) ? YB : YA) : (last ? Z : ((s & 1) ? YB : YA));
            const double ca = a.cacc[s], cyv = last ? 0.0 : a.cy[s];
            // Rounds of up to blockDim cells, cell c of a round on thread c.
            // The FP64 pipe takes a warp instruction in the same time
            // whether 1 or 32 lanes are active (measured on GB300), so
            // cells are packed into as few warps as possible.  A warp
            // with no cell skips the round (warp-uniform); in the others
            // every lane runs, so the model's warp-uniform paths see whole
            // warps: surplus lanes repeat the round's last cell and store
            // nothing.
            const int wid = (int)(threadIdx.x >> 5);
            for (int base = 0; base < n; base += blockDim.x) {
                const int m = min(n - base, (int)blockDim.x);
                if ((wid << 5) >= m) continue;
                const int c = base + (int)threadIdx.x;
                const bool act = c < base + m;
                const int cc = act ? c : base + m - 1;
                const int gx = exl + cc % w, gy = eyl + cc / w;
                const int sx = map_idx(gx, nx, bc), sy = map_idx(gy, ny, bc);   // identity inside the grid
                int li = at(gx, gy), ls = at(sx, sy);
                bool act_ok = act;
                if constexpr (BOUNDS_CHECK) {
                    // the slot, the source cell and its eight neighbours
                    // inside the window; a failed check computes a harmless
                    // interior cell instead and stores nothing (whole warps
                    // stay)
                    if (!(in_window(gx, gy) && in_window(sx - 1, sy - 1) && in_window(sx + 1, sy + 1))) {
                        bad |= CG_DEV_BOUNDS;
                        li = ls = WX + 1;
                        act_ok = false;
                    }
                }
                double zc[NV];
#pragma unroll
                for (int f = 0; f < NV; ++f) zc[f] = Yin[f * WS + ls];
                double F[NV];
                MD::local(coef, mp, zc, F);
#pragma unroll
                for (int f = 0; f < ND; ++f) {
                    const double *Q = Yin + f * WS;
                    const double Wv = Q[ls - 1], Ev = Q[ls + 1];
                    if (ST == CG_STENCIL9) {
                        const double Rl = Q[ls - WX - 1] + Q[ls - WX + 1];
                        const double Rh = Q[ls + WX - 1] + Q[ls + WX + 1];
                        const double Tl = fma(wt[f], Q[ls - WX], Rl), Th = fma(wt[f], Q[ls + WX], Rh);
                        const double acc_f = fma(wd[f], Tl + Th, F[f]);
                        F[f] = fma(wx[f], Wv + Ev, acc_f);
                    } else {
                        double acc_f = fma(wy[f], Q[ls - WX] + Q[ls + WX], F[f]);
                        F[f] = fma(wx[f], Wv + Ev, acc_f);
                    }
                }
                if (act_ok) {
#pragma unroll
                    for (int f = 0; f < NV; ++f) {
                        const int o = f * WS + li;
                        if (NS == 1) {
                            Yout[o] = fma(ca, F[f], zc[f]);
                        } else if (s == 0) {
                            ACC[o] = fma(ca, F[f], zc[f]);
                            Yout[o] = fma(cyv, F[f], zc[f]);
                        } else if (!last) {
                            ACC[o] = fma(ca, F[f], ACC[o]);
                            Yout[o] = fma(cyv, F[f], Z[o]);
                        } else {
                            Yout[o] = fma(ca, F[f], ACC[o]);
                        }
                    }
                }
            }
            __syncthreads();
            Yin = Yout;
        }
        // write the tile back
        {
            const int w = x1 - x0, n = w * (y1 - y0);
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                const int gx = x0 + c % w, gy = y0 + c / w;
                if constexpr (BOUNDS_CHECK) {
                    if (!in_window(gx, gy) || gx < 0 || gx >= nx || gy < 0 || gy >= ny || bad_ptr(dst)) {
                        bad |= CG_DEV_BOUNDS;
                        continue;
                    }
                }
#pragma unroll
                for (int f = 0; f < NV; ++f) {
                    const double v = Yin[f * WS + at(gx, gy)];
                    bad |= nonfinite_bit(v);
                    __stcg(dst + f * plane + (int64_t)gy * nx + gx, v);
                }
            }
        }
    };

    auto pass_end = [&](int64_t p) {
        if (p + 1 < P) {
            const unsigned extra = (p == 0 && a.stuck_barrier) ? 1u : 0u;
            if (t.nbr)
                return tb_neighbor_sync(a.flags, a.status, a.timeout_ns, (unsigned)(p + 1), (unsigned)(p + 1) + extra,
                                        t);
            const unsigned long long target = (unsigned long long)(p + 1) * a.nblocks_expect + extra;
            return grid_barrier(reinterpret_cast<unsigned long long *>(a.sync), a.status, a.timeout_ns, target);
        }
        return true;
    };
    auto pass_depth = [&](int64_t p) {
        const int64_t rest = t.n_steps - p * t.k;
        return (int)(rest < t.k ? rest : t.k) * NS;
    };
    if (t.n_tiles <= (int)gridDim.x) {
        // at most one tile per block (a single instance): its constants once
        TbCtx c;
        const bool has = (int)blockIdx.x < t.n_tiles;
        if (has) c = make_ctx(blockIdx.x);
        for (int64_t p = 0; p < P; ++p) {
            if (has) run_tile(c, p, pass_depth(p));
            if (!pass_end(p)) return;
        }
    } else {
        // a batch: the blocks take tiles blockIdx.x, + gridDim.x, ... of all
        // instances in every pass
        for (int64_t p = 0; p < P; ++p) {
            const int H = pass_depth(p);
            for (int tile = blockIdx.x; tile < t.n_tiles; tile += gridDim.x) {
                const TbCtx c = make_ctx(tile);
                run_tile(c, p, H);
                // the next tile reuses the arrays (block-uniform)
                if (tile + (int)gridDim.x < t.n_tiles) __syncthreads();
            }
            if (!pass_end(p)) return;
        }
    }
    bad = __reduce_or_sync(CG_FULL, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicOr(a.status, bad);
}

// Kernel table for one model: [stencil][scheme] (explicit schemes only).
template <int M>
inline const void *pick_tb_kernel(int stencil, int scheme)
{
#define CG_TB(ST)                                                                               \
    switch (scheme) {                                                                           \
    case CG_EULER: return reinterpret_cast<const void *>(&k_tblock<M, ST, 1>);                  \
    case CG_HEUN: return reinterpret_cast<const void *>(&k_tblock<M, ST, 2>);                   \
    case CG_RK4: return reinterpret_cast<const void *>(&k_tblock<M, ST, 4>);                    \
    default: return nullptr;                                                                    \
    }
    if (stencil == CG_STENCIL5) { CG_TB(CG_STENCIL5) }
    if (stencil == CG_STENCIL9) { CG_TB(CG_STENCIL9) }
#undef CG_TB
    return nullptr;
}

// Shared memory of k_tblock (bytes) for a window of wmax cells per array.
inline size_t tb_smem_bytes(int nv, int ns, int wmax)
{
    return sizeof(double) * (size_t)nv * (ns == 1 ? 2 : 4) * (size_t)wmax;
}

}  // namespace cgk
