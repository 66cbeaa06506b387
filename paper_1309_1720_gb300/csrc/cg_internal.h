// Internal definitions shared by the host library and the kernels of
// libcardiac_gb300.so.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "cardiac_gb300.h"

namespace cgk {

constexpr int MAXF = 4;     // fields per cell (BOCF: u, v, w, s)
constexpr int NMP = 64;     // model constants shared by all instances of a plan
constexpr int EXP_TAB = 4096; // entries 2^(j/4096) of the exponential's table (cg_fastmath.cuh)

// One grid instance, resident in a plan-owned device table.  Coefficients
// carry D/dx^2 and the stencil weights; the centre weight is folded into the
// model constants so that a cell's right-hand side is one FMA chain.
struct Inst {
    int32_t nx, ny;
    int32_t tiles_x, tiles_y;
    int32_t tile_begin;      // global tile id of this instance's first tile
    int32_t vec_ok;          // nx even and packed offset even: rows start 16-byte aligned
    int32_t tb_tiles_x;      // temporal blocking: tiles along x of this instance
    int32_t tb_tile_begin;   // temporal blocking: global index of its first tile
    int64_t off;             // element offset of the instance in packed state buffers
    int64_t ws_off;          // element offset of the instance's scratch block in the workspace
    double wx[MAXF], wy[MAXF], wd[MAXF], wc[MAXF];   // off-centre / centre stencil weights
    double wt[MAXF];         // wy / wd (0 where wd = 0): the 9-point stencil's row-sum form
    double mi[4];            // instance-dependent folds of centre weight and model constants
    const double *tab;       // plan-owned table 2^(j/4096), j = 0..4095 (exponentials)
};

// A warp's share of one stage under the static schedule: columns
// [x0, x0 + 32*CX) of rows y0..y1 of instance `inst`.  Row mrow_a only owns
// columns [ma0, ma1) and row mrow_b only [mb0, mb1) (the partial rows at the
// ends of a block's cell range); -1 disables a mask.
struct Seg {
    int32_t inst, x0, y0, y1;
    int32_t mrow_a, ma0, ma1;
    int32_t mrow_b, mb0, mb1;
};

// SCHED_TBLOCK: temporally blocked tiles (cg_tblock.cuh) for cg_run; the
// plan's other kernels keep the static schedule.
enum { SCHED_STATIC = 0, SCHED_QUEUE = 1, SCHED_TBLOCK = 2 };

// Kernel argument block (passed by value).
struct RunArgs {
    const Inst *inst;
    const Seg *segs;             // static schedule: segments of every warp
    const int32_t *warp_seg;     // warp w of the grid owns segs[warp_seg[w] .. warp_seg[w+1])
    int32_t sched;               // SCHED_STATIC or SCHED_QUEUE
    int32_t n_inst, n_tiles;
    int32_t bc, rows;            // ghost mode, rows per warp tile
    const double *z_in;
    double *z_out;
    const double *const *zin_tab;   // optional per-instance input/output pointers (plan order);
    double *const *zout_tab;        // when set they replace z_in + off and z_out + off
    double *ws;                  // base of the per-instance scratch blocks
    double *store;               // optional: keep every stage input (single instance; see Bufs)
    unsigned *flags;             // per-block count of finished stages (neighbour sync)
    const int2 *deps;            // blocks [deps[b].x, deps[b].y] own the halo of block b
    int32_t sync_mode;           // SYNC_GRID or SYNC_NEIGHBOR between stages
    int32_t pad_sync;
    unsigned *sync;              // [0..1] 64-bit grid-barrier arrival counter, [2..4] tile queues
    uint32_t *status;            // device status word (CG_DEV_*)
    int64_t g_begin, g_end;      // global stage range [g_begin, g_end) of this launch
    int32_t parity;              // step k stores its result in z_out iff (k + parity) is even
    int32_t persistent;          // 1: loop over stages with grid barriers; 0: one stage
    int32_t rhs_only;            // 1: write F(z) = D L z + N[z] itself to z_out (one-stage kernels)
    uint32_t nblocks_expect;     // arrivals the grid barrier waits for
    uint32_t stuck_barrier;      // testing knob: first barrier waits for one extra block
    uint64_t timeout_ns;         // bound on a barrier wait
    double cacc[4], cy[4];       // per-stage combine weights (b_s dt and a_{s+1,s} dt)
    double mp[NMP];              // model constants (layout per model, see cg_stepper.cuh)
};

// Scratch block of one instance (doubles): zb | acc | Ya | Yb, each n_v planes.
constexpr int SCRATCH_PLANES = 4;

// Workspace header (bytes): status word and sync counters.
constexpr size_t WS_HEADER = 8192;
constexpr size_t WS_STATUS_OFF = 0;
constexpr size_t WS_SYNC_OFF = 64;
constexpr int SYNC_WORDS = 8;
constexpr size_t WS_FLAGS_OFF = 512;                               // per-block stage counters
constexpr int MAX_FLAG_BLOCKS = (int)((WS_HEADER - WS_FLAGS_OFF) / 4);

enum { SYNC_GRID = 0, SYNC_NEIGHBOR = 1 };

// MODEL_BOCFH: the four-field model with its tanh terms replaced by smoothed
// steps (CG_FLAG_TANH_AS_HK); an internal kernel family, not an ABI model id.
enum { MODEL_FHN = CG_FHN, MODEL_BOCF = CG_BOCF, MODEL_KARMA = CG_KARMA, MODEL_DIFF = CG_DIFFUSION, MODEL_BOCFH = 5 };

// Kernel lookup, one function per model translation unit.  Returns nullptr
// for an unsupported combination.
const void *fwd_kernel_fhn(int stencil, int scheme, int cx);
const void *fwd_kernel_bocf(int stencil, int scheme, int cx);
const void *fwd_kernel_diff(int stencil, int scheme, int cx);
const void *fwd_kernel_bocfh(int stencil, int scheme, int cx);
const void *tb_kernel_fhn(int stencil, int scheme);
const void *tb_kernel_bocf(int stencil, int scheme);
const void *tb_kernel_diff(int stencil, int scheme);
const void *tb_kernel_bocfh(int stencil, int scheme);
const void *tlm_kernel_bocfh(int stencil, int scheme, int cx);
const void *adj_kernel_bocfh(int stencil, int scheme, int cx);
const void *tlm_kernel_fhn(int stencil, int scheme, int cx);
const void *tlm_kernel_bocf(int stencil, int scheme, int cx);
const void *tlm_kernel_diff(int stencil, int scheme, int cx);
const void *adj_kernel_fhn(int stencil, int scheme, int cx);
const void *adj_kernel_bocf(int stencil, int scheme, int cx);
const void *adj_kernel_diff(int stencil, int scheme, int cx);
const void *fwd_kernel_karma(int stencil, int scheme, int cx);
const void *tb_kernel_karma(int stencil, int scheme);
const void *tlm_kernel_karma(int stencil, int scheme, int cx);
const void *adj_kernel_karma(int stencil, int scheme, int cx);

// Host: the four-field model's s-gate rates 1/ts1 and 1/(ts1 + dts) as the
// kernels' own reciprocal computes them (out[0], out[1]); runs one tiny
// kernel on the current device and waits for it.
cudaError_t bocf_rcp_constants(double ts1, double dts, double *out);

// Host: fill tab[j] = 2^(j / n), j = 0..n-1, each rounded once to double
// from extended precision (the exponential's table).
void exp_table(double *tab, int n);

// Record a message for cg_last_error() on the calling thread; returns st.
cg_status set_last_error(cg_status st, const char *msg);

// A named NVTX range for the duration of one API call, so that a timeline
// profiler shows which library call issued which kernels (a few tens of
// nanoseconds per call when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace cgk
