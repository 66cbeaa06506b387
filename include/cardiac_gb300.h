/*
 * cardiac_gb300.h -- C ABI of the GB300 FP64 cardiac reaction-diffusion stepper.
 *
 * The library advances the two-dimensional reaction-diffusion system
 *
 *     dz/dt = div(D grad z) + N[z],    z = (u, gates)            Eq. (rdeqn), Sect. 2
 *
 * on an nx x ny grid with no-flux boundaries (Eq. BC:N) imposed by ghost
 * points that flip stencil displacements back into the grid (Sect. 3,
 * Fig. 1) or with periodic ghosts, a 5-point or 9-point Laplacian (Eq.
 * diffusion) and a fixed-step integrator (explicit Euler, Heun or classic
 * RK4, or Rush-Larsen / implicit Euler on the four-field model's gates,
 * Sect. 3), in FP64 throughout, on one NVIDIA GB300 (sm_103a).  Batches of
 * uneven grids, exact tangent-linear and adjoint runs, a Newton-Krylov step
 * and the right-hand side itself are exported too.  The problem statement
 * follows the paper's: model and its parameters, grid with dx and dy,
 * diffusivity D, time step dt, scheme, state in, state out, number of steps.
 *
 * Conventions for every entry point:
 *  - Every state is a caller-owned DEVICE buffer of float64 laid out
 *    [n_v][ny][nx] (field planes, row-major, x contiguous; no padding).
 *  - The caller owns the stream (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream) and the workspace (device memory of at least the
 *    size the matching *_workspace_size call returns, 256-byte aligned).
 *    The run path never allocates device memory.
 *  - Calls are asynchronous on the stream unless stated otherwise.  They can
 *    be captured into a CUDA graph (they issue only kernel launches,
 *    cudaMemsetAsync and device-to-device cudaMemcpyAsync).
 *  - Errors are returned as cg_status codes, never by abort or exception; a
 *    human-readable message for the calling thread is available from
 *    cg_last_error().  Errors detected on the device (non-finite output, a
 *    grid barrier that gave up waiting) are recorded in a status word inside
 *    the workspace and read back with cg_read_status().
 *  - A plan is immutable after creation and may be shared between threads
 *    and streams, provided each concurrent run has its own workspace.
 */
#ifndef CARDIAC_GB300_H
#define CARDIAC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CG_ABI_VERSION 1

/* Largest n_steps (period_steps) any entry point accepts; larger counts, and
 * workspace sizes that would not fit in 2^62 bytes, return CG_EINVAL. */
#define CG_MAX_STEPS ((int64_t)1 << 56)

typedef enum cg_status {
    CG_OK = 0,
    CG_EINVAL = 1,          /* invalid argument (message in cg_last_error) */
    CG_ENOMEM = 2,          /* host or plan-time device allocation failed */
    CG_ECUDA = 3,           /* a CUDA runtime call failed */
    CG_EUNSTABLE = 4,       /* dt above the scheme's linear diffusive stability bound */
    CG_ENAN = 5,            /* a non-finite value was written (device status) */
    CG_ETIMEOUT = 6,        /* a bounded device wait gave up (device status) */
    CG_EUNSUPPORTED = 7,    /* valid request this build does not implement */
    CG_EBOUNDS = 8          /* checked build: a device-side index check failed (device status) */
} cg_status;

/* Models (Sect. 2): FitzHugh-Nagumo (u, v both diffusive), Bueno-Orovio-
 * Cherry-Fenton (u, v, w, s; u diffusive), the two-variable Karma model of
 * Eq. (karma) (u, v; u diffusive with D_u = gamma).  CG_DIFFUSION is the
 * linear case N = 0 with one field, useful for checking the stencil and
 * integrators against closed forms. */
enum { CG_FHN = 0, CG_BOCF = 1, CG_KARMA = 2, CG_DIFFUSION = 3 };
/* Laplacian (Eq. diffusion): 5-point, or 9-point with diagonal weight alpha_d. */
enum { CG_STENCIL5 = 0, CG_STENCIL9 = 1 };
/* Ghost points (Fig. 1): MIRROR maps index -1 to 1 and n to n-2 (the
 * displacement is flipped back into the grid); CLAMP maps -1 to 0, n to n-1;
 * PERIODIC maps -1 to n-1 and n to 0 (opposite-edge values, Sect. 3).  Under
 * PERIODIC, CG_FLAG_NEIGHBOR_SYNC is ignored (the grid barrier is used). */
enum { CG_BC_MIRROR = 0, CG_BC_CLAMP = 1, CG_BC_PERIODIC = 2 };
/* Integrators of Sect. 3.  EULER, HEUN and RK4 are explicit for every field.
 * RUSH_LARSEN and IMPLICIT_EULER (Table 2) apply to the four-field model
 * only: u takes an explicit Euler step and each gate x = v, w, s, whose
 * equation is linear in x (dx/dt = al(u) x + be(u)), is advanced with al, be
 * taken at the step's starting state, by x_inf + (x - x_inf) e^(al dt) with
 * x_inf = -be/al (Rush-Larsen) or by (x + dt be)/(1 - dt al) (implicit
 * Euler).  They need positive time constants; the tangent-linear, adjoint
 * and Newton entry points return CG_EUNSUPPORTED for them. */
enum { CG_EULER = 0, CG_HEUN = 1, CG_RK4 = 2, CG_RUSH_LARSEN = 3, CG_IMPLICIT_EULER = 4 };

/* cg_problem.flags */
#define CG_FLAG_ALLOW_UNSTABLE   (1u << 0)  /* skip the dt stability check */
#define CG_FLAG_PER_STAGE_LAUNCH (1u << 1)  /* one kernel launch per RK stage instead of one
                                               persistent cooperative launch per run */
#define CG_FLAG_NEIGHBOR_SYNC    (1u << 2)  /* static schedule only: between stages each block
                                               waits for the blocks that own its halo instead of
                                               a grid-wide barrier (an autotuner option) */
#define CG_FLAG_TANH_AS_HK       (1u << 3)  /* four-field and Karma models: the model variant of
                                               Sect. 6, each (1 + tanh(kk x))/2 replaced by the
                                               smoothed step H_{kk/3}(x) (same value and slope at
                                               x = 0).  Changes the model, not only its cost. */
#define CG_FLAG_TEST_STUCK_BARRIER (1u << 8) /* testing only: the first wait between stages
                                               expects one arrival (or one stage) more than can
                                               happen, so it must give up after
                                               barrier_timeout_s and report CG_ETIMEOUT */

/* Device status bits (cg_read_status). */
#define CG_DEV_NONFINITE 1u   /* a non-finite value was stored */
#define CG_DEV_TIMEOUT   2u   /* a grid barrier wait gave up */
#define CG_DEV_BOUNDS    4u   /* checked build only: a stage worker found an index outside the
                                 grid (or its shared-memory window) before using it and skipped
                                 the access */

typedef struct cg_problem {
    int32_t abi_version;   /* must be CG_ABI_VERSION */
    int32_t model;         /* CG_FHN, CG_BOCF or CG_DIFFUSION */
    int64_t nx, ny;        /* grid size, each >= 2 (N x N in the paper) */
    double dx, dy;         /* grid spacing (dx = dy = 0.04 for FHN, 0.03 cm for BOCF) */
    double Dxx[4], Dyy[4]; /* per-field diagonal diffusion tensor; 0 = field not diffusive.
                              FHN: (1, delta = 1.5); BOCF: (1.171e-3 cm^2/ms, 0, 0, 0) */
    int32_t stencil;       /* CG_STENCIL5 / CG_STENCIL9 */
    int32_t bc;            /* CG_BC_MIRROR / CG_BC_CLAMP / CG_BC_PERIODIC */
    int32_t scheme;        /* CG_EULER / CG_HEUN / CG_RK4 / CG_RUSH_LARSEN / CG_IMPLICIT_EULER */
    uint32_t flags;        /* CG_FLAG_* */
    double alpha_d;        /* 9-point diagonal weight (axial weight 1 - 2 alpha_d); ignored for 5-point */
    double dt;             /* fixed time step */
    const double *params;  /* host array of cg_n_params(model) model constants, copied at plan
                              creation; NULL selects the defaults (cg_default_params) */
    int32_t n_params;      /* length of params (ignored when params is NULL) */
    int32_t reserved0;
    double barrier_timeout_s; /* bound on any device-side wait; <= 0 selects 10 s */
} cg_problem;

/* Optional launch shape (the autotuner's search space).  Zero fields take
 * the library's defaults. */
typedef struct cg_tuning {
    int32_t cells_x;       /* cells per lane along x: 1 or 2 (warp tile width 32 or 64) */
    int32_t rows;          /* rows per warp tile, >= 1 */
    int32_t threads;       /* threads per block: a multiple of 32 from 64 to 512 */
    int32_t blocks_per_sm; /* persistent blocks per SM, >= 1 (capped by occupancy) */
    int32_t schedule;      /* 0: static (equal cells per block, equal strip-rows per warp,
                              computed at plan creation); 1: atomic tile queue per stage
                              (tiles of 32*cells_x columns by `rows` rows, largest
                              instances first); 2: temporal blocking of cg_run and
                              cg_batch_run for small grids: the instances are cut into
                              tiles (one per block for a single instance; the blocks loop
                              over the tiles of a batch), each advanced with its halo
                              through `rows` steps (default 2) in shared memory per grid
                              barrier, with `threads` per block (default 256); MIRROR or
                              CLAMP ghosts, EULER/HEUN/RK4 only (else CG_EUNSUPPORTED), the
                              same results bit for bit; the plan's other entry points use
                              the default launch shape */
} cg_tuning;

typedef struct cg_plan_s *cg_plan;

/* ---------------------------------------------------------------- plans */

/* Validate a problem and build an immutable plan (coefficients, tile table,
 * launch shape).  Returns CG_EINVAL for a bad argument, CG_EUNSUPPORTED for a
 * gate integrator with a model other than CG_BOCF or CG_FLAG_TANH_AS_HK with
 * a model other than CG_BOCF and CG_KARMA, and
 * CG_EUNSTABLE when dt exceeds the linear bound 2/rho (Euler, Heun and the
 * u step of the gate integrators) or 2.785/rho (RK4), rho
 * the spectral radius of the diffusion operator, unless
 * CG_FLAG_ALLOW_UNSTABLE is set.  Allocates a small device table on the
 * current device; *out is NULL on error. */
cg_status cg_plan_create(const cg_problem *prob, cg_plan *out);

/* Same with an explicit launch shape (tuning may be NULL). */
cg_status cg_plan_create_tuned(const cg_problem *prob, const cg_tuning *tuning, cg_plan *out);

/* Build one plan for n_inst independent problems (uneven nx, ny and D
 * allowed; the same model, stencil, bc, scheme, dt, params and flags).  The
 * instances' states are packed back to back in one buffer: instance i starts
 * at element offset offsets[i] (cg_batch_offsets), each in the [n_v][ny][nx]
 * layout.  All instances advance together in one persistent launch. */
cg_status cg_batch_create(const cg_problem *probs, int32_t n_inst, const cg_tuning *tuning,
                          cg_plan *out);

/* Element offsets of the packed batch layout: offsets[0..n_inst], the last
 * entry being the total number of doubles.  A single-instance plan reports
 * {0, n_v*nx*ny}. */
cg_status cg_batch_offsets(cg_plan plan, int64_t *offsets);

/* Number of instances of a plan (1 for cg_plan_create). */
int32_t cg_plan_n_instances(cg_plan plan);

/* Release a plan and its device table.  NULL is accepted. */
cg_status cg_plan_destroy(cg_plan plan);

/* Bytes of device workspace that cg_run needs for this plan. */
cg_status cg_workspace_size(cg_plan plan, size_t *bytes);

/* ------------------------------------------------------------- stepping */

/* Advance the state(s) by n_steps >= 0 explicit steps (Sect. 3) of
 * dz/dt = D L z + N[z].  z_in and z_out are device buffers in the plan's
 * layout (packed for a batch); z_in == z_out is allowed, partial overlap is
 * not.  n_steps == 0 copies z_in to z_out.  Clears the device status word. */
cg_status cg_run(cg_plan plan, const double *z_in, double *z_out, int64_t n_steps,
                 void *workspace, void *stream);

/* cg_run for a batch plan whose instances live in separate caller buffers:
 * z_in and z_out are HOST arrays of cg_plan_n_instances(plan) DEVICE
 * pointers, entry i the state of instance i (user order) in the
 * [n_v][ny][nx] layout, 8-byte aligned.  z_in[i] == z_out[i] steps instance
 * i in place; otherwise its two buffers must not overlap (buffers of
 * different instances are not checked against each other and must not
 * overlap).  The pointer arrays are read during the call only (they are
 * written into the workspace by a kernel launch, so the call can be
 * captured into a CUDA graph, which then replays with these pointers).
 * Same workspace (cg_workspace_size), status word and results as cg_run on
 * the packed layout. */
cg_status cg_batch_run(cg_plan plan, const double *const *z_in, double *const *z_out, int64_t n_steps,
                       void *workspace, void *stream);

/* Same as cg_run, for callers that cannot allocate device memory when they
 * step: code running while a stream is captured into a CUDA graph (where
 * allocation is not allowed), programs whose device memory belongs to their
 * own pool allocator, and real-time loops that forbid allocation after
 * start-up.  The paper has no counterpart; this is a library convenience.
 * The scratch comes from one statically allocated 32 MiB device array inside
 * the library (every GPU that loads the library holds it until the process
 * exits) instead of a caller workspace, so the call allocates nothing.
 * Plans whose cg_workspace_size exceeds 32 MiB (e.g. a two-field 1024^2
 * grid) are rejected with CG_EINVAL and a message.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current: make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (each call
 * clears its status and synchronisation words itself), so calls that
 * overlap on the GPU race: issue them on one stream or otherwise serialise
 * them.  status_dev (device, may be NULL) receives the call's CG_DEV_* bits
 * once the run has finished on the stream.  Because every call's status
 * word lives in the shared array, cg_get_device_status on a plan whose
 * latest run went through this call reports the status of whichever
 * cg_run_noalloc call ran last on that device; use status_dev for the
 * status of one particular call. */
cg_status cg_run_noalloc(cg_plan plan, const double *z_in, double *z_out, int64_t n_steps,
                         uint32_t *status_dev, void *stream);

/* The right-hand side F(z) = D L z + N[z] of Eq. (rdeqn) (stencil, ghosts
 * and local terms exactly as the steps use them) for the plan's state z
 * (device, plan layout, packed for a batch) into f (device, same layout, not
 * overlapping z).  Asynchronous; clears the device status word, which
 * records non-finite values of f.  Valid for every scheme (it evaluates F,
 * no integrator).  Newton-Krylov solvers for periodic orbits need it for the
 * phase condition and the derivative of the flow map in the period. */
cg_status cg_rhs(cg_plan plan, const double *z, double *f, void *workspace, void *stream);

/* cg_run for a state held in HOST memory: copies z_in_host to the device,
 * advances it by n_steps exactly as cg_run does, copies the result to
 * z_out_host and waits for the stream.  z_in_host and z_out_host are host
 * buffers in the plan's layout (page-locked memory lets the copies run as
 * asynchronous DMA; pageable memory works too) and may be the same buffer.
 * The workspace (device, 256-byte aligned) must hold cg_host_workspace_size
 * bytes: the cg_run workspace followed by two device copies of the state.
 * Returns after the result is in z_out_host, with CG_ENAN / CG_ETIMEOUT if
 * the run recorded a device error (as cg_read_status).  The paper's own
 * host loop (Matlab driving OpenCL, Sect. 3) moves the state the same way
 * around each call. */
cg_status cg_host_workspace_size(cg_plan plan, size_t *bytes);
cg_status cg_run_host(cg_plan plan, const double *z_in_host, double *z_out_host, int64_t n_steps,
                      void *workspace, void *stream);

/* Synchronise the stream and return the device status bits (CG_DEV_*)
 * recorded by the last run that used this workspace.  Returns CG_EBOUNDS,
 * CG_ETIMEOUT or CG_ENAN when the matching bit is set (in that order of
 * precedence), CG_OK otherwise. */
cg_status cg_read_status(cg_plan plan, const void *workspace, void *stream, uint32_t *flags);

/* The same for the latest run issued with this plan (cg_run, cg_batch_run,
 * cg_rhs, the tangent-linear, adjoint and Newton calls): the plan records the
 * workspace and stream of each run it issues.  flags = 0 and CG_OK when the
 * plan has not run yet.  The workspace of that run must still be allocated.
 * With one plan used on several streams at once, the latest issue wins; use
 * cg_read_status with an explicit workspace there. */
cg_status cg_get_device_status(cg_plan plan, uint32_t *flags);

/* ------------------------------------------------- tangent-linear model */

/* The paper's motivation (Sect. 1) is matrix-free Newton-Krylov solvers that
 * need the Jacobian of finite-time flows, which it obtains by finite
 * differences of nearby double-precision solutions.  These calls give the
 * exact Jacobian-vector products of the discrete flow instead: each RK
 * stage Y_s of the primal run is differentiated, dk_s = D L dY_s +
 * dN/dz(Y_s) dY_s, dY_s = dz + dt a_s dk_{s-1}, dz' = dz + dt sum b_s dk_s. */

/* Bytes of workspace cg_tlm_run needs for n_tangents tangents (single-
 * instance plans only; CG_EUNSUPPORTED for a batch plan). */
cg_status cg_tlm_workspace_size(cg_plan plan, int32_t n_tangents, size_t *bytes);

/* Advance the primal state z0 -> zT and n_tangents >= 0 tangents dz0 -> dzT
 * (device buffers; tangents packed [n_tangents][n_v][ny][nx]) by n_steps
 * explicit steps: dzT[i] = (d Phi / d z)(z0) dz0[i] with Phi the n-step
 * discrete flow map.  All tangents share the primal trajectory, advanced
 * once.  In-place (zT == z0, dzT == dz0) is allowed for Heun and RK4. */
cg_status cg_tlm_run(cg_plan plan, const double *z0, const double *dz0, double *zT, double *dzT,
                     int32_t n_tangents, int64_t n_steps, void *workspace, void *stream);

/* Linearized tangent-linear runs, for many Jacobian-vector products at one
 * base point z0 (the Krylov iterations of a Newton step).  cg_tlm_linearize
 * advances z0 -> zT (the same values as cg_run) and keeps the local Jacobian
 * dN/dz of every RK stage in the workspace; cg_tlm_apply then advances
 * n_tangents tangents dz0 -> dzT through the same n_steps with those
 * Jacobians and no primal work, giving bit for bit the dzT of cg_tlm_run
 * from the same z0.  The workspace (size from
 * cg_tlm_linearized_workspace_size for the largest n_tangents to apply, and
 * the same n_steps) holds n_steps * n_stages stored Jacobians of
 * round32(NJ nx ny) doubles each (NJ = 1 FHN and diffusion, 10 BOCF) and
 * must not be touched between the two calls; the plan, n_steps and the
 * workspace pointer must be the same in both.  Layouts and in-place rules as
 * cg_tlm_run.  CG_EINVAL for NULL buffers, negative counts, a misaligned
 * workspace, partial overlap, or (cg_tlm_apply) a workspace that the plan
 * did not linearize over the same n_steps (the plan remembers its latest 16
 * linearized workspaces); CG_EUNSUPPORTED for batch plans and the gate
 * integrators. */
cg_status cg_tlm_linearized_workspace_size(cg_plan plan, int32_t n_tangents, int64_t n_steps, size_t *bytes);
cg_status cg_tlm_linearize(cg_plan plan, const double *z0, double *zT, int64_t n_steps, void *workspace,
                           void *stream);
cg_status cg_tlm_apply(cg_plan plan, const double *dz0, double *dzT, int32_t n_tangents, int64_t n_steps,
                       void *workspace, void *stream);

/* ------------------------------------------------------ discrete adjoint */

/* Bytes of workspace cg_adjoint_run needs (single-instance plans): the
 * primal scratch, ceil(n_steps / c) checkpoints, the c*n_stages + 1 stage
 * inputs of one segment, four adjoint states and one partial sum per warp,
 * c = checkpoint_every (0 selects ceil(sqrt(n_steps))). */
cg_status cg_adjoint_workspace_size(cg_plan plan, int64_t n_steps, int32_t checkpoint_every, size_t *bytes);

/* Reverse-mode derivative of the n-step discrete flow map z0 -> zT (the
 * transpose of the Jacobian that cg_tlm_run applies).  Given lamT = dL/dzT
 * (device, [n_v][ny][nx]) it writes lam0 = dL/dz0 (device, may equal lamT)
 * and, for each diffusive field f, dLdD[f] = dL/dD_f (device, n_diffusive
 * doubles: 2 for FHN, 1 otherwise), where field f's tensor is
 * D_f diag(1, Dyy_f/Dxx_f) with the anisotropy ratio held fixed.
 *
 * The forward trajectory is rebuilt from checkpoints: one forward sweep
 * stores z every c steps; then, segment by segment in reverse, the segment
 * is recomputed keeping every RK stage input and swept back with the
 * adjoint stage kernel (transposed stencil W L W^-1 under MIRROR ghosts,
 * transposed local Jacobian).  Cost: two forward runs plus one adjoint run.
 * dL/dD partial sums are reduced in a fixed order (bitwise reproducible).
 * dLdD may be NULL: the run then skips the dL/dD dot products and their
 * reduction (state-only gradients) and writes the same lam0 bit for bit. */
cg_status cg_adjoint_run(cg_plan plan, const double *z0, const double *lamT, double *lam0, double *dLdD,
                         int64_t n_steps, int32_t checkpoint_every, void *workspace, void *stream);

/* The same gradient split at the end of the forward run, for callers that
 * run z0 -> zT first and want the gradient later (a training step: the
 * forward pass needs zT anyway, so it can leave the checkpoints behind and
 * the backward pass skips cg_adjoint_run's own forward sweep: one forward
 * run plus one adjoint run instead of two plus one).
 *
 * cg_adjoint_checkpoint_size: bytes of the checkpoint buffer,
 * ceil(n_steps / c) states of round32(n_v nx ny) doubles (c as in
 * cg_adjoint_run).
 *
 * cg_adjoint_forward advances z0 -> zT (device, plan layout, not
 * overlapping each other partially nor the buffer) bit for bit as cg_run
 * does, and keeps z0 and every c-th state in `checkpoints` (device,
 * 256-byte aligned, caller-owned); workspace: cg_workspace_size bytes.
 *
 * cg_adjoint_reverse then writes lam0 (not overlapping the buffer) and
 * dLdD (NULL allowed) for lamT exactly as cg_adjoint_run(plan, z0, lamT,
 * ...) would, bit for bit, from those checkpoints: same plan, n_steps and checkpoint_every, the buffer
 * untouched in between (it is only read, so one forward serves several
 * reverse calls); workspace: cg_adjoint_workspace_size bytes.  The plan
 * remembers the buffers of its latest 16 cg_adjoint_forward calls with
 * their n_steps and c: CG_EINVAL for any other buffer or count.  Other
 * errors as cg_adjoint_run. */
cg_status cg_adjoint_checkpoint_size(cg_plan plan, int64_t n_steps, int32_t checkpoint_every, size_t *bytes);
cg_status cg_adjoint_forward(cg_plan plan, const double *z0, double *zT, int64_t n_steps, int32_t checkpoint_every,
                             double *checkpoints, void *workspace, void *stream);
cg_status cg_adjoint_reverse(cg_plan plan, const double *checkpoints, const double *lamT, double *lam0,
                             double *dLdD, int64_t n_steps, int32_t checkpoint_every, void *workspace,
                             void *stream);

/* ------------------------------------------------- Newton-Krylov step */

/* Sect. 1 names matrix-free Newton-Krylov solvers (e.g. for periodic orbits
 * of the flow) as the reason double precision is needed.  One Newton step on
 * the period-T flow map Phi_T solves
 *     (J_T - I) dz = -(Phi_T(z0) - z0),   J_T = d Phi_T / d z (z0)
 * by restarted GMRES(restart) with modified Gram-Schmidt, J_T v from
 * cg_tlm_run (exact, not finite differences).  All vector work runs on the
 * device with fixed-order reductions; the (restart+1) x restart Hessenberg
 * least-squares problem is solved on the host with Givens rotations.
 * Stops when the residual drops below rtol * |b| or after max_restarts
 * cycles.  dz: device output (plan layout).  res_hist: optional host array
 * of restart*max_restarts + 1 residual norms (entry 0 = |b|).  n_iter:
 * optional host output, Arnoldi steps taken.  Synchronous on the stream
 * (it reads dot products back).  Single-instance plans only. */
cg_status cg_newton_workspace_size(cg_plan plan, int32_t restart, size_t *bytes);
cg_status cg_newton_gmres_step(cg_plan plan, const double *z0, int64_t period_steps, int32_t restart,
                               int32_t max_restarts, double rtol, double *dz, double *res_hist,
                               int32_t *n_iter, void *workspace, void *stream);

/* The same Newton step with J_T v from cg_tlm_apply after one
 * cg_tlm_linearize at z0: each Krylov iteration skips the primal run, at the
 * cost of storing period_steps * n_stages stage Jacobians (workspace from
 * cg_newton_linearized_workspace_size).  Results equal cg_newton_gmres_step's
 * bit for bit. */
cg_status cg_newton_linearized_workspace_size(cg_plan plan, int32_t restart, int64_t period_steps, size_t *bytes);
cg_status cg_newton_gmres_step_linearized(cg_plan plan, const double *z0, int64_t period_steps, int32_t restart,
                                          int32_t max_restarts, double rtol, double *dz, double *res_hist,
                                          int32_t *n_iter, void *workspace, void *stream);

/* Deterministic vector kernels used by the Newton-Krylov step.
 * cg_dot: *result (device) = sum_i x[i] y[i], summed in a fixed order; the
 * workspace needs 256 doubles.  cg_axpby: y = a x + b y (device vectors). */
cg_status cg_dot(const double *x, const double *y, int64_t n, double *result, void *workspace, void *stream);
cg_status cg_axpby(double a, const double *x, double b, double *y, int64_t n, void *stream);

/* ----------------------------------------------------------------- misc */

/* Message describing the last error on the calling thread ("" if none). */
const char *cg_last_error(void);

/* Number of fields n_v of a model (2 FHN, 4 BOCF, 2 Karma, 1 diffusion), -1
 * if unknown. */
int32_t cg_n_fields(int32_t model);

/* Number of model constants (3 FHN: eps, a1, a0; 29 BOCF; 8 Karma: tau_u,
 * tau_v, u*, u_h, u_v, Re, M, k; 0 diffusion).  Karma: tau_u, tau_v and Re
 * must be non-zero; an integer M in [0, 64] takes v^M by repeated squaring,
 * any other M by pow(). */
int32_t cg_n_params(int32_t model);

/* Write the default constants of a model to out[0 .. cg_n_params(model)-1]
 * (host memory).  FHN: Sect. 2 values; BOCF: the epicardial set of the
 * model the paper cites, then k = 28.4 for H_k; Karma: (Re, M) = (1, 6) and
 * k = 28.4 of Sect. 2 with tau_u = 2.5, tau_v = 250, u* = 1.5415, u_h = 3,
 * u_v = 1 of the model paper it cites (gamma = 0.0011 cm^2/ms is D_u). */
cg_status cg_default_params(int32_t model, double *out);

/* Host-only preview of the static schedule that plans use (no device
 * needed): the cells of instances 0..n_inst-1 (in the given order, row-major
 * inside each) are split into n_blocks equal ranges and each range into
 * warps_per_block pieces of equal strip-rows, strips being 32*cells_x
 * columns wide.  Writes *n_segs segments of 10 int32 each to segs_out (when
 * not NULL and segs_cap allows): {inst, x0, y0, y1, mrow_a, ma0, ma1,
 * mrow_b, mb0, mb1}, meaning columns [x0, x0 + 32*cells_x) of rows y0..y1,
 * except that row mrow_a keeps only columns [ma0, ma1) and row mrow_b only
 * [mb0, mb1); and n_blocks*warps_per_block + 1 prefix offsets to
 * warp_seg_out (warp w owns segments [warp_seg_out[w], warp_seg_out[w+1])).
 * deps_out (optional, 2*n_blocks int32): for each block the first and last
 * block whose cells lie within one row and one column of its own (the
 * blocks it waits for between stages). */
cg_status cg_static_schedule(const int32_t *nx, const int32_t *ny, int32_t n_inst, int32_t cells_x,
                             int32_t n_blocks, int32_t warps_per_block, int32_t *segs_out,
                             int64_t segs_cap, int32_t *warp_seg_out, int64_t *n_segs, int32_t *deps_out);

/* Host-only preview of the schedule the adjoint's reverse stages use on a
 * single-instance plan with mirror ghosts and grid barriers (other plans'
 * adjoints use cg_static_schedule's): the same segments and warp split, but
 * the n_blocks cell ranges have equal COST, a cell on the scaled boundary
 * path (rows 0, 1, ny-2, ny-1 and the column strips starting at column <= 1
 * or reaching column nx-2) counting 1.4.  Outputs as cg_static_schedule. */
cg_status cg_adjoint_schedule(int32_t nx, int32_t ny, int32_t cells_x, int32_t n_blocks, int32_t warps_per_block,
                              int32_t *segs_out, int64_t segs_cap, int32_t *warp_seg_out, int64_t *n_segs);

/* CG_ABI_VERSION of the loaded library. */
int32_t cg_abi_version(void);

/* 1 for the checked build (libcardiac_gb300_checked.so, compiled with
 * CG_BOUNDS_CHECK): every stage worker of the forward, tangent-linear,
 * adjoint and temporally blocked kernels checks the grid and window indices
 * it is about to use, skips an access that would leave them and reports
 * CG_DEV_BOUNDS; results are otherwise bit for bit those of the plain build.
 * 0 for the plain build. */
int32_t cg_bounds_checked(void);

#ifdef __cplusplus
}
#endif

#endif /* CARDIAC_GB300_H */
