/*
 * swof.h -- C ABI of libswof, a GB300 (sm_103a) implementation of the time
 * step of FullSWOF_2D's well-balanced finite-volume shallow-water solver
 * (arXiv 1307.4839, "FullSWOF_Paral", Sec. 2-3 and Algorithm 1).
 *
 * The problem (Sec. 2.1, Eq. (SW2D)): unknowns h [m], qx = hu, qy = hv
 * [m^2/s] on an nx x ny Cartesian grid of cells dx x dy, fixed topography z,
 * rain R(t), Green-Ampt infiltration I (Sec. 3.5), the friction laws of
 * Sec. 2.1, ghost-cell boundary conditions (Sec. 2.2).  One step
 * (Algorithm 1) is two Heun stages (Sec. 3.2), each: boundary conditions ->
 * MUSCL-minmod reconstruction (Sec. 3.4) -> hydrostatic reconstruction ->
 * HLL flux (Sec. 3.3) -> scheme Eq. (SW1Dscheme) in x and y -> semi-implicit
 * friction (Sec. 3.2); then the Heun average, rain and infiltration, with dt
 * from the CFL condition Eq. (cfl) on the MUSCL face values.  The
 * first-order variant (Sec. 3.3) drops the reconstruction and takes one
 * explicit Euler stage per step.
 *
 * Conventions (all entry points):
 *   - Return SWOF_OK (0) or a negative SWOF_E* code; nothing throws or exits.
 *   - Host arrays are row-major [ny][nx] float64, x fastest; they are copied,
 *     the caller keeps ownership.  Output arrays are caller-allocated.
 *   - A context owns all of its device memory; it is bound to the CUDA
 *     device current at swof_create and to one stream (params.stream, or an
 *     internal stream when NULL).  A context is not thread-safe.
 *   - Work is enqueued asynchronously; swof_get_* synchronise the stream.
 *   - Errors raised on the device (non-finite state, exhausted dt
 *     sequence, CFL violation in fixed-dt mode) are latched in the context:
 *     later steps become no-ops and the code is returned by the next call
 *     that synchronises (swof_step with info != NULL, swof_get_*).
 */
#ifndef SWOF_H
#define SWOF_H

#if defined(__GNUC__)
#define SWOF_API __attribute__((visibility("default")))
#else
#define SWOF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SWOF_OK            0
#define SWOF_EINVAL       -1   /* bad argument (NULL, size, enum, layout) */
#define SWOF_ENOMEM       -2   /* device allocation failed */
#define SWOF_ECUDA        -3   /* a CUDA runtime call failed */
#define SWOF_ENONFINITE   -4   /* NaN/Inf in the state or in the wave speeds */
#define SWOF_ENEGATIVE    -5   /* negative water depth in a state passed in */
#define SWOF_ECFL         -6   /* fixed dt larger than the CFL bound Eq. (cfl) */
#define SWOF_EDTSEQ       -7   /* replayed dt sequence exhausted */
#define SWOF_ETIMEOUT     -8   /* a bounded device wait ran out */
#define SWOF_EDTUNDERFLOW -9   /* CFL dt below params.dt_min */
#define SWOF_ESTATE      -10   /* call not valid in the context's state */
#define SWOF_EBOUNDS     -11   /* debug build: a kernel index check failed (the access was clamped) */

/* ---- enums ---- */
#define SWOF_FP64 0            /* all arithmetic in FP64 (parity path) */
#define SWOF_FP32 1            /* bulk FP32 stencil; FP64 dt, time, budgets */
#define SWOF_CFL_SUM 0         /* dt = n_CFL / (lx/dx + ly/dy) */
#define SWOF_CFL_MIN 1         /* dt = n_CFL * min(dx/lx, dy/ly) */
#define SWOF_BC_WALL 0         /* mirror ghosts, normal discharge negated */
#define SWOF_BC_OUTFLOW 1      /* free outflow: edge cell extended */
/* Imposed edges (Sec. 2.2): both ghost layers hold one boundary state made
 * from the edge cell.  The Riemann invariant w - 2 sqrt(g h) that leaves the
 * domain (w = normal velocity, positive inwards) is kept and the imposed
 * value replaces the entering one (fluvial edges); a torrential inflow
 * imposes both.  The tangential velocity is the edge cell's (H, Q) or zero
 * (HQ).  No switching by flow regime: the caller picks the type.  The
 * boundary state also enters the CFL speed. */
#define SWOF_BC_IMPOSED_H 2    /* depth bc_h imposed */
#define SWOF_BC_IMPOSED_Q 3    /* discharge per unit width bc_q >= 0 imposed (inflow) */
#define SWOF_BC_IMPOSED_HQ 4   /* both imposed (supercritical inflow) */
/* Friction laws (Sec. 2.1), S_f = C_f |u| u / h^p, semi-implicit (Sec. 3.2):
 * q = q* / (1 + dt g C_f |u^s| / (h*)^p), u^s the stage input's velocity. */
#define SWOF_FRIC_NONE 0
#define SWOF_FRIC_MANNING 1    /* C_f = n^2, p = 4/3 */
#define SWOF_FRIC_STRICKLER 2  /* C_f = 1/K^2, p = 4/3 */
#define SWOF_FRIC_DARCY 3      /* Darcy-Weisbach, C_f = f/(8g), p = 1 */
#define SWOF_FRIC_CHEZY 4      /* C_f = 1/C^2, p = 1 */
#define SWOF_ORDER_2 0         /* MUSCL + Heun (n_CFL 0.5 in the paper); 2 means the same */
#define SWOF_ORDER_1 1         /* no reconstruction, one Euler stage (n_CFL 1 in the paper) */

typedef struct swof_ctx swof_ctx;

typedef struct swof_params {
    double g;              /* gravity, 9.81 (Sec. 2.1) */
    double cfl;            /* n_CFL, 0.5 at second order (Sec. 3.3) */
    double h_dry;          /* dry threshold [m]: u = v = 0 and q := 0 below */
    double dt_max;         /* dt cap; dt when every wave speed is zero */
    double dt_min;         /* CFL dt below this -> SWOF_EDTUNDERFLOW (0: off) */
    double t_end;          /* the last step is clamped to end here */
    int precision;         /* SWOF_FP64 | SWOF_FP32 */
    int cfl_mode;          /* SWOF_CFL_SUM | SWOF_CFL_MIN */
    int bc[4];             /* W, E, S, N edges: SWOF_BC_* */
    int friction;          /* SWOF_FRIC_* */
    double friction_coef;  /* the law's coefficient (n, K, f or C) when friction_map is NULL */
    const double *friction_map;  /* per-cell coefficient [ny][nx], host, copied; nullable */
    double rain_rate;      /* uniform rain R [m/s] (Eq. (SW2D)) */
    double rain_t_on, rain_t_off;  /* rain falls for t in [on, off) */
    int infiltration;      /* 1: Green-Ampt (Sec. 3.5) */
    double ks;             /* K_s [m/s] when ks_map is NULL */
    const double *ks_map;  /* per-cell K_s [ny][nx], host, copied; nullable */
    double psi;            /* wetting-front suction head h_f [m], > 0 */
    double dtheta;         /* theta_s - theta_i */
    int check_cfl;         /* 1: count steps whose dt breaks Eq. (cfl) at U* */
    double dt_fixed;       /* > 0: fixed dt (Eq. (cfl) violation -> SWOF_ECFL) */
    void *stream;          /* cudaStream_t to enqueue on; NULL: an internal
                              non-blocking stream (the legacy default stream
                              is handle 0, so it cannot be selected here) */
    int order;             /* SWOF_ORDER_2 (default) | SWOF_ORDER_1 */
    double bc_h[4];        /* imposed depth per edge [m] (SWOF_BC_IMPOSED_H, _HQ) */
    double bc_q[4];        /* imposed discharge per unit width into the domain
                              [m^2/s] (SWOF_BC_IMPOSED_Q, _HQ) */
} swof_params;

typedef struct swof_step_info {
    double t;              /* simulated time after the call */
    double dt;             /* last dt */
    long long steps;       /* steps taken since creation */
    int status;            /* latched device status (SWOF_OK or SWOF_E*) */
} swof_step_info;

typedef struct swof_diag {
    double t, last_dt;
    long long steps;
    double volume;         /* sum h dx dy, deterministic fixed-order tree */
    double rain_in;        /* rain volume added [m^3] */
    double infiltrated;    /* volume infiltrated [m^3] */
    double outflow;        /* net volume out through the edges [m^3] */
    double min_h;          /* smallest interior depth */
    long long cfl_viol;    /* steps with dt above the CFL bound at U* */
} swof_diag;

/* Fill *p with the defaults: g 9.81, cfl 0.5, h_dry 1e-6, dt_max 0.1,
 * dt_min 0, t_end 1e30, FP64, CFL_SUM, second order, walls, no
 * friction/rain/infiltration. */
SWOF_API void swof_default_params(swof_params *p);

/* Create a solver for an nx x ny grid (nx, ny >= 2) of cells dx x dy with
 * topography z [ny][nx] (host, copied; ghost z by the boundary rule).
 * Allocates every device buffer (padded SoA, 2 ghost layers); the state
 * starts dry (h = q = 0) at t = 0.  Sec. 2.1 / Sec. 6.1 (2 ghost layers at
 * second order).  Errors: SWOF_EINVAL, SWOF_ENOMEM, SWOF_ECUDA. */
SWOF_API int swof_create(int nx, int ny, double dx, double dy, const double *z,
                const swof_params *p, swof_ctx **out);

/* Destroy a context and free its device memory; NULL-safe.  Synchronises. */
SWOF_API void swof_destroy(swof_ctx *ctx);

/* Set the conservative state (h, hu, hv), host [ny][nx] float64, copied and
 * converted to the context precision; ghosts are refilled.  Rejects NaN/Inf
 * (SWOF_ENONFINITE) and h < 0 (SWOF_ENEGATIVE) before touching the state.
 * The arrays are copied to a device staging buffer (3 nx ny doubles,
 * allocated on the first host exchange and kept) and checked there; pinned
 * host memory makes the copy a direct DMA.  Synchronises. */
SWOF_API int swof_set_state(swof_ctx *ctx, const double *h, const double *hu, const double *hv);

/* Copy the state to host arrays [ny][nx] float64 (FP32 values widened,
 * through the same device staging buffer).  Synchronises; returns a latched
 * device status if one is set. */
SWOF_API int swof_get_state(swof_ctx *ctx, double *h, double *hu, double *hv);

/* Same with device pointers of dense [ny][nx] arrays of the given dtype
 * (SWOF_FP64: double, SWOF_FP32: float), e.g. torch tensors' data_ptr();
 * enqueued on the context stream.  Values are converted when the dtype
 * differs from the context precision.  No validation of the values. */
SWOF_API int swof_set_state_device(swof_ctx *ctx, const void *h, const void *hu, const void *hv, int dtype);
SWOF_API int swof_get_state_device(swof_ctx *ctx, void *h, void *hu, void *hv, int dtype);

/* Infiltrated depth V_inf (Sec. 3.5), host [ny][nx] float64. */
SWOF_API int swof_get_infiltrated(swof_ctx *ctx, double *vinf);
SWOF_API int swof_set_infiltrated(swof_ctx *ctx, const double *vinf);

/* V_inf from / to a dense device array [ny][nx] of dtype (SWOF_FP64 or
 * SWOF_FP32), enqueued on the context stream; no validation of values. */
SWOF_API int swof_set_infiltrated_device(swof_ctx *ctx, const void *vinf, int dtype);
SWOF_API int swof_get_infiltrated_device(swof_ctx *ctx, void *vinf, int dtype);

/* Simulated time (FP64), enqueued on the context stream (ordered before
 * later steps); resets nothing else. */
SWOF_API int swof_set_time(swof_ctx *ctx, double t);

/* Advance n full steps (Algorithm 1: two Heun stages; one Euler stage at
 * first order), each with one dt from Eq. (cfl)
 * (or the replayed sequence, or dt_fixed).  Asynchronous when info is NULL;
 * with info non-NULL the call synchronises and reports t, dt, steps and the
 * latched status (also the return value). n = 0 is allowed. */
SWOF_API int swof_step(swof_ctx *ctx, int n, swof_step_info *info);

/* Replay the given dt values (host, copied) for the next n steps instead of
 * Eq. (cfl), e.g. the oracle's sequence for parity.  n = 0 switches replay
 * off.  Running past the end latches SWOF_EDTSEQ.  Errors: SWOF_EINVAL,
 * SWOF_ENONFINITE (a value is not finite), SWOF_ENOMEM, SWOF_ECUDA; a call
 * that fails leaves the previous replay (or none) in place. */
SWOF_API int swof_set_dt_sequence(swof_ctx *ctx, const double *dts, int n);

/* dt of each step taken so far (up to max values, oldest first) into host
 * out; *count gets how many were written.  Synchronises. */
SWOF_API int swof_get_dt_history(swof_ctx *ctx, double *out, int max, int *count);

/* Diagnostics (volume by a deterministic reduction, budgets, min h).
 * Synchronises. */
SWOF_API int swof_get_diagnostics(swof_ctx *ctx, swof_diag *d);

/* Water volume sum(h) dx dy and minimum depth of a caller-owned depth
 * field, computed without allocating any device memory.  The paper has no
 * counterpart: this is a service for callers that may not call cudaMalloc
 * (hosts whose device memory all belongs to their own pool allocator, where
 * an allocation behind the pool's back could fail or fragment it; real-time
 * loops where an allocation is not allowed because it can synchronise the
 * device).
 *   h      : device pointer, dense row-major [ny][nx] of dtype (SWOF_FP64
 *            double or SWOF_FP32 float) on the current device; caller-owned.
 *   out    : device pointer to 2 doubles, caller-owned: out[0] = volume
 *            [m^3], out[1] = min h (NaN if h holds a NaN).
 *   stream : cudaStream_t to enqueue on (NULL = the default stream); the
 *            call is asynchronous and returns once the kernels are queued.
 * Scratch is one fixed file-scope device array of 2 * SWOF_NOALLOC_MAX_ROWS
 * doubles (1 MiB), held by every GPU that loads the library until the
 * process exits; ny > SWOF_NOALLOC_MAX_ROWS is rejected with SWOF_EINVAL.
 * The first call on a device looks up that array's device address and loads
 * this entry point's kernels (once per device), so make the first call on
 * each device before any stream capture.
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller.  The sum is a fixed-order reduction (per row,
 * then over rows), so repeated calls on the same data agree bit for bit.
 * Errors: SWOF_EINVAL (NULL, size, dtype), SWOF_ECUDA (a launch failed; or
 * a CUDA error was already pending on the calling thread: then nothing is
 * launched and that error is left for the caller to read). */
#define SWOF_NOALLOC_MAX_ROWS 65536
SWOF_API int swof_volume_noalloc(const void *h, int nx, int ny, int dtype, double dx, double dy,
                                 double *out, void *stream);

/* ---- outputs along the run ---------------------------------------------
 * Maximum water depth (flood extent): swof_track_max_depth(ctx, 1) starts a
 * running maximum from the current depth, updated after every later step by
 * one small pass (launched only while tracking); 0 stops it and frees it.  swof_get_max_depth
 * copies it to a host array [ny][nx] (float64); the maximum water level is
 * that plus z.  Synchronises.  Errors: SWOF_ESTATE when not tracking. */
SWOF_API int swof_track_max_depth(swof_ctx *ctx, int on);
SWOF_API int swof_get_max_depth(swof_ctx *ctx, double *hmax);

/* Gauges: record, after every step, t and (h, hu, hv) at n cells given as
 * (i, j) pairs in cells[2n] (host, copied), up to `capacity` records (later
 * steps are not recorded).  Replaces earlier gauges; n = 0 switches them
 * off.  swof_get_gauges copies up to max_records records of 1 + 3n doubles
 * (t, then h, hu, hv per gauge) to host out and the number recorded to
 * *count.  Synchronises.  Errors: SWOF_EINVAL (cell outside the grid; the
 * earlier gauges stay), SWOF_ENOMEM / SWOF_ECUDA (gauges end up off). */
SWOF_API int swof_set_gauges(swof_ctx *ctx, const int *cells, int n, int capacity);
SWOF_API int swof_get_gauges(swof_ctx *ctx, double *out, int max_records, int *count);

/* Dry-tile skipping (second order only): a stage tile whose cells and those
 * of its 8 neighbour tiles all hold h = 0 exactly, with no rain falling and
 * no imposed edge beside it, keeps U^{n+1} = U^n (every flux of the step is
 * zero there), so both stage kernels leave it after one flag test.  The
 * results are bit for bit those of the full step.  Switching it on selects
 * the shallowest tile shape (64 threads x 16 rows) for both stages: a sparse
 * wet region then spreads over many short column walks (a later
 * swof_set_tile_shape(s) may pick another; both stages keep one shape).
 * Every state change marks all tiles wet again.
 * swof_get_tile_activity reports the tiles processed and the tiles offered
 * since the last swof_set_dry_tile_skip(ctx, 1).  Synchronises.  Not in the
 * paper: an activity mask over the GPU tiles. */
SWOF_API int swof_set_dry_tile_skip(swof_ctx *ctx, int on);
SWOF_API int swof_get_tile_activity(swof_ctx *ctx, long long *live_tiles, long long *tiles);

/* D8 flow direction of a DEM (Sec. 5.2, the eight-neighbour example): for
 * each cell the neighbour of smallest elevation among those strictly below
 * it, as code 1..8 = E, NE, N, NW, W, SW, S, SE (counter-clockwise from +x,
 * row j + 1 north of row j), 0 when none is lower; ties go to the first
 * code.  Neighbours outside the grid are no candidates, nor those with
 * z <= *nodata when nodata (a host pointer) is not NULL (0: the
 * non-positive no-data convention).  NaN never compares lower.  z: device
 * float [ny][nx]; dir: device uint8 [ny][nx]; both caller-owned, enqueued
 * on stream.  Errors: SWOF_EINVAL. */
SWOF_API int swof_flow_directions(const float *z, int nx, int ny, const float *nodata, unsigned char *dir,
                                  void *stream);

/* Device time of the last swof_step call's kernels, split per kernel
 * family (wave-speed/dt, stage 1, stage 2) in milliseconds, when timing was
 * switched on with swof_enable_timing(ctx, 1).  Synchronises. */
SWOF_API int swof_enable_timing(swof_ctx *ctx, int on);
SWOF_API int swof_get_timing(swof_ctx *ctx, double *ms_lambda, double *ms_stage1, double *ms_stage2, int *launches);

/* Capture the next n-step sequence into a CUDA graph and replay it on later
 * swof_step calls with the same n (0 switches graphs off). Launch-bound
 * small grids gain the most. */
SWOF_API int swof_use_graph(swof_ctx *ctx, int on);

/* FP64 multiply-add contraction (SWOF_FP64 contexts; SWOF_EINVAL for
 * SWOF_FP32).  Off (the default), every FP64 kernel follows the oracle's
 * operation order with no a*b+c contracted, so states and the dt sequence
 * equal the oracle's bit for bit.  On, the same kernels compiled with
 * contraction run instead (~15 % faster on GB300's FP64 pipe): each fused
 * multiply-add rounds once instead of twice, so results differ from the
 * oracle by roundoff -- within relative L-inf 1e-12 under the oracle's dt
 * sequence -- and the CFL dt may differ in its last bits.  Takes effect
 * from the next swof_step; synchronises; a captured step graph is
 * re-captured.  Not in the paper: a GB300 build choice.  The ensemble
 * kernel always runs without contraction. */
SWOF_API int swof_set_fp64_contraction(swof_ctx *ctx, int on);

/* Stage-kernel tile shapes.  The stage kernels walk columns down the grid;
 * a shape is (threads per CTA along x, rows per CTA).  swof_tile_shapes
 * writes up to max shapes (ntx[k], rows[k]) and returns how many exist:
 * the first half stage their input rows through a TMA ring (with a fast
 * path for rows dry across the CTA), the second half are the same
 * (ntx, rows) with a one-row register prefetch instead.
 * swof_set_tile_shape(s) select the shape of both stages, or of stage 1 and
 * stage 2 separately (results do not depend on it).  swof_autotune times
 * each stage kernel with every shape `reps` times on the context's current
 * state (stage 2 on scratch copies, which it allocates and frees: the
 * state, time and budgets are left as they are), selects the fastest per
 * stage, writes the average ms to ms (nullable; 2 x shapes entries, stage 1
 * first) and the choices to best[0] (stage 1) and best[1] (stage 2).
 * Synchronises.  Not in the paper: a GB300 launch-shape choice. */
SWOF_API int swof_tile_shapes(int *ntx, int *rows, int max);
SWOF_API int swof_set_tile_shape(swof_ctx *ctx, int shape);
SWOF_API int swof_set_tile_shapes(swof_ctx *ctx, int shape1, int shape2);
SWOF_API int swof_autotune(swof_ctx *ctx, int reps, double *ms, int *best);

/* ---- batched ensemble ---------------------------------------------------
 * A batch of independent grids of uneven sizes, each with its own dt (the
 * paper's scheme per member, Sec. 2-3), advanced together by ONE persistent
 * kernel launch per swof_ensemble_step call, replayed from a CUDA graph.
 * The launch works through a queue of (step, phase, member, tile) items;
 * an item waits (bounded) only for earlier phases of its own member, so
 * members never wait on each other.  Each member is an ordinary context
 * (swof_ensemble_member) whose results equal what its own swof_step would
 * give, bit for bit.  Not in the paper: the GB300 batching of its method. */
typedef struct swof_ens swof_ens;

typedef struct swof_scenario {
    int nx, ny;                    /* grid (>= 2 x 2) */
    double dx, dy;
    const double *z;               /* [ny][nx] host, copied */
    const double *h, *hu, *hv;     /* initial state [ny][nx] host, copied */
    double manning_n;              /* > 0: Manning friction with this n */
    double rain_rate, rain_t_on, rain_t_off;
    int bc[4];                     /* W, E, S, N: wall, outflow or an imposed edge (Sec. 2.2) */
    double bc_h[4], bc_q[4];       /* imposed depth / discharge per edge (as in swof_params) */
} swof_scenario;

/* Create `count` members from specs; every other parameter (precision, g,
 * cfl, h_dry, dt_max, t_end, infiltration off...) comes from *common.  The
 * launch runs the second-order step: common->order = SWOF_ORDER_1 is
 * SWOF_EINVAL.  Errors: as swof_create / swof_set_state. */
SWOF_API int swof_ensemble_create(int count, const swof_scenario *specs, const swof_params *common,
                                  swof_ens **out);
SWOF_API void swof_ensemble_destroy(swof_ens *e);   /* NULL-safe; destroys the members */
SWOF_API int swof_ensemble_size(const swof_ens *e);
/* Borrow member k's context (state, diagnostics, dt history; owned by e). */
SWOF_API int swof_ensemble_member(swof_ens *e, int k, swof_ctx **ctx);
/* Advance every member by n steps in one launch.  Asynchronous when status
 * is NULL; otherwise synchronises and reports SWOF_OK, a member's latched
 * status, or SWOF_ETIMEOUT when a bounded wait ran out (latched: later
 * calls return it). */
SWOF_API int swof_ensemble_step(swof_ens *e, int n, int *status);
/* Member tile shapes (CTA width ntx, rows per tile): swof_ensemble_shapes
 * writes up to max of them and returns how many exist.  One launch has one
 * CTA width, each member its own tile height among that width's shapes.
 * swof_ensemble_set_shape gives every member `shape` (and its width);
 * swof_ensemble_set_member_shape gives member k a shape of the current
 * width (SWOF_EINVAL otherwise); swof_ensemble_get_member_shape returns
 * member k's.  swof_ensemble_autotune times launches of `steps` steps: for
 * each width, every member on that width's first shape, then per member
 * size class (grid nx x ny) each other height of the width, kept when the
 * launch gets faster; the fastest width's choice is applied.  ms (nullable,
 * 2 entries: widths 128 and 64) gets the ms per step of each width's best,
 * best the shape of member 0, member_shapes (nullable, count entries) every
 * member's.  Every member is put back as it was after each timed launch.
 * Not in the paper: a GB300 launch-shape choice. */
SWOF_API int swof_ensemble_shapes(int *ntx, int *rows, int max);
SWOF_API int swof_ensemble_set_shape(swof_ens *e, int shape);
SWOF_API int swof_ensemble_set_member_shape(swof_ens *e, int k, int shape);
SWOF_API int swof_ensemble_get_member_shape(const swof_ens *e, int k);
SWOF_API int swof_ensemble_autotune(swof_ens *e, int steps, double *ms, int *best, int *member_shapes);
/* Bound on the polls of each wait (default 4M, about a second), and a test
 * hook: block_member >= 0 makes that member's waits impossible so the
 * bound is exercised (-1: off). */
SWOF_API int swof_ensemble_set_wait_limit(swof_ens *e, long long polls, int block_member);

/* ---- tensor-core building block ------------------------------------------
 * C[M x N] (fp32, row stride ldc) = A[M x K] . B[N x K]^T (+ bias[N]) with
 * A, B row-major bf16 device arrays (K contiguous), on the tcgen05 tensor
 * cores with FP32 accumulation in tensor memory.  N in {16, 32, 64, 128,
 * 256}, K a multiple of 64, any M.  *err (device int) is set to 1 if a
 * bounded wait inside the kernel ran out.  Enqueued on stream.  Not in the
 * paper: the GEMM of the learned surrogate's layers. */
SWOF_API int swof_gemm_bf16_nt(const void *A, const void *B, float *C, const float *bias, int M, int N, int K,
                               int ldc, int *err, void *stream);

/* ---- learned surrogate ---------------------------------------------------
 * A 4-level convolutional U-Net on coarsened fields (base width `base`,
 * 3x3 convolutions with GELU, 2x2 average pooling, 2x2 stride-2 transposed
 * convolutions, skip concatenations, a 1x1 output convolution), trained
 * and run on the tcgen05 tensor cores: BF16 weights and activations, FP32
 * accumulation, FP32 master weights, gradients and AdamW moments.  It maps
 * a coarse state (h, hu, hv, z) to the state a fixed number of solver steps
 * later; the plain solver is its fallback and the judge of its error.  Not
 * in the paper: the learned part built around its method.
 *
 * Memory is allocated at creation for batches up to max_batch of H x W
 * (H, W multiples of 8, >= 16).  base in {16, 32, 48, 64}; in_ch, out_ch <= 16.
 * Weights are Kaiming-normal from `seed`.  Parameters are one flat FP32
 * array: each layer's weights as [columns][Kp] rows (K = taps x padded
 * input channels, zero-padded to a multiple of 64), then all biases;
 * swof_unet_layout describes layer `layer` in info[9] = {kind (0 3x3,
 * 1 1x1, 2 transposed 2x2), cin, cin_padded, cout, columns, Kp, weight
 * offset, bias offset, gelu} and returns the number of layers. */
typedef struct swof_unet swof_unet;
SWOF_API int swof_unet_create(int base, int in_ch, int out_ch, int H, int W, int max_batch,
                              unsigned long long seed, swof_unet **out);
SWOF_API void swof_unet_destroy(swof_unet *u);
SWOF_API long long swof_unet_param_count(const swof_unet *u);
SWOF_API int swof_unet_layout(const swof_unet *u, int layer, int *info);
SWOF_API int swof_unet_get_params(swof_unet *u, float *host);
SWOF_API int swof_unet_set_params(swof_unet *u, const float *host);
SWOF_API int swof_unet_get_grads(swof_unet *u, float *host);
/* Input normalisation (x - mean) / scale_in per input channel and output
 * scale: the network predicts (next - in) / scale_out. */
SWOF_API int swof_unet_set_norm(swof_unet *u, const float *mean, const float *scale_in, const float *scale_out);
/* Raw network: x bf16 [B*H*W][16] NHWC device -> y fp32 [B*H*W][16]. */
SWOF_API int swof_unet_forward_raw(swof_unet *u, const void *x, int B, float *y, void *stream);
/* Mean-squared-error gradients (no update) for raw x and targets tgt fp32
 * [B*H*W][out_ch]; synchronises; *loss_host = sum of squared errors, or
 * SWOF_ETIMEOUT if a bounded tensor-core wait ran out. */
SWOF_API int swof_unet_grads_raw(swof_unet *u, const void *x, const float *tgt, int B, double *loss_host,
                                 void *stream);
SWOF_API int swof_unet_adamw(swof_unet *u, float lr, float beta1, float beta2, float eps, float weight_decay,
                             void *stream);
/* Diagnostics: an internal activation of the last forward as fp32 on the
 * host (which: 0 input, 1 first conv out, 2 its pre-activation, 3 concat
 * buffer, 4 pooled input, 5/6 decoder convs, 7 bottom, 8 output; level l;
 * n values, NHWC).  Synchronises the device. */
SWOF_API int swof_unet_activation(swof_unet *u, int which, int level, float *host, long long n);
/* State-level training step and prediction (FP32 NCHW device arrays):
 * in [B][in_ch][H][W], next / out [B][out_ch][H][W]; out = in[:out_ch] +
 * scale_out * net((in - mean) / scale_in). */
SWOF_API int swof_surrogate_train_step(swof_unet *u, const float *in, const float *next, int B, float lr,
                                       float weight_decay, double *loss_host, void *stream);
SWOF_API int swof_surrogate_predict(swof_unet *u, const float *in, int B, float *out, void *stream);

/* Coarsen a context's state: block means of h, hu, hv and the infiltrated
 * depth V_inf over f x f cells (FP64 sums) into out, a device fp32 array
 * [4][ny/f][nx/f] (nx, ny multiples of f), enqueued on the context's
 * stream.  The surrogate's training data and its judge (the fine solver,
 * coarsened).  Errors: SWOF_EINVAL. */
SWOF_API int swof_coarsen(swof_ctx *ctx, int f, float *out);

/* The surrogate's static input channels from a fine bed z and K_s map
 * (device float64 [ny][nx], caller-owned; ks NULL: the scalar ks_const
 * everywhere), coarsened by block means over f x f cells (FP64 sums in a
 * fixed order): channel 0 = dz_c/dx, 1 = dz_c/dy -- central differences of
 * the block-mean bed z_c with spacings f dx, f dy, one-sided at the edges --
 * and 2 = the block-mean K_s, written as device fp32 to
 * out[k * snap_stride + c * (ny/f)(nx/f) + J (nx/f) + I] for every snapshot
 * k < nsnap (out points at channel 0 of snapshot 0), enqueued on stream.
 * nx, ny multiples of f, nx/f and ny/f >= 2, snap_stride >= 3 (ny/f)(nx/f).
 * Not in the paper: the network's inputs (the dynamics depend on the bed's
 * slopes, not its height).  Errors: SWOF_EINVAL. */
SWOF_API int swof_coarsen_static(const double *z, const double *ks, double ks_const, int nx, int ny, double dx,
                                 double dy, int f, float *out, long long snap_stride, int nsnap, void *stream);

/* Per-member FP64 statistics of a batch of states [B][C][H][W] (device
 * fp32; channels h, hu, hv, then V_inf when C >= 4) into the device array
 * out[5B]: out[5b..5b+4] = {sum h, sum min(h, 0), discharge leaving through
 * the edges in outmask [m^3/s], sum V_inf (0 when C < 4), min h}.  outmask
 * bits: 1 W, 2 E, 4 S, 8 N (the edge order of swof_params.bc); discharge is
 * the normal q of the edge cells times the edge length (dx or dy).
 * Fixed-order sums (deterministic).  Enqueued on stream. */
SWOF_API int swof_batch_stats(const float *states, int B, int C, int H, int W, int outmask, double dx,
                              double dy, double *out, void *stream);

/* Rollout: advance B coarse members `calls` times by one span each with
 * the network, checking every prediction and falling back to the plain
 * solver where the check fails.
 *   states      device fp32 [B][in_ch][H][W]: channels 0..out_ch-1 are the
 *               state (h, hu, hv[, V_inf]), the rest the network's other
 *               inputs; updated in place (the rain channel gets the rain
 *               rate of each member's next span, averaged over its steps).
 *   t           host [B]: each member's time, advanced by span per call.
 *   rain        host [B][3]: rain rate [m/s], t_on, t_off per member.
 *   fallback    host array of contexts on the same H x W grid (W = nx),
 *               FP64 or FP32, created with dt_fixed = span / fallback_steps
 *               and the member's z, friction, rain, infiltration and edges;
 *               fallback_of[b] indexes it (members may share a context: it is
 *               reset from the member's state, V_inf and time before use).
 *   accepted    host [calls][B] (nullable): 1 where the prediction passed.
 *   checks      host [calls][B][2] (nullable): mass and positivity errors.
 * Check (after the prediction, before any clamp), relative to the water
 * present plus the span's rain, with area A = dx dy per cell:
 *   mass       |dV - (rain in - (V_inf increase) A - discharge out)| <= tol,
 *              the discharge the trapezoid of the edge discharge before and
 *              after, the rain that of the fallback_steps steps of the span
 *              (rain falls in a step that starts in [t_on, t_off));
 *   positivity -sum min(h, 0) A <= tol.
 * Passing members take the prediction with h < 0 set to 0, q = 0 where
 * h <= h_dry and V_inf never decreasing; the others take the solver's
 * state after fallback_steps steps.  Synchronises once per call.  Errors:
 * SWOF_EINVAL; SWOF_ESTATE if a failing member has no fallback (it stays
 * at its pre-call state and time; the rollout stops after that call); a
 * fallback context's own error.  inject_* is a test hook: add inject_dh to
 * member inject_member's predicted depth at call inject_call (-1: off). */
typedef struct swof_rollout_opts {
    int calls;
    int fallback_steps;
    double span;
    double dx, dy;
    double tol;
    double h_dry;
    int rain_channel;          /* input channel of the rain rate, or -1 */
    int outflow_mask;          /* edges where water leaves (bits as above) */
    int inject_member, inject_call;
    double inject_dh;
} swof_rollout_opts;
SWOF_API int swof_surrogate_rollout(swof_unet *u, float *states, int B, double *t, const double *rain,
                                    swof_ctx *const *fallback, const int *fallback_of,
                                    const swof_rollout_opts *opts, int *accepted, double *checks, void *stream);

/* Human-readable text for a status code (static storage). */
SWOF_API const char *swof_strerror(int code);

/* Library build information (static storage). */
SWOF_API const char *swof_version(void);

/* Debug build (libswof_debug.so, compiled with SWOF_BOUNDS_CHECK): every
 * padded-array index the stencil kernels form, every ring slot the stage
 * kernels read and every tensor-copy origin is checked on the device; a
 * failed check clamps the index to element 0 (no access leaves the arrays)
 * and latches SWOF_EBOUNDS in the context's status word, which swof_step
 * (with info), swof_get_diagnostics and every later launch see.  Not in the
 * paper: a checking aid.
 * swof_debug_build returns 1 in the debug build, 0 otherwise.
 * swof_debug_probe_index runs one thread that forms the padded index of
 * cell (i, j) of ctx's grid (i, j may lie outside [-2, nx+1] x [-2, ny+1])
 * through the checked path and reads the element there, so a test can see a
 * failed check latch SWOF_EBOUNDS without any out-of-range access.
 * Synchronises; returns the latched status (SWOF_OK when the index was in
 * range), or SWOF_ESTATE in the release build. */
SWOF_API int swof_debug_build(void);
SWOF_API int swof_debug_probe_index(swof_ctx *ctx, int i, int j);

#ifdef __cplusplus
}
#endif
#endif /* SWOF_H */
