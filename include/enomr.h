/*
 * enomr.h -- C ABI of libenomr.so, a GB300 (sm_103a) FP64 implementation of
 * the ENO-MR semi-discrete right-hand side and its SSP-RK3 stage update.
 *
 * Method: "An efficient class of increasingly high-order ENO schemes with
 * multi-resolution" (arXiv 2311.15504).
 *
 * Conventions shared by every entry point
 * --------------------------------------
 * Memory.   Every array argument is a DEVICE pointer on the current CUDA
 *           device unless its description says "host".  The caller owns all
 *           state, output and selection buffers; the library owns only the
 *           scratch it allocates in enomr_init() and frees in enomr_free().
 *           No entry point allocates device memory after enomr_init().
 * Layout.   FP64, component-major ("structure of arrays"), x fastest:
 *             scalar advection   U[nx]
 *             1D Euler           U[3][nx]       (rho, rho u, rho e)
 *             2D Euler           U[4][ny][nx]   (rho, rho u, rho v, rho e)
 *           Pointers must be 8-byte aligned; arrays are dense (pitch = nx).
 * Streams.  All work is enqueued on the stream given to enomr_init() (or
 *           enomr_set_stream()); calls return without synchronising unless
 *           stated.  Entry points that do not synchronise can be recorded
 *           into a CUDA graph by the caller.
 * Errors.   Argument errors are detected on the host and returned at once
 *           (ENOMR_EINVAL); nothing is launched then.  CUDA launch/runtime
 *           errors give ENOMR_ECUDA.  Non-physical states met on the device
 *           (rho <= 0, p <= 0, Roe c^2 <= 0, NaN/Inf) set a device status
 *           word that enomr_get_status() reads; the kernels never trap,
 *           abort or print.
 * Grid.     Uniform spacing dx (dy).  Boundary: periodic (requires
 *           nx, ny >= 2g, g = (order+1)/2) or transmissive (zeroth-order
 *           extrapolation into g ghost cells).
 */
#ifndef ENOMR_H
#define ENOMR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ENOMR_API __attribute__((visibility("default")))
#else
#define ENOMR_API
#endif

typedef enum {
    ENOMR_OK = 0,
    ENOMR_EINVAL = 1,   /* bad argument; nothing was launched              */
    ENOMR_ENOMEM = 2,   /* scratch allocation failed in enomr_init          */
    ENOMR_ECUDA = 3,    /* a CUDA runtime call or launch failed             */
    ENOMR_ENONPHYS = 4, /* a kernel met a non-physical state (status word)  */
    ENOMR_ETIMEOUT = 5  /* a bounded device wait gave up (status word)      */
} enomr_status;

typedef enum { ENOMR_ADVECTION = 0, ENOMR_EULER = 1, ENOMR_BURGERS = 2 } enomr_eq;
typedef enum { ENOMR_PERIODIC = 0, ENOMR_TRANSMISSIVE = 1 } enomr_bc;

typedef struct enomr_ctx enomr_ctx;

/*
 * enomr_init -- create a solver context for one problem.
 *   eq         ENOMR_ADVECTION (f(u) = adv_speed * u, ndim must be 1),
 *              ENOMR_EULER (ideal gas, gamma > 1; ndim 1 or 2) or
 *              ENOMR_BURGERS (f(u) = u^2/2, Sec. 4.2; ndim must be 1).
 *              Burgers: where u keeps one sign over the line (f' = u) the
 *              flux is not split (f^+ = f, f^- = 0, or the mirror), as the
 *              paper does for its test; otherwise the global Lax-Friedrichs
 *              split with alpha = max |u| (Eq. LF_Flux_Split).  The CFL step
 *              is cfl * dx / max |u| (0 for u = 0, a steady state).
 *   nx, ny     cells per direction (ny = 1 for ndim = 1).
 *   dx, dy     spacing h of Sec. 2.1 (dy ignored in 1D).
 *   order      R = 2r-1 in {5,7,9,11,13,15,17}: the (2r-1)-point ENO-MR scheme
 *              (Sec. 3.1, Eq. Candidates, candidates with m,n <= r-1).
 *   bc         ENOMR_PERIODIC or ENOMR_TRANSMISSIVE.
 *   stream     cudaStream_t (NULL = legacy default stream).
 * Allocates the context's device scratch (per-line alpha, status word,
 * CFL reduction, two stage buffers and, in 2D, one partial-RHS buffer).
 * On success *out receives the context; release it with enomr_free().
 */
ENOMR_API enomr_status enomr_init(enomr_ctx **out, int eq, int ndim, int64_t nx, int64_t ny,
                                  double dx, double dy, int order, double gamma, int bc,
                                  double adv_speed, void *stream);

/* enomr_free -- release the context and its scratch (NULL is ignored). */
ENOMR_API void enomr_free(enomr_ctx *ctx);

/* enomr_strerror -- static description of a status code. */
ENOMR_API const char *enomr_strerror(int status);

/* enomr_set_stream -- change the stream later calls are enqueued on. */
ENOMR_API enomr_status enomr_set_stream(enomr_ctx *ctx, void *stream);

/*
 * enomr_rhs -- dUdt = L(U), Eq. (1DWENOFD):
 *   L(U)_i = -(F_{i+1/2} - F_{i-1/2})/dx [ - (G_{j+1/2} - G_{j-1/2})/dy in 2D ],
 * with F from the global Lax-Friedrichs split (Eq. LF_Flux_Split; for
 * Euler per characteristic field k, alpha_k = max |lambda_k| over the
 * cells of the line), Roe-averaged characteristic projection (Sec. 4),
 * ENO-MR selection (Sec. 3.2 Steps 1-3) and reconstruction
 * (Eq. ReconstructedFlux) on each side, and back-projection.
 * U and dUdt: device, layout above, must not overlap.
 */
ENOMR_API enomr_status enomr_rhs(enomr_ctx *ctx, const double *U, double *dUdt);

/*
 * enomr_stage -- one stage s in {1,2,3} of SSP-RK3 (Eq. TVD3rdRK):
 *   s=1: Uout = Un + dt L(Un)                     (Us must equal Un)
 *   s=2: Uout = 3/4 Un + 1/4 (Us + dt L(Us))
 *   s=3: Uout = 1/3 Un + 2/3 (Us + dt L(Us))
 * The RHS is fused with the combination, rounded as written: stage 1 as
 * fma(dt, L, Un), stages 2 and 3 as fma(c0, Un, c1 * fma(dt, L, Us)).
 * dt > 0 (host value).  Uout may alias Un but not Us.
 */
ENOMR_API enomr_status enomr_stage(enomr_ctx *ctx, int stage, const double *Un, const double *Us,
                                   double *Uout, double dt);

/*
 * enomr_step -- one full SSP-RK3 step in place on U (device).
 *   dt > 0: use dt.  dt <= 0: dt = cfl-based step computed on the device
 *   from U^n (1D: cfl*dx/max(|u|+c); 2D: cfl/max((|u|+c)/dx+(|v|+c)/dy);
 *   advection: cfl*dx/|a|).
 *   dt_used (host, may be NULL): if non-NULL the call synchronises the
 *   stream and stores the dt that was used.
 * Uses the context's two stage buffers; the call is not re-entrant on one
 * context.
 */
ENOMR_API enomr_status enomr_step(enomr_ctx *ctx, double *U, double dt, double cfl,
                                  double *dt_used);

/*
 * enomr_step_lssp -- one step of the linear SSP-RK(m, m-1) scheme of
 * Eq. (lSSPRK), in place on U (device), with fixed dt > 0, 2 <= m <= 32:
 *   u(0) = U;  u(s) = u(s-1) + dt/2 L(u(s-1)), s = 1..m-1;
 *   U <- sum_{k=0}^{m-2} a_k u(k) + a_{m-1} (u(m-1) + dt/2 L(u(m-1))),
 * with a_k = alpha_{m,k} of Eq. (lSSPRK_Coe) (alpha_{m,m-1} read as
 * (2/m) alpha_{m-1,m-2}).  Meant for linear problems (advection), where it
 * has order m-1; uses the context's stage buffers.
 */
ENOMR_API enomr_status enomr_step_lssp(enomr_ctx *ctx, double *U, double dt, int m);

/* enomr_cfl_dt -- the CFL step of enomr_step for state U, returned in
 * *dt_host (host).  Synchronises the stream. */
ENOMR_API enomr_status enomr_cfl_dt(enomr_ctx *ctx, const double *U, double cfl, double *dt_host);

/*
 * Boundary sides and body force of the 2D problems of Sec. 4.4 (double Mach
 * reflection, Rayleigh-Taylor instability) for 2D Euler contexts created
 * with ENOMR_TRANSMISSIVE.  The domain is [0, nx dx] x [0, ny dy]; a side's
 * along-side coordinate of a line is the cell centre of the row (x sides)
 * or column (y sides).  A side is split at position split0 + split_rate t
 * (t the time of the stage; split0 = +inf: one kind everywhere): kind_lo
 * applies below it, kind_hi above.  Kinds:
 *   ENOMR_SIDE_TRANSMISSIVE  copy of the nearest cell (the default);
 *   ENOMR_SIDE_REFLECTIVE    mirror image of the interior, normal momentum
 *                            negated (needs at least g = (order+1)/2 cells
 *                            across);
 *   ENOMR_SIDE_INFLOW        the given conserved state (rho, rho u, rho v, E)
 *                            in every ghost cell.
 * Sides: 0 x low, 1 x high, 2 y low, 3 y high.  The adjoint entry points
 * reject a context with sides set or a body force.
 */
typedef enum {
    ENOMR_SIDE_TRANSMISSIVE = 1,
    ENOMR_SIDE_REFLECTIVE = 2,
    ENOMR_SIDE_INFLOW = 3
} enomr_side_kind;

typedef struct {
    int kind_lo, kind_hi;
    double split0, split_rate;
    double state_lo[4], state_hi[4];
} enomr_side;

/* enomr_set_side -- set one side (copied; synchronous: waits for the work
 * already queued on the context's stream, which may read the sides, before
 * it replaces them).  ENOMR_EINVAL for a
 * context that is not 2D Euler with transmissive boundaries, a bad kind or
 * side, a reflective side across fewer than g cells, or a non-physical
 * inflow state. */
ENOMR_API enomr_status enomr_set_side(enomr_ctx *ctx, int side, const enomr_side *desc);

/* enomr_set_body_force -- add S = (0, rho gx, rho gy, rho u gx + rho v gy)
 * to the right-hand side after the two directional flux differences
 * (2D Euler only); (0, 0) removes it.  The first non-zero force of a
 * context without sides waits for the work queued on its stream. */
ENOMR_API enomr_status enomr_set_body_force(enomr_ctx *ctx, double gx, double gy);

/* enomr_set_time / enomr_get_time -- the time of the state the next
 * enomr_step starts from (device scalar, 0 after enomr_init), which only
 * boundary sides depend on.  With sides or a body force set, enomr_step and
 * enomr_step_lssp advance it by their dt; the SSP-RK3 stages see t,
 * t + dt, t + dt/2; enomr_rhs and enomr_debug_selection see t; stage s of
 * enomr_stage sees t + c_s dt (c = 0, 1, 1/2).  Both synchronise the
 * stream. */
ENOMR_API enomr_status enomr_set_time(enomr_ctx *ctx, double t);
ENOMR_API enomr_status enomr_get_time(enomr_ctx *ctx, double *t);

/*
 * enomr_debug_selection -- the stencil chosen at every interface, field and
 * side for state U (same arithmetic as enomr_rhs).  sel (device, uint8):
 *   advection  [2][nx+1]
 *   1D Euler   [2][3][nx+1]
 *   2D Euler   x sweep [2][4][ny][nx+1] followed by y sweep [2][4][nx][ny+1]
 * side 0 = f^+, 1 = f^-; interface k is x_{k-1/2} (between cells k-1, k).
 * Field order: (u-c, u, [shear], u+c) in the sweep's normal velocity.
 * Value: t in [0,T) = t-th tested candidate of Eq. (Candidates) (filtered to
 * the order), T, T+1, T+2 = minmod outcome S(0,1), S(1,0), S(0,0)
 * (Step 3.2).  T = 4,7,10,14,18,22,26 for orders 5..17.
 */
ENOMR_API enomr_status enomr_debug_selection(enomr_ctx *ctx, const double *U, uint8_t *sel);

/*
 * enomr_stage_frozen -- one SSP-RK3 stage as enomr_stage(), with the discrete
 *   choices of the right-hand side taken from the reference state Uref
 *   instead of Us: the stencil or minmod branch of every interface, field
 *   and side (Sec. 3.2) and the cell attaining every per-line alpha_k
 *   (Eq. LF_Flux_Split read per field); every interface is evaluated in full
 *   with those choices, so the result is a smooth function of Us.  This is
 *   the map that enomr_step_vjp transposes: finite differences of it check
 *   the adjoint at any horizon, where those of the plain step cross
 *   selection changes.  With Uref = Us it equals enomr_stage to rounding
 *   (the one-state flat interfaces' shortcut aside).  2D Euler without
 *   boundary sides or body force only (else ENOMR_EINVAL); Uout must not
 *   alias Us or Uref.  Uses the context's adjoint scratch.
 */
ENOMR_API enomr_status enomr_stage_frozen(enomr_ctx *ctx, int s, const double *Un,
                                          const double *Us, double *Uout, double dt,
                                          const double *Uref);

/* enomr_get_status -- synchronise the stream, read and clear the device
 * status word: ENOMR_OK, ENOMR_ENONPHYS, or ENOMR_ETIMEOUT when a sweep's
 * bounded wait for a tile copy ran out (that launch stopped early and its
 * output is incomplete). */
ENOMR_API enomr_status enomr_get_status(enomr_ctx *ctx);

/*
 * enomr_set_staging -- how the 2D Euler sweeps bring a tile of cells (with
 * its g-cell halos, Sec. 2.1) into shared memory:
 *   ENOMR_STAGING_AUTO  (default) both sweeps by TMA where the state
 *                       allows it (nx even, U 16-byte aligned, no boundary
 *                       sides or body force; the faster staging for both
 *                       sweeps on GB300), otherwise plain loads;
 *   ENOMR_STAGING_LOADS plain coalesced loads by the CTA's threads;
 *   ENOMR_STAGING_TMA   the TMA path only: calls whose state does not allow
 *                       it return ENOMR_EINVAL.
 * The TMA sweeps are persistent (one CTA per resident slot, a two-slot ring
 * of tile copies per CTA, the next tile's copy in flight during this
 * tile's arithmetic); all stagings give the same results bit for bit.
 * Host-only setting, no synchronisation.
 */
enum { ENOMR_STAGING_AUTO = 0, ENOMR_STAGING_LOADS = 1, ENOMR_STAGING_TMA = 2 };
ENOMR_API enomr_status enomr_set_staging(enomr_ctx *ctx, int mode);

/*
 * enomr_set_occupancy -- which instance of the 2D Euler sweeps runs:
 *   ENOMR_OCCUPANCY_HIGH  many warps per SM (40 with plain loads, 32 with
 *                         TMA), few registers per thread: hides latency on
 *                         large grids dominated by flat interfaces;
 *   ENOMR_OCCUPANCY_LOW   16 warps per SM, 128 registers per thread (the
 *                         long path's windows stay in registers): for grids
 *                         of few tiles, whose launches last as long as a
 *                         few tiles in sequence;
 *   ENOMR_OCCUPANCY_AUTO  (default) LOW when the x sweep has fewer tiles
 *                         than four waves of the HIGH instance (grids up to
 *                         about 900^2), else HIGH.
 * On smooth data, where every interface takes the long path, LOW with TMA
 * staging is the fastest instance (about 4 % on a 4096^2 vortex); on
 * piecewise-constant data HIGH is (LOW is 40 % slower there).
 * Same results bit for bit.  Host-only setting, no synchronisation.
 */
enum { ENOMR_OCCUPANCY_AUTO = 0, ENOMR_OCCUPANCY_HIGH = 1, ENOMR_OCCUPANCY_LOW = 2 };
ENOMR_API enomr_status enomr_set_occupancy(enomr_ctx *ctx, int mode);

/*
 * Adjoint.  With the discrete choices of the forward pass frozen -- the
 * stencil (or minmod branch) chosen at every interface, field and side, and
 * the cell attaining each per-line alpha -- L is a smooth function of U.
 * The paper has no adjoint; these are its exact transposes.
 *
 * enomr_rhs_vjp -- Ubar = scale * J(U)^T Lbar (accumulate = 0) or
 *   Ubar += scale * J(U)^T Lbar (accumulate != 0), J = dL/dU at U with the
 *   choices L(U) makes.  U, Lbar, Ubar: device, state layout; Ubar must not
 *   alias U or Lbar.  Contributions of cells shared by neighbouring tiles
 *   are added with atomics, so the last bits may vary from run to run.
 *   Advection and Euler only: ENOMR_EINVAL for a Burgers context.
 */
ENOMR_API enomr_status enomr_rhs_vjp(enomr_ctx *ctx, const double *U, const double *Lbar,
                                     double *Ubar, double scale, int accumulate);

/* enomr_debug_alpha -- copy (device to device, on the context's stream) the
 * per-line split speeds alpha [lines][3] (max|u-c|, max|u|, max|u+c|) of the
 * last enomr_rhs/enomr_stage/enomr_rhs_vjp call, and the alpha cotangents
 * and the frozen maximising cells (index along the line) of the last
 * enomr_rhs_vjp call; x-sweep rows [ny][3] and, in 2D, y-sweep columns
 * [nx][3].  Any pointer may be NULL.  A diagnostic of the adjoint. */
ENOMR_API enomr_status enomr_debug_alpha(enomr_ctx *ctx, double *alpha_x, double *alpha_y,
                                         double *alpha_bar_x, double *alpha_bar_y,
                                         uint64_t *argmax_x, uint64_t *argmax_y);

/*
 * enomr_step_vjp -- transpose of one SSP-RK3 step (Eq. TVD3rdRK) taken from
 *   U_n with step dt (> 0, held fixed): U_n_bar = (dU_{n+1}/dU_n)^T U_np1_bar.
 *   The stage states are recomputed from U_n (a per-step checkpoint) in the
 *   context's stage buffers; three enomr_rhs_vjp evaluations follow.
 *   U_n_bar is overwritten and must not alias U_n or U_np1_bar.
 *   Advection and Euler only: ENOMR_EINVAL for a Burgers context.
 */
ENOMR_API enomr_status enomr_step_vjp(enomr_ctx *ctx, const double *U_n, double dt,
                                      const double *U_np1_bar, double *U_n_bar);

/*
 * enomr_step_vjp_cfl -- as enomr_step_vjp for a step that enomr_step took
 *   with its CFL dt (dt <= 0, cfl > 0): the dt is recomputed on the device
 *   from U_n by the same kernels (so it is the forward step's dt bit for
 *   bit) and held fixed.  No host synchronisation, so a long adjoint sweep
 *   runs without a round trip per step.
 */
ENOMR_API enomr_status enomr_step_vjp_cfl(enomr_ctx *ctx, const double *U_n, double cfl,
                                          const double *U_np1_bar, double *U_n_bar);

/*
 * Batched problems: many independent 1D Euler problems of uneven size
 * advanced together, one persistent launch per SSP-RK3 stage.
 *
 * Packing: problem p's state is a dense [3][n[p]] block (rho, rho u, rho e);
 * the blocks follow each other in problem order in one device array, so
 * problem p starts at 3 * (n[0] + ... + n[p-1]) doubles.
 * Each problem has its own spacing dx[p], split speeds alpha_k (over its own
 * cells, Eq. LF_Flux_Split) and CFL step; boundaries and order are shared.
 * The per-interface, per-cell and per-problem arithmetic equals that of
 * enomr_step() with dt <= 0 on the problem alone, so every problem's result
 * is bitwise the same as advancing it on its own.
 */
typedef struct enomr_batch enomr_batch;

/* enomr_batch_init -- n (host, nprob entries, each >= 1; periodic needs
 * n >= order+1), dx (host, nprob entries > 0), order, gamma, bc, stream as in
 * enomr_init().  Builds the tile tables and allocates the scratch (two stage
 * buffers, per-problem alpha and dt). */
ENOMR_API enomr_status enomr_batch_init(enomr_batch **out, int64_t nprob, const int64_t *n,
                                        const double *dx, int order, double gamma, int bc,
                                        void *stream);
ENOMR_API void enomr_batch_free(enomr_batch *b);
ENOMR_API enomr_status enomr_batch_set_stream(enomr_batch *b, void *stream);
/* enomr_batch_total_cells -- sum of n (or -1 for NULL). */
ENOMR_API int64_t enomr_batch_total_cells(const enomr_batch *b);

/* enomr_batch_step -- one SSP-RK3 step in place on the packed state U
 * (device), each problem with its own CFL step cfl*dx[p]/max(|u|+c).
 * Launches: alpha of U^n, per-problem dt, three persistent stage kernels.
 * Does not synchronise; no allocation (graph-capturable by the caller). */
ENOMR_API enomr_status enomr_batch_step(enomr_batch *b, double *U, double cfl);

/* enomr_batch_autotune -- time the stage kernel on state U (read only) for
 * every tile size (32, 64, 128 interfaces), persistent grid (2, 4, 8, 16
 * CTAs per SM) and work-item size (1, 2, 4 consecutive tiles per item, so
 * each thread evaluates that many interfaces per item), reps launches each,
 * and keep the fastest for later steps.  *tile and *grid (host, may be NULL)
 * receive the choice (enomr_batch_config gives all three).  Synchronises.
 * Every setting gives the same results bit for bit. */
ENOMR_API enomr_status enomr_batch_autotune(enomr_batch *b, const double *U, int reps, int *tile,
                                            int *grid);
/* enomr_batch_config -- the tile size, grid and tiles per work item in use
 * (host outputs, each may be NULL). */
ENOMR_API enomr_status enomr_batch_config(const enomr_batch *b, int *tile, int *grid,
                                          int *tiles_per_item);

/* enomr_batch_get_status -- as enomr_get_status(). */
ENOMR_API enomr_status enomr_batch_get_status(enomr_batch *b);

/*
 * Measurement hooks (not part of the method).
 * enomr_profile_begin -- record CUDA events around the next max_launches
 *   launches of one kernel of this context: 1 = the x sweep (1D: the sweep,
 *   advection: the advection kernel), 2 = the y sweep (2D), 3 = the per-line
 *   alpha reduction, 0 = stop.  Creates the events (host call, not for use
 *   inside stream capture).
 * enomr_profile_end -- synchronise the stream and return how many launches
 *   were timed and their summed device time in milliseconds.
 */
ENOMR_API enomr_status enomr_profile_begin(enomr_ctx *ctx, int kernel, int max_launches);
ENOMR_API enomr_status enomr_profile_end(enomr_ctx *ctx, int *n_launches, double *total_ms);

/*
 * enomr_probe_fp64_fma -- FP64 FMA throughput of the current device: a
 * kernel of eight independent fma chains per thread (8 CTAs of 256 threads
 * per SM) runs iters iterations once to warm up and once timed on stream.
 * Returns the timed seconds and the flops it performed (2 per fma).
 * sink: device scratch of at least 8 * SM-count doubles (never written in
 * practice).  Synchronises the stream.
 */
ENOMR_API enomr_status enomr_probe_fp64_fma(void *stream, int64_t iters, double *sink,
                                            double *seconds, double *flops);

/*
 * enomr_rhs_euler2d_noalloc -- the 2D Euler right-hand side of enomr_rhs()
 * for callers that cannot allocate device memory: host frameworks that keep
 * the device memory for their own caching allocator, programs with a fixed
 * device-memory budget, and latency-sensitive loops where cudaMalloc and
 * cudaFree would synchronise the device.  It needs no context and calls no
 * cudaMalloc, cudaFree or other allocating routine.  The paper has no
 * counterpart; this is a service of the library.
 *   U, dUdt   device, [4][ny][nx] (layout above); must not overlap.
 *   nx, ny    at most ENOMR_NOALLOC_MAX_LINES each (else ENOMR_EINVAL).
 *   dx, dy, order, gamma, bc   as in enomr_init(); stream as there.
 * Result: dUdt equals enomr_rhs() of a context with the same parameters.
 * Scratch: the per-line alpha maxima and a status word live in one static
 * device array of the library (about 0.8 MB), held on every GPU that loads
 * the library until the process exits.  Each call made outside stream
 * capture looks up that array's device address on the current device (a
 * host-side step; a device reset may move the array), and calls made during
 * capture reuse the address of the last call outside capture, so make the
 * first call on each device before any stream capture.  All calls share the array and it keeps the last call's
 * contents (each call clears what must start at zero): calls that overlap
 * on the GPU -- on different streams, or from several host threads -- race
 * and give wrong results; serialise them.  Non-physical states are not
 * reported by this entry point.
 */
#define ENOMR_NOALLOC_MAX_LINES 16384
ENOMR_API enomr_status enomr_rhs_euler2d_noalloc(const double *U, double *dUdt, int64_t nx,
                                                 int64_t ny, double dx, double dy, int order,
                                                 double gamma, int bc, void *stream);

/* enomr_num_tested -- T for an order (see above), or -1. */
ENOMR_API int enomr_num_tested(int order);

#ifdef __cplusplus
}
#endif
#endif /* ENOMR_H */
