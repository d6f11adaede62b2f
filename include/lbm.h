/*
 * lbm.h -- C ABI of the GB300 (sm_103a) library for the Galilean-invariant
 * preconditioned cascaded central-moment lattice Boltzmann method on the D2Q9
 * lattice (Hajabdollahi & Premnath, arXiv 1806.10251).
 *
 * What one step computes (pull form of Eq. 2): every fluid cell pulls its nine
 * post-collision populations from the upwind neighbours (Eq. 2b; half-way
 * bounce-back with the moving-wall momentum term at walls and solid cells),
 * forms raw moments (Eq. 3), the density gradient by central differences, the
 * diagonal strain rates from the second-order non-equilibrium moments
 * (Eqs. 51-55), the extended-equilibrium corrections (Eqs. 33, 45-47), and
 * relaxes through the cascaded kernel of Sec. 5 (Eq. 4 when uncorrected), then
 * stores f~ = fbar + K g + S (Eq. 2a).
 *
 * Conventions
 *  - Every call returns an lbm_status; nothing throws across the ABI.
 *    lbm_last_error() gives a thread-local message for the last failure.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Outputs go
 *    to caller-owned host arrays.  Field arrays are nx*ny doubles, index
 *    y*nx + x (x fastest).  Population arrays are 9*nx*ny doubles, index
 *    alpha*nx*ny + y*nx + x, with the velocity ordering
 *      0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *  - A context owns its device memory and is not thread-safe; different
 *    contexts may be used from different threads.
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    needs one returns LBM_ERR_CUDA.
 *  - Observation point: after lbm_step(n) the stored state is the
 *    post-collision array of step n.  lbm_fields returns the density and
 *    velocity that step n's collision used: rho = sum f~, rho u = sum f~ e -
 *    F/(2 gamma) (the collision conserves rho and adds exactly F/gamma to rho u).
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID = -1,        /* bad argument (message says which)          */
    LBM_ERR_OOM = -2,            /* device or host allocation failed            */
    LBM_ERR_CUDA = -3,           /* CUDA runtime error or no device             */
    LBM_ERR_DIVERGED = -4,       /* NaN/Inf in the fields                       */
    LBM_ERR_NOT_CONVERGED = -5,  /* max_steps reached above the tolerance       */
    LBM_ERR_TIMEOUT = -6,        /* wall-clock limit reached                    */
    LBM_ERR_IO = -7              /* checkpoint file could not be read/written   */
} lbm_status;

/* Side kinds.  The two open kinds are those of the square-cylinder channel of
 * Sec. 6:
 *   LBM_SIDE_INLET  (west side only) fully developed parabolic velocity
 *                   profile u(y) = 4 U (y + 1/2)(ny - y - 1/2) / ny^2 between
 *                   walls at y = -1/2 and ny - 1/2, U = ux (|U| < 0.5),
 *                   imposed by half-way bounce-back with the moving-wall term
 *                   (rho0 = 1), u taken where the link crosses the inlet plane;
 *   LBM_SIDE_OUTLET (east side only) convective outflow d_t u + U d_x u = 0 of
 *                   Sec. 6 with U = ux (0 <= U <= 1): a ghost column at x = nx
 *                   carries a velocity advanced by that equation (explicit,
 *                   upwind, unit lattice steps) and supplies the populations
 *                   entering the domain as the equilibrium (Eq. 15) at the
 *                   reference density rho0 = 1 and that velocity plus the last
 *                   column's non-equilibrium part (the reference density fixes
 *                   the pressure level).  The ghost column starts from the last
 *                   column's velocity whenever the populations are set
 *                   (lbm_init_fields, lbm_set_populations, a storage change) and
 *                   is carried by checkpoints.
 * Open-sided domains are stepped by lbm_step; batches refuse them. */
typedef enum {
    LBM_SIDE_PERIODIC = 0,
    LBM_SIDE_WALL = 1,
    LBM_SIDE_MOVING_WALL = 2,
    LBM_SIDE_INLET = 3,
    LBM_SIDE_OUTLET = 4
} lbm_side_kind;

typedef struct {
    int kind;          /* lbm_side_kind                                              */
    double ux, uy;     /* wall velocity (MOVING_WALL); peak speed (INLET, ux);       */
                       /* convection speed (OUTLET, ux)                              */
} lbm_side;

/* Opposite sides must both be periodic or both non-periodic.  A link whose
 * source lies beyond one side takes that side's wall velocity; a link whose
 * source lies beyond two sides (a corner) sees a stationary wall.  The solid
 * mask (optional, nx*ny bytes, non-zero = solid, copied) adds stationary
 * bounce-back obstacles. */
typedef struct {
    lbm_side west, east, south, north;
    const uint8_t *solid;
} lbm_boundaries;

typedef struct lbm_ctx lbm_ctx;

/* Storage formats of the population arrays (collision is FP32 for the first
 * three, FP64 for the last).  Populations are stored as deviations
 * f_alpha - w_alpha rho0 from the rest state (rho0 = 1). */
enum { LBM_STORAGE_F32 = 0, LBM_STORAGE_F16 = 1, LBM_STORAGE_BF16 = 2, LBM_STORAGE_F64 = 3 };
/* Collision kernels: Eq. 4 (uncorrected), Eq. 4 with the gamma^2-scaled cubic
 * third-order equilibria only, and the full Sec. 5 kernel (default). */
enum { LBM_GI_UNCORRECTED = 0, LBM_GI_CUBIC_ONLY = 1, LBM_GI_FULL = 2 };

/* Create a domain of nx x ny cells (nx, ny >= 3) with kinematic viscosity nu
 * (> 0; omega4 = omega5 = 1/(3 nu/gamma + 1/2), Eq. 49), preconditioning
 * parameter gamma in (0, 1], and reference speed U (>= 0).  bnd == NULL gives
 * the lid-driven cavity: stationary west/east/south walls, north wall moving
 * at (U, 0).  The state starts at rest (rho = 1, u = 0).  *out receives the
 * context on success and NULL on failure. */
lbm_status lbm_create(int nx, int ny, double nu, double gamma, double U,
                      const lbm_boundaries *bnd, lbm_ctx **out);

/* Options (before or between steps):
 *   "omega3", "omega6", "omega7", "omega8"  relaxation rates in (0, 2), default 1
 *   "gi_mode"   LBM_GI_* (default LBM_GI_FULL)
 *   "storage"   LBM_STORAGE_* (default F32); changing it re-encodes the state
 *   "fx", "fy"  uniform body force (default 0)
 *   "guard"     1 = drop the velocity-dependent parts of the strain-rate solve
 *               where |D| < 0.1 |D0| (Eqs. 53-55; off by default), counted
 *   "fd"        density gradient of the GI correction (Eq. 54): 0 (default)
 *               central differences, 1 the isotropic stencil
 *               d_i rho = 3 sum_a w_a e_ai rho(x + e_a) (Sec. 5 names both; a
 *               missing neighbour takes the cell's own density either way);
 *               single-domain contexts only (batches use central differences)
 *   "cells_per_item" rows per work item of the step kernel (tuning; >= 1)
 *   "stochastic_rounding" FP16/BF16 storage: 1 (default) rounds each stored
 *               deviation up or down with probability given by its distance
 *               to the two neighbours (random bits: a hash of step, cell and
 *               direction, so runs are reproducible); 0 rounds to nearest
 *               (ties away from zero) */
lbm_status lbm_set_option(lbm_ctx *ctx, const char *key, double value);
lbm_status lbm_get_option(lbm_ctx *ctx, const char *key, double *value);

/* Launch on this CUDA stream (a cudaStream_t; NULL = the context's own). */
lbm_status lbm_set_stream(lbm_ctx *ctx, void *stream);

/* Per-cell body force (host arrays nx*ny, copied); NULL, NULL removes it. */
lbm_status lbm_set_force_field(lbm_ctx *ctx, const double *fx, const double *fy);

/* Initialise the state to f~0 = f_eq(rho, u) - S/2 with the Eq. 15 raw
 * equilibria (fourth moment such that the central fourth moment is rho/9).
 * NULL fields mean rho = 1 / u = 0.  Resets the step counter. */
lbm_status lbm_init_fields(lbm_ctx *ctx, const double *rho, const double *ux, const double *uy);

/* Advance n >= 0 steps.  Asynchronous with respect to the host. */
lbm_status lbm_step(lbm_ctx *ctx, long n);

/* March to steady state: every check_every steps compute
 * r = ||u^n - u^(n - check_every)||_2 / ||u^n||_2 over fluid cells in FP64 and
 * stop when r < tol.  NaN/Inf gives LBM_ERR_DIVERGED; reaching max_steps gives
 * LBM_ERR_NOT_CONVERGED; wall_seconds > 0 bounds the wall time (LBM_ERR_TIMEOUT).
 * steps_done / final_residual may be NULL. */
lbm_status lbm_run_to_steady(lbm_ctx *ctx, double tol, long check_every, long max_steps,
                             double wall_seconds, long *steps_done, double *final_residual);

/* Convergence history of the last lbm_run_to_steady call on this context (the
 * residual histories the paper plots per gamma, Sec. 6): one entry per check,
 * the step count after it (as lbm_steps_done) and r.  Copies the first
 * min(capacity, count) entries into the caller-owned arrays steps / residuals
 * (either may be NULL, capacity >= 0) and stores the number of entries in
 * *count (not NULL).  Empty before the first run; each run starts a new one.
 * Host bookkeeping only: no device call. */
lbm_status lbm_residual_history(lbm_ctx *ctx, long *steps, double *residuals, long capacity, long *count);

/* One convergence check now: residual against the previous check (or the
 * initial state), then the snapshot is replaced.  sums (may be NULL) receives
 * {sum |du|^2, sum |u|^2, sum rho, sum rho ux, sum rho uy} over fluid cells. */
lbm_status lbm_residual(lbm_ctx *ctx, double *residual, double sums[5]);

/* Density and velocity (see the observation point above); NULL skips a field;
 * solid cells give NaN.  Synchronises the context's stream. */
lbm_status lbm_fields(lbm_ctx *ctx, double *rho, double *ux, double *uy);

/* Full populations f (not deviations), 9*nx*ny doubles, for checks and restart. */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f);
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f);

lbm_status lbm_steps_done(lbm_ctx *ctx, long *steps);
lbm_status lbm_guard_count(lbm_ctx *ctx, long *count);

/* Momentum-exchange force on the solid cells of the mask (Sec. 6, square
 * cylinder; the standard method the paper names): over every link from a
 * fluid cell x to a solid cell x + e_a, the post-collision population f~_a(x),
 * which half-way bounce-back returns at the next step, hands the solid
 * 2 e_a f~_a(x).  force (caller-owned, 2 doubles) receives the sum in lattice
 * momentum per step of the current state, in FP64.  The preconditioned
 * momentum equation carries every flux divided by gamma (Eq. 1), so the
 * physical force is gamma times this value: C_D = 2 gamma force[0] / (rho0 U^2 D). */
lbm_status lbm_drag(lbm_ctx *ctx, double force[2]);

/* Failure-path self-test (no counterpart in the paper).  Every mbarrier wait of
 * the step kernels gives up after 2 s, raises the context's device error flag
 * and lets its warp return; the next synchronising call then returns
 * LBM_ERR_CUDA once, clears the flag and leaves the context usable.  This call
 * drives that path without a fault: one thread of a one-block kernel waits,
 * with the same bounded wait, on an mbarrier that nothing completes, and the
 * call reports the raised flag like a step would.  Expected result:
 * LBM_ERR_CUDA ("bounded wait expired"), *waited_s (optional) >= 2 s; LBM_OK
 * would mean the wait did not expire.  The populations are not touched. */
lbm_status lbm_bounded_wait_selftest(lbm_ctx *ctx, double *waited_s);

/* Checkpoint: the stored post-collision array (in its storage format), step
 * count and parameters (storage format, gi_mode, gamma, nu, omega3..omega8,
 * uniform force).  lbm_load needs a context of the same size; it restores
 * those and keeps the context's own sides, solid mask, force field and the
 * options "guard", "fd", "stochastic_rounding" and "cells_per_item".  Errors:
 * LBM_ERR_IO for an unreadable, foreign or truncated file, LBM_ERR_INVALID
 * for a size mismatch. */
lbm_status lbm_save(lbm_ctx *ctx, const char *path);
lbm_status lbm_load(lbm_ctx *ctx, const char *path);

void lbm_destroy(lbm_ctx *ctx);           /* NULL-safe */
const char *lbm_last_error(void);         /* thread-local, never NULL */

/* Device memory provider (process-wide).  alloc returns a device pointer of at
 * least `bytes` bytes aligned to 256 bytes, or NULL; release frees it.  NULL
 * restores cudaMalloc/cudaFree.  Set it before creating contexts. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*release)(void *ptr, void *user);
    void *user;
} lbm_allocator;
lbm_status lbm_set_allocator(const lbm_allocator *a);

/* Number of step-kernel launches made by this context so far. */
lbm_status lbm_kernel_launches(lbm_ctx *ctx, long *launches);

/* ---- Batches of steady solves and the serving loop ---------------------------
 * A batch keeps many independent domains resident and advances all running
 * ones together: one launch of the batched step kernel is one step (Eq. 2) of
 * every running domain, the work list spanning all their (strip, row segment)
 * items.  A tick of K steps is replayed from one captured CUDA graph (or run
 * by the persistent kernel, option "persistent"); after each tick the
 * convergence residual (as in lbm_run_to_steady) of every running domain whose
 * own check interval has passed is computed in FP64, and converged, diverged or
 * exhausted domains retire while the others go on (per-domain masking).
 * Requests wait in a queue and are admitted, in arrival order or smallest
 * first (option "admission"), when their device footprint fits the batch's
 * memory budget (and the option "max_running_cells"); finished requests keep
 * their populations until released.
 * Storage and collision kernel are per batch; the device memory of a batch is
 * allocated with cudaMalloc.  A domain's results do not depend on the other
 * domains in the batch.  submit/poll/fields/release may be called from any
 * thread while the engine runs (lbm_batch_start) or between lbm_batch_run calls. */
typedef struct lbm_batch lbm_batch;
enum { LBM_REQ_QUEUED = 0, LBM_REQ_RUNNING = 1, LBM_REQ_CONVERGED = 2, LBM_REQ_NOT_CONVERGED = 3,
       LBM_REQ_DIVERGED = 4, LBM_REQ_FAILED = 5, LBM_REQ_CANCELLED = 6 };
typedef struct {
    int nx, ny;              /* >= 3                                                 */
    double nu, gamma, U;     /* as lbm_create                                        */
    lbm_boundaries bnd;      /* sides and optional host solid mask (copied at submit) */
    int use_bnd;             /* 0: lid-driven cavity with lid speed U                */
    double fx, fy;           /* uniform body force                                   */
    double tol;              /* steady when r < tol between checks (> 0)              */
    long max_steps;          /* give up after this many steps (> 0)                  */
    long check_every;        /* steps between this request's convergence checks:     */
                             /* 0 = the batch's check_every, else rounded up to a    */
                             /* multiple of it (a slow domain's residual is then     */
                             /* taken over a longer interval, as lbm_run_to_steady   */
                             /* with that check_every); a check is also made when     */
                             /* max_steps is reached                                 */
} lbm_request;
typedef struct {
    int state;               /* LBM_REQ_*                                             */
    long steps;              /* steps taken                                          */
    double residual;         /* last convergence residual                            */
    double t_submit, t_admit, t_done;  /* seconds since the batch was created        */
} lbm_result;

/* storage: LBM_STORAGE_*; gi_mode: LBM_GI_*; hbm_budget_bytes bounds the sum of
 * the admitted requests' footprints (2 population buffers + residual snapshot
 * + mask and its row table, + the window sums below).  Options: "check_every" (K, even, default
 * 1000: steps between convergence checks, one CUDA graph of K launches),
 * "rows_per_item" (rows of a warp's work item; 0 = chosen by timing a few
 * steps whenever the running work has changed by more than 2x), "persistent"
 * (-1, default: chosen by the same timing; 0: a launch per step and force
 * variant, replayed from the tick's CUDA graph; 1: the persistent kernel, the
 * steps between two velocity samples in one cooperative launch with a bounded
 * grid barrier between steps, launched directly -- FP32/FP16/BF16 storage,
 * full GI kernel, running domains of one force variant; otherwise per-step
 * launches),
 * "admission" (0, default: first come first served; 1: the smallest queued
 * domain, by cell count, first -- the oldest among equals), "max_running_cells"
 * (0, default: no cap; else a request is admitted only while the running
 * domains and it hold at most this many cells, or when nothing runs: the cap
 * bounds the time of a step of the batch and so of a tick, which is the
 * granularity of admission, retirement and cancellation),
 * "stochastic_rounding" (as lbm_set_option, default 1, for domains admitted
 * afterwards), "average_samples" (M, set before the first submit; default 16
 * for FP16/BF16 storage, 0 otherwise): the velocity of every domain is sampled
 * M times per check interval (every K/M steps) and the convergence residual
 * compares these window averages instead of single states; a finished request
 * returns the velocity average of its last window (lbm_batch_fields: rho is the
 * final state's).  Stochastic rounding leaves an unbiased noise on a 16-bit
 * state near its steady state, which the average removes from the residual and
 * the result.  The error status of create is LBM_ERR_INVALID for bad
 * arguments, LBM_ERR_CUDA without a device, LBM_ERR_OOM when the batch's own
 * tables cannot be allocated.  A request is initialised at rest (rho = 1,
 * u = 0); its step count includes autotuning steps. */
lbm_status lbm_batch_create(size_t hbm_budget_bytes, int storage, int gi_mode, lbm_batch **out);
lbm_status lbm_batch_set_option(lbm_batch *b, const char *key, double value);
lbm_status lbm_batch_submit(lbm_batch *b, const lbm_request *req, long *id);   /* non-blocking */
lbm_status lbm_batch_poll(lbm_batch *b, long id, int *done, lbm_result *res);  /* done: finished */
lbm_status lbm_batch_fields(lbm_batch *b, long id, double *rho, double *ux, double *uy);
lbm_status lbm_batch_release(lbm_batch *b, long id);  /* frees a finished request's memory */
/* Cancel a request: a queued one leaves the queue at once, a running one stops
 * at the end of the engine tick in progress (a request that converges in that
 * tick keeps its result); either ends LBM_REQ_CANCELLED and keeps its state
 * until released.  The other requests are unaffected (their arithmetic does not
 * depend on the mix).  LBM_ERR_INVALID for an unknown or finished request. */
lbm_status lbm_batch_cancel(lbm_batch *b, long id);
/* Run engine ticks on the calling thread until nothing is queued or running,
 * or wall_seconds (> 0) have passed. */
lbm_status lbm_batch_run(lbm_batch *b, double wall_seconds);
lbm_status lbm_batch_start(lbm_batch *b);  /* engine on a background thread */
lbm_status lbm_batch_stop(lbm_batch *b);
/* stats: {cell updates, step launches, ticks, running, queued, device bytes in use} */
lbm_status lbm_batch_stats(lbm_batch *b, double stats[6]);
void lbm_batch_destroy(lbm_batch *b);

/* ---- Convergence sums without any device allocation -------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot let the library call cudaMalloc while they run: applications whose
 * device memory is all handed out by their own pool or arena, loops that must
 * not pay or risk an allocation between steps, and code recorded into a CUDA
 * graph, where an allocation call cannot be recorded.  The caller passes its
 * own device buffers; the reduction's scratch is a fixed array inside the
 * library (2.5 MiB on every GPU that loads the library, held until exit).
 *
 * Computes, over the fluid cells of the population array f_dev (device,
 * layout [9][ny][pitch], deviations f - w of the given storage type), the same
 * five FP64 sums as lbm_residual: {sum |u - u_snap|^2, sum |u|^2, sum rho,
 * sum rho ux, sum rho uy}, with rho u = sum f e - F/(2 gamma); then replaces
 * the snapshot snap_ux_dev / snap_uy_dev (device, nx*ny doubles, index
 * y*nx + x) by u.  sums_dev (device, 5 doubles) receives the sums.  Work is
 * queued on `stream` (a cudaStream_t; NULL = the default stream) and nothing
 * is allocated, freed or synchronised.
 *
 * The first call on a device (and the first after a cudaDeviceReset of it)
 * looks up the scratch array's device address in the current context; make
 * that call before any stream capture.  First calls from several host threads
 * at once are safe.  All calls share the one array: calls that overlap on the
 * GPU race, so order them (e.g. one stream).  nx*ny above
 * LBM_NOALLOC_MAX_CELLS gives LBM_ERR_INVALID. */
#define LBM_NOALLOC_MAX_PARTIALS 65536
#define LBM_NOALLOC_MAX_CELLS (65536LL * 256LL)
typedef struct {
    int nx, ny;                /* cells                                           */
    int pitch;                 /* row stride of each plane in elements, >= nx      */
    int storage;               /* LBM_STORAGE_* element type of f_dev              */
    double gamma;              /* preconditioning parameter                        */
    double fx, fy;             /* uniform body force (0 if none)                   */
    const uint8_t *solid_dev;  /* optional device mask [ny][pitch], non-zero solid */
} lbm_population_desc;
lbm_status lbm_residual_sums_noalloc(const lbm_population_desc *desc, const void *f_dev, double *snap_ux_dev,
                                     double *snap_uy_dev, double *sums_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif
