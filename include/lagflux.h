/*
 * lagflux.h -- C ABI of the GB300 (sm_103a) Lagrange-flux solver.
 *
 * The library advances the 1D/2D/3D compressible Euler equations with a
 * perfect-gas equation of state (arXiv:1607.08710, Sec. 3, eq. 1) by the
 * second-order Lagrange-flux scheme of Sec. 4: MUSCL reconstruction of the
 * primitive variables with a limited slope (eq. "sweby"), the Lagrangian
 * HLL / acoustic interface solver (Sec. 4.1, eqs. 13-14), the upwind
 * Lagrange flux (eq. 12) and the two-stage Heun time integrator (Sec. 4,
 * steps 1-11) under a CFL time step.  A state may also carry up to
 * LF_MAX_SPECIES transported mass fractions y_k (Sec. 5: the conservative
 * form d(rho y_k)/dt + div(rho y_k u) = 0), reconstructed and upwinded with
 * the gas state by the same Lagrange flux.
 *
 * Conventions shared by every entry point:
 *   - Mesh: a uniform Cartesian mesh of nx x ny (x nz) cells on
 *     [xmin, xmax] x [ymin, ymax] (x [zmin, zmax]); ny == 1 in 1D, nz == 1
 *     (or 0) below 3D.  3D applies the same face formulas on a third axis
 *     (the finite-volume form of Sec. 4 holds for any cell shape).
 *   - Fields are passed as separate planes of nx*ny elements, x fastest
 *     (element (i, j) at index j*nx + i), of the configured precision:
 *     double for LF_FP64, float for LF_FP32.  The conservative planes are
 *     (rho, rho u, rho v, rho E); the primitive planes (rho, u, v, p).
 *     Species planes (nspecies > 0) are passed as one buffer of nspecies
 *     consecutive planes (nx*ny*nz values each in 3D): partial densities
 *     rho y_k or mass fractions y_k.
 *     The whole-state calls (lf_set_conservative and friends) take one
 *     buffer of all nfields planes: (rho, rho u, rho v, [rho w,] rho E,
 *     rho y_k) or (rho, u, v, [w,] p, y_k), nfields = 4 (5 in 3D) + nspecies,
 *     each plane nx*ny*nz values, x fastest, then y, then z.
 *   - Ownership: the caller owns every buffer it passes and keeps it; the
 *     library copies in and out and never retains a caller pointer.  The
 *     context owns its device state, scratch and scalars.
 *   - `on_device` = 1: the pointers are device pointers (e.g. the data_ptr of
 *     a contiguous CUDA tensor) readable on the context's device; 0: host
 *     pointers.  Host transfers complete before the call returns.
 *   - Streams: all device work is enqueued on the stream given to lf_init
 *     (NULL = the legacy default stream).  Calls return once the work is
 *     enqueued, except where they must return a host value (dt_out,
 *     steps_done, t_out, sums) or touch host memory; those synchronise the
 *     stream first.
 *   - Errors: no call aborts or throws.  Invalid arguments return
 *     LF_ERR_ARG and change nothing.  A CUDA failure returns LF_ERR_CUDA.
 *     Device kernels never trap: a non-positive density or pressure, or a
 *     non-finite wave speed, sets a sticky flag in the context; the next
 *     synchronising call returns LF_ERR_NONPHYSICAL and the time loop stops
 *     advancing (dt becomes 0).  lf_last_error describes the last failure.
 *   - Thread safety: one context must not be used from two host threads at
 *     once; distinct contexts are independent.
 */
#ifndef LAGFLUX_H
#define LAGFLUX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lf_status {
  LF_OK = 0,
  LF_ERR_ARG = 1,         /* invalid argument or configuration */
  LF_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed */
  LF_ERR_OOM = 3,         /* device memory allocation failed */
  LF_ERR_NONPHYSICAL = 4, /* non-positive rho or p, or non-finite wave speed */
  LF_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  LF_ERR_STATE = 6        /* call out of order (e.g. step before a state was set) */
} lf_status;

/* Slope limiters: Sweby's phi(a,b) of Sec. 4 (eq. "sweby") with beta in
 * [1, 2]; beta = 1 is minmod (Sec. 4.2, last tube).  Van Leer's
 * (ab>0) 2ab/(a+b) is the one limiter offered beyond the paper's. */
enum { LF_LIMITER_MINMOD = 0, LF_LIMITER_SWEBY = 1, LF_LIMITER_VANLEER = 2 };
/* Boundary conditions: transmissive (two ghost layers copying the boundary
 * cell) or periodic (wrap-around). */
enum { LF_BC_TRANSMISSIVE = 0, LF_BC_PERIODIC = 1 };
/* Arithmetic precision of the state, fluxes and updates.  In LF_FP32 the
 * time, dt, the dt reduction's input and the conservation sums stay FP64. */
enum { LF_FP64 = 0, LF_FP32 = 1 };
/* Interface solver: eqs. (13)-(14) with a = max(c_L, c_R) (default), or the
 * acoustic solver with per-side impedances Z_k = rho_k c_k. */
enum { LF_RIEMANN_MAXC = 0, LF_RIEMANN_PER_SIDE = 1 };
/* Time integrator (Sec. 4 leaves the Runge-Kutta family open): the Heun scheme of Sec. 4 (0 or 2),
 * or the third-order strong-stability-preserving Runge-Kutta scheme of Shu
 * and Osher (3), U1 = U + dt L(U), U2 = 3/4 U + 1/4 (U1 + dt L(U1)),
 * U' = 1/3 U + 2/3 (U2 + dt L(U2)).  SSP-RK3 needs one more state buffer and
 * is offered by lf_init contexts only. */
enum { LF_TIME_HEUN = 2, LF_TIME_SSPRK3 = 3 };
/* Largest number of transported mass fractions (lf_config.nspecies). */
#define LF_MAX_SPECIES 2

typedef struct lf_config {
  int32_t dim;       /* 1, 2 or 3 */
  int32_t nx, ny;    /* cells per direction; ny == 1 when dim == 1.  A field plane
                        (rows padded to 128 bytes) holds fewer than 2^31 elements:
                        e.g. at most 46336 x 46340 cells in FP32 (LF_ERR_ARG otherwise) */
  int32_t limiter;   /* LF_LIMITER_* */
  int32_t bc;        /* LF_BC_* */
  int32_t precision; /* LF_FP64 or LF_FP32 */
  int32_t riemann;   /* LF_RIEMANN_* */
  int32_t device;    /* CUDA device ordinal */
  int32_t time_order; /* LF_TIME_* (0 = LF_TIME_HEUN) */
  int32_t nspecies;  /* transported mass fractions, 0 .. LF_MAX_SPECIES (Sec. 5);
                        lf_init contexts (0 for batches, the adjoint and
                        lf_step_noalloc) */
  double xmin, xmax; /* domain in x */
  double ymin, ymax; /* domain in y (ignored in 1D) */
  double gamma;      /* ratio of specific heats, 1 < gamma <= 3 (Sec. 3) */
  double cfl;        /* CFL number, 0 < cfl <= 1 */
  double beta;       /* Sweby coefficient, 1 <= beta <= 2 (LF_LIMITER_SWEBY) */
  int32_t nz;        /* cells in z (dim == 3); 0 or 1 otherwise */
  int32_t tile_rows; /* rows per tile of the 2D stage kernels, 1 .. 4096; 0: chosen
                        by lf_init from the mesh size and the GPU's SM count (64-row
                        tiles unless that leaves the GPU short of work).  A launch
                        shape only: results do not depend on it, bit for bit. */
  double zmin, zmax; /* domain in z (dim == 3) */
} lf_config;

typedef struct lf_ctx lf_ctx;

/* Creates a solver for one mesh.  `stream` is a cudaStream_t (NULL: default
 * stream).  Allocates the device state (nfields planes), one
 * intermediate Heun state (as many planes; two for SSP-RK3) and a few
 * scalars.  The species planes start at 0.  *out is set only on LF_OK. */
lf_status lf_init(const lf_config* cfg, void* stream, lf_ctx** out);

/* Frees everything the context owns.  NULL is ignored. */
void lf_destroy(lf_ctx* ctx);

/* Copies in a conservative state (rho, rho u, rho v, rho E); in 1D rhov may
 * be NULL (taken as 0).  Resets t to 0 and the step count to 0 and computes
 * the wave-speed maximum for the first dt (Sec. 4, Heun step 1).  The
 * species planes are left as they are. */
lf_status lf_set_state(lf_ctx* ctx, const void* rho, const void* rhou, const void* rhov,
                       const void* rhoE, int on_device);

/* As lf_set_state from primitive planes (rho, u, v, p); the conversion uses
 * the perfect-gas EOS of eq. (1) and runs on the device. */
lf_status lf_set_primitive(lf_ctx* ctx, const void* rho, const void* u, const void* v,
                           const void* p, int on_device);

/* Copies out the current conservative state; rhov may be NULL in 1D. */
lf_status lf_get_state(lf_ctx* ctx, void* rho, void* rhou, void* rhov, void* rhoE,
                       int on_device);

/* Copies out the current primitive state (rho, u, v, p) via eq. (1). */
lf_status lf_get_primitive(lf_ctx* ctx, void* rho, void* u, void* v, void* p, int on_device);

/* Whole-state transfers for any dim and species count (the only state calls
 * of 3D contexts; lf_set_state / lf_set_primitive / lf_get_state /
 * lf_get_primitive return LF_ERR_ARG there).  U / q hold all nfields planes
 * (see the conventions above).  The set calls reset t and the step count
 * and compute the wave-speed maximum for the first dt, like lf_set_state;
 * the primitive conversions use eq. (1) and run on the device. */
lf_status lf_set_conservative(lf_ctx* ctx, const void* U, int on_device);
lf_status lf_get_conservative(lf_ctx* ctx, void* U, int on_device);
lf_status lf_set_primitives(lf_ctx* ctx, const void* q, int on_device);
lf_status lf_get_primitives(lf_ctx* ctx, void* q, int on_device);

/* Species (Sec. 5), for contexts with nspecies > 0 (LF_ERR_ARG otherwise).
 * Partial densities: rho_y holds nspecies planes of rho y_k, copied in or
 * out as they are.  Mass fractions: y holds nspecies planes of y_k; setting
 * stores rho y_k = rho * y_k with the density of the current state (so call
 * it after lf_set_state / lf_set_primitive), getting returns
 * (rho y_k) / rho.  The species never enter the pressure, the sound speed or
 * dt, so none of these calls touches t, the step count or the dt scalars. */
lf_status lf_set_partial_densities(lf_ctx* ctx, const void* rho_y, int on_device);
lf_status lf_get_partial_densities(lf_ctx* ctx, void* rho_y, int on_device);
lf_status lf_set_mass_fractions(lf_ctx* ctx, const void* y, int on_device);
lf_status lf_get_mass_fractions(lf_ctx* ctx, void* y, int on_device);

/* One Heun step (Sec. 4, steps 1-11) with the CFL time step
 * dt = cfl / max_K[(|u|+c)/dx + (|v|+c)/dy]  (1D: cfl / max_K[(|u|+c)/dx]).
 * dt_out (nullable) receives the dt used; passing it synchronises. */
lf_status lf_step(lf_ctx* ctx, double* dt_out);

/* One Heun step with a caller-chosen dt > 0 (e.g. to replay a recorded dt
 * sequence).  Does not synchronise. */
lf_status lf_step_fixed(lf_ctx* ctx, double dt);

/* Advances until t reaches t_end (t_end <= 0: no final time) or max_steps
 * steps are done.  The last dt is clipped so that t lands on t_end.  dt stays
 * on the device; steps are issued in batches of 32, each one replay of a
 * CUDA graph recorded on first use (direct launches while stage tracing is
 * on), and the host polls t only between batches.
 * steps_done and t_out are nullable; the call synchronises. */
lf_status lf_run(lf_ctx* ctx, double t_end, int32_t max_steps, int32_t* steps_done, double* t_out);

/* Current time and completed step count (synchronises). */
lf_status lf_get_time(lf_ctx* ctx, double* t, int64_t* steps);

/* Compensated (Neumaier) FP64 sums of the nfields conservative fields
 * (rho, rho u, rho v, [rho w,] rho E, rho y_k) over all cells, in a fixed
 * (deterministic) reduction order.  out holds nfields doubles;
 * synchronises. */
lf_status lf_conservation_sums(lf_ctx* ctx, double* out);

/* Waits for the context's stream and reports any device-side error flag. */
lf_status lf_sync(lf_ctx* ctx);

/* Launch shape of the stage kernels: rows per tile of the y-march (2D) or
 * planes per z-tile (3D).  lf_init picks it from the mesh size and the SM
 * count unless lf_config.tile_rows sets it.  Results do not depend on it,
 * bit for bit.  lf_set_tile_rows: 1 <= rows <= 4096, LF_ERR_ARG for 1D
 * meshes; synchronises.  lf_get_tile_rows: the current value (0 in 1D). */
lf_status lf_set_tile_rows(lf_ctx* ctx, int32_t rows);
lf_status lf_get_tile_rows(lf_ctx* ctx, int32_t* rows);

/* Times trial_steps CFL steps (after one warm-up step) for each candidate
 * tile height (2D: 4, 8, 16, 32, 64, 128 rows; 3D: 8, 16, 32, 64 planes) on
 * the current state, keeps the fastest and restores the state, t, dt and the
 * step count (the trial steps leave no trace).  Allocates a temporary copy of
 * the state.  chosen_rows (nullable) receives the pick.  Needs a state
 * (LF_ERR_STATE) and a 2D or 3D mesh (LF_ERR_ARG).  Synchronises. */
lf_status lf_autotune(lf_ctx* ctx, int32_t trial_steps, int32_t* chosen_rows);

/* Stage tracing.  While enabled, every predictor (stage 0) and corrector
 * (stage 1) kernel launch is bracketed by CUDA events recorded on the
 * context's stream.  lf_profile_read synchronises and returns, per stage,
 * the summed device time in milliseconds and the number of launches timed
 * since tracing was (re-)enabled.  Enabling resets the accumulators.  Timing
 * adds two event records per launch; leave it off for throughput runs. */
lf_status lf_profile_enable(lf_ctx* ctx, int enable);
lf_status lf_profile_read(lf_ctx* ctx, double ms[2], int64_t launches[2]);

/* ------------------------------------------------------------------------
 * Discrete adjoint of the Heun/RK2 step (Sec. 4) with the dt sequence frozen,
 * for 2D meshes and the eqs. 13-14 interface solver.  Limiter branches are
 * differentiated piecewise; at non-smooth points max/min take the first
 * argument on ties, the limiter has zero derivative where ab <= 0, and the
 * upwind side follows the sign of u*.
 *
 * The paper states the step (Sec. 4, steps 1-11) but no adjoint; the calls
 * below differentiate exactly that step.  The adjoint needs dJ/dU(T), which
 * for most objectives depends on U(T), so the work is split in two calls:
 * lf_adjoint_forward (run and record) and lf_adjoint_backward (sweep back
 * from a given dJ/dU(T)).  lf_adjoint runs both in one call for objectives
 * whose dJ/dU(T) is known before the run (linear functionals of U(T), or a
 * cotangent computed from an earlier run of the same state).
 * ------------------------------------------------------------------------ */

/* Runs nsteps CFL steps from the context's current state (as lf_step does),
 * keeping a checkpoint of the state every ceil(sqrt(nsteps)) steps and the
 * dt of every step; the context ends at the final state U(T).  Allocates the
 * checkpoints (ceil(nsteps / ceil(sqrt(nsteps))) states), one segment of
 * recomputed states and adjoint work buffers; they are kept for reuse until
 * lf_destroy.  dts_out (nullable, host, nsteps doubles) receives the dt
 * sequence.  Synchronises. */
lf_status lf_adjoint_forward(lf_ctx* ctx, int32_t nsteps, double* dts_out);

/* Given lambda_T = dJ/dU(T) (4 dense planes of the configured precision,
 * conservative variables, x fastest), computes dJ/dU(0) of the last recorded
 * forward run by sweeping its checkpoints backwards.
 * grad_U0 (nullable): 4 dense planes of dJ/dU(0).
 * grad_q0 (nullable): 4 dense planes of dJ/d(rho, u, v, p) at t = 0.
 * on_device: 1 = the three buffers are device pointers, 0 = host pointers.
 * The context's state (U(T)) is left unchanged.  Synchronises. */
lf_status lf_adjoint_backward(lf_ctx* ctx, const void* lambda_T, void* grad_U0, void* grad_q0, int on_device);

/* lf_adjoint_forward(ctx, nsteps, dts_out) followed by
 * lf_adjoint_backward(ctx, lambda_T, grad_U0, grad_q0, on_device): the
 * gradient of an objective with the given dJ/dU(T) with respect to the
 * context's current state.  The context ends at U(T).  Synchronises. */
lf_status lf_adjoint(lf_ctx* ctx, int32_t nsteps, const void* lambda_T, void* grad_U0, void* grad_q0,
                     double* dts_out, int on_device);

/* How the reverse sweep forms the forward quantities it differentiates (the
 * primitives, limited slopes and limiter derivatives of a state).
 * LF_ADJOINT_PASSES_TABLES: one prep pass per state writes them to tables
 * (28 values per cell) that the face and cell passes read;
 * LF_ADJOINT_PASSES_DIRECT: every face and cell thread recomputes them from
 * the state.  The two give the same derivative up to rounding order.
 * LF_ADJOINT_PASSES_AUTO (default): tables in FP64 (divisions dominate
 * there), direct in FP32 (the extra passes and table traffic dominate). */
enum { LF_ADJOINT_PASSES_AUTO = 0, LF_ADJOINT_PASSES_TABLES = 1, LF_ADJOINT_PASSES_DIRECT = 2 };
lf_status lf_adjoint_set_passes(lf_ctx* ctx, int32_t passes);

/* ------------------------------------------------------------------------
 * Batched mode: many independent 2D meshes of uneven sizes advanced together
 * by the same Heun/RK2 Lagrange-flux step (Sec. 4), each problem with its own
 * CFL time step, time and step count.  One persistent kernel launch per
 * stage covers all problems; the step loop is recorded once as a CUDA graph.
 * ------------------------------------------------------------------------ */
typedef struct lf_batch lf_batch;

/* cfgs[0..nprob-1]: one configuration per problem.  dim must be 2; nx, ny
 * and the domain may differ; limiter, bc, precision, riemann, gamma, cfl,
 * beta and device must be equal across problems.  Allocates two state pools
 * (sum over problems of 4 planes, rows padded to 128 bytes), per-problem
 * scalars and the work-unit table. */
lf_status lf_batch_init(const lf_config* cfgs, int32_t nprob, void* stream, lf_batch** out);
void lf_batch_destroy(lf_batch* b);

/* Sets problem p's state from primitive planes (rho, u, v, p), each
 * cfgs[p].nx * cfgs[p].ny elements, x fastest; resets that problem's time and
 * step count and computes its first wave-speed maximum. */
lf_status lf_batch_set_primitive(lf_batch* b, int32_t p, const void* rho, const void* u, const void* v,
                                 const void* pr, int on_device);

/* Copies out problem p's conservative planes. */
lf_status lf_batch_get_state(lf_batch* b, int32_t p, void* rho, void* rhou, void* rhov, void* rhoE,
                             int on_device);

/* Enqueues nsteps Heun steps of every problem.  use_graph = 1: the loop of
 * nsteps steps is recorded once as a CUDA graph (re-recorded when nsteps or
 * the tile height changes) and replayed on the context's stream; 0: direct
 * launches.  Does not synchronise.  Every problem must have a state. */
lf_status lf_batch_run(lf_batch* b, int32_t nsteps, int32_t use_graph);

/* Times trial_steps steps for each candidate tile height (rows per work
 * unit: 16, 24, 32, 48, 64, 96, 128) on the current states, keeps the
 * fastest and restores the states and times to what they were (the trial
 * steps leave no trace).  Allocates a temporary copy of the state pool.
 * chosen_rows (nullable) receives the pick.  Synchronises. */
lf_status lf_batch_autotune(lf_batch* b, int32_t trial_steps, int32_t* chosen_rows);

/* Sets the tile height directly (1 <= rows <= 4096). */
lf_status lf_batch_set_rows(lf_batch* b, int32_t rows);

/* Per-problem time and step count (arrays of nprob, nullable); synchronises
 * and returns LF_ERR_NONPHYSICAL if any problem has raised a device error. */
lf_status lf_batch_get_times(lf_batch* b, double* t, int64_t* steps);

/* Runs nsteps Heun steps of every problem with direct launches (no graph),
 * each stage launch bracketed by CUDA events on the batch's stream, and
 * returns in ms[0] / ms[1] the summed device time of the predictor and
 * corrector launches.  The problems advance as with lf_batch_run.
 * Synchronises after every step. */
lf_status lf_batch_profile(lf_batch* b, int32_t nsteps, double ms[2]);

/* Description of the last failure on this batch (NULL: the last failed
 * lf_batch_init). */
const char* lf_batch_last_error(const lf_batch* b);

/* One Heun step that allocates no device memory (the paper has no
 * counterpart; this is a deployment convenience).  For callers that must not
 * call cudaMalloc -- code living inside another framework's memory manager,
 * code that may not allocate in a time-critical loop (cudaMalloc/cudaFree can
 * synchronise the device), hosts that reserve all GPU memory up front -- and
 * so cannot use lf_init.  The predictor state U* and the step's scalars live
 * in one static device array compiled into the library
 * (LF_NOALLOC_SCRATCH_BYTES, held on every GPU that loads the library until
 * the process exits).
 *   cfg    : mesh and scheme, as for lf_init; nx*ny must not exceed
 *            LF_NOALLOC_MAX_CELLS, else LF_ERR_ARG and nothing is launched.
 *   U_in   : device buffer of 4 dense planes (rho, rho u, rho v, rho E), each
 *            nx*ny elements of the configured precision, x fastest; read only.
 *   U_out  : device buffer of the same layout receiving U^{n+1}; may equal
 *            U_in (in-place step) but must not partially overlap it.
 *   dt     : > 0 uses this time step; <= 0 uses the CFL time step of U_in.
 *   dt_used: nullable; if given, the call synchronises `stream`, stores the dt
 *            used and returns LF_ERR_NONPHYSICAL if the new state has a
 *            non-positive density or pressure.  If NULL the call only
 *            enqueues and reports no device-side error.
 *   stream : cudaStream_t (NULL: default stream) on device cfg->device.
 * On LF_ERR_NONPHYSICAL, and whenever dt_used is NULL and U_in is not a
 * valid state, U_out is unspecified: a non-physical input or a bad CFL dt
 * stops the step before the update, so U_out may keep what it held before
 * the call.  Only LF_OK with dt_used given certifies U_out.
 * The first successful call on a device looks up the array's device address
 * (once per device; a failed lookup is retried by the next call); make that
 * first call before any stream capture: a first call on a capturing stream
 * returns LF_ERR_ARG.  All calls share
 * the array: calls whose GPU work overlaps (e.g. on two streams) race.
 * Error text: lf_last_error(NULL). */
#define LF_NOALLOC_MAX_CELLS (1LL << 18)
#define LF_NOALLOC_SCRATCH_BYTES (256 + 4 * 8 * LF_NOALLOC_MAX_CELLS)
lf_status lf_step_noalloc(const lf_config* cfg, const void* U_in, void* U_out, double dt, double* dt_used,
                          void* stream);

/* ------------------------------------------------------------------------
 * Measurement helper (the paper has no counterpart: its roofline analysis is
 * for multicore CPUs).  Measures the arithmetic peak that the ALU rooflines
 * of the stage kernels are taken against: eight independent fused
 * multiply-add chains per thread over 8 CTAs of 256 threads per SM, the
 * iteration count calibrated to about target_ms per launch, best of three
 * timed launches (CUDA events) after two calibration launches.
 *   device   : CUDA device ordinal (made current for the call, then restored).
 *   kind     : LF_PEAK_FP64 (DFMA), LF_PEAK_FP32 (FFMA) or
 *              LF_PEAK_FP32_PAIRED (the paired FP32 FMA the FP32 stage
 *              kernels use: two lanes per instruction).
 *   target_ms: in (0, 1000].
 *   tflops   : receives the measured rate, counting a fused multiply-add as
 *              two flops.
 * Allocates and frees a small result buffer, a stream and two events;
 * synchronises.  The SM clock is whatever the GPU runs at: sample it beside
 * the call to compare with a nominal rate. */
enum { LF_PEAK_FP64 = 0, LF_PEAK_FP32 = 1, LF_PEAK_FP32_PAIRED = 2 };
lf_status lf_measure_peak(int32_t device, int32_t kind, double target_ms, double* tflops);

/* Human-readable name of a status code (static storage). */
const char* lf_status_string(lf_status s);

/* Description of the last failure on this context (static per context;
 * valid until the next call on it).  NULL ctx: the last lf_init or
 * lf_step_noalloc failure. */
const char* lf_last_error(const lf_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LAGFLUX_H */
