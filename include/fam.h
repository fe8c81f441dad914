/*
 * fam.h -- C ABI of the B300 (sm_103a) library for the time step of the
 * compact finite-average-moment (FAM) schemes with single-step oscillation
 * elimination (Fan & Wu, "Compact Finite-Average-Moment Schemes with
 * Single-Step Oscillation Elimination for Hyperbolic Conservation Laws").
 *
 * Problem statement (Sec. 2.1, eq. 1dHCLS; Sec. 2.2, eq. 10): a scalar law or
 * the Euler equations (Sec. 2.3) on a uniform Cartesian mesh of [x0,x1] or
 * [x0,x1]x[y0,y1], order k = 3..6, boundary condition, end time T and CFL
 * number (Sec. 4, "Time stepping").  The evolved state is the P1 moment
 * state: per cell and conserved component the cell average and the scaled
 * first moment(s) (Sec. 2.1 / 2.2).
 *
 * STATE LAYOUT (all entry points that take a state): a dense array
 *     U[c][m][j][i]    (1D: U[c][m][i])
 * c = conserved component (scalar: 1; Euler 1D: rho, rho u, E; Euler 2D:
 * rho, rho u, rho v, E), m = 0 cell average, 1 scaled x-moment
 * (1/|I| int u (x-x_i)/dx), 2 scaled y-moment (2D); j = row (y), i = column
 * (x).  Element type: double for precision 64, float for precision 32.
 *
 * OWNERSHIP: the library owns all device memory of a handle; buffers passed
 * by the caller are only read or written during the call (host buffers) or
 * during the call's stream work (device buffers).  A handle is not
 * thread-safe.  Device pointers must be on the handle's device.
 *
 * ERRORS: every call returns a fam_status; no call aborts the process.
 * fam_last_error() returns a message for the last failing call of a handle.
 * Kernels flag non-finite states, non-physical averages (rho <= 0 or
 * p <= 0) and bounded-wait timeouts in a device status word; fam_sync()
 * reports them as FAM_E_NONPHYSICAL / FAM_E_TIMEOUT.
 */
#ifndef FAM_H
#define FAM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fam_handle* fam_t;

typedef enum {
  FAM_OK = 0,
  FAM_E_INVAL = 1,        /* invalid argument */
  FAM_E_NOMEM = 2,        /* device allocation failed */
  FAM_E_CUDA = 3,         /* CUDA runtime / driver error */
  FAM_E_NONPHYSICAL = 4,  /* non-finite or non-physical state detected */
  FAM_E_TIMEOUT = 5,      /* a kernel's bounded wait gave up */
  FAM_E_STATE = 6,        /* call out of order (e.g. step before set_state) */
  FAM_E_UNSUPPORTED = 7   /* option combination not built */
} fam_status;

/* FAM_BUCKLEY: the Buckley-Leverett equation of Example 4.3,
 * f(u) = 4u^2 / (4u^2 + (1-u)^2), 1D only; every wave speed it uses is the
 * bound max |f'| = 2.33203... (f' vanishes at u = 0 and 1). */
typedef enum { FAM_ADVECTION = 0, FAM_BURGERS = 1, FAM_EULER = 2, FAM_BUCKLEY = 3 } fam_equation;
/* Side conditions (Remark in Sec. 2.3).  fam_create takes PERIODIC or
 * OUTFLOW for every side; fam_set_bc sets any of the four per side. */
typedef enum { FAM_BC_PERIODIC = 0, FAM_BC_OUTFLOW = 1, FAM_BC_REFLECTIVE = 2, FAM_BC_INFLOW = 3 } fam_bc;

typedef struct {
  int d;           /* dimension: 1 or 2 */
  int nx, ny;      /* cells per direction (ny ignored for d = 1); >= 4 */
  double x0, x1;   /* domain [x0, x1] */
  double y0, y1;   /* domain [y0, y1] (d = 2) */
} fam_grid;

/* Create a solver.  k in {3,4,5,6} selects FAM-k (Sec. 2.4).  gamma: ratio of
 * specific heats for FAM_EULER (the paper uses 1.4), advection speed a in
 * both directions for FAM_ADVECTION (change per direction with the options
 * "ax"/"ay"), ignored for FAM_BURGERS and FAM_BUCKLEY.  bc applies on every side (Remark in
 * Sec. 2.3: periodic, or outflow ghost cells copying average and moments).
 * precision: 64 (FP64) or 32 (FP32).  stream: a cudaStream_t to run on, or
 * NULL for a stream the library creates.  On success *out receives the
 * handle; the state is undefined until fam_set_state().
 * Errors: FAM_E_INVAL (bad argument), FAM_E_NOMEM, FAM_E_CUDA,
 * FAM_E_UNSUPPORTED (FAM_BUCKLEY in 2D). */
fam_status fam_create(fam_t* out, const fam_grid* grid, int k, int equation, int bc, double gamma,
                      int precision, void* stream);

/* Set an option (before or between steps).  Keys:
 *   "oe_type"    0 = no OE, 1 = Type I (grid-wide mean and maximum deviation
 *                of the cell averages), 2 = Type II (default); Tab. sigma1d /
 *                sigma2d
 *   "gamma_k"    OE constant; <= 0 restores the paper's defaults (1D: 25 for
 *                k = 3,4 and 12.5 for k = 5,6; 2D: 25 and 15; Sec. 2.1/2.2)
 *   "oe_jump_q6" 2D k = 6 only: 1 (default) takes the OE jumps from the full
 *                auxiliary Q6, which reproduces the printed jump matrices
 *                (App. J); 0 takes them from p6 = Pi_5 Q6
 *   "smooth_dt"  1: time step with dx^(k/3) (smooth runs, Sec. 4); 0: dx
 *   "ax", "ay"   advection speeds (FAM_ADVECTION)
 *   "dt_max"     upper bound on the step size (<= 0: none)
 *   "tile2d"     2D tile shape of the stage / OE kernels: 0 = 32 x 8 (default),
 *                1 = 32 x 4, 2 = 16 x 8 cells (see fam_tune)
 *   "pp_limiter" FAM_BUCKLEY: 1 scales each stage's reconstruction
 *                towards the cell average until the check points below lie
 *                in [0, 1] (the bound-preserving form for this scalar).
 *                Euler: 1 turns on the BP/PP safeguard the paper
 *                applies after RK substeps in some tests (Sec. 2.3 remarks,
 *                Alg. 1; it cites its construction without defining it).
 *                Built as the Zhang-Shu scaling of every stage's
 *                reconstruction towards the cell average, so that density
 *                and pressure are admissible at the points of a
 *                Gauss-Lobatto decomposition of the average (3 points for
 *                k <= 4, 4 for k = 5, 6) and at the volume Gauss points; the
 *                CFL rule then takes its speeds at those points, and a
 *                forward-Euler step keeps the averages admissible for CFL
 *                numbers up to 1/6 (k <= 4) or 1/12 (k = 5, 6), stage by
 *                stage: a step whose stage averages leave the admissible set
 *                is discarded and retried with half the step size
 *                (fam_rejected_steps).  The final stage and the OE then run
 *                split; no adjoint.  0 (default): off, the scheme of the
 *                paper's tests without BP/PP
 *   "fused_oe"   2D only: 1 runs the final RK stage and the OE in one
 *                persistent launch (not in the paper: tiles of the final
 *                stage and, once the tiles around them are done, the OE of
 *                each tile, taken from an ordered task list; the final stage's
 *                output stays in L2 between the two); 0 (default) runs them
 *                as two kernels.  Results agree to rounding; Type-I OE
 *                (grid-wide statistics of the final stage) always runs split.
 *                fam_tune chooses it per problem
 *   "profile"    1: fam_step() brackets each of its four kernel launches with
 *                CUDA events (read with fam_profile); setting it resets the
 *                accumulated times
 * Errors: FAM_E_INVAL (unknown key or value), FAM_E_UNSUPPORTED. */
fam_status fam_set_option(fam_t h, const char* key, double value);

/* Boundary condition of one side (Remark in Sec. 2.3): side 0 = x-low,
 * 1 = x-high, 2 = y-low, 3 = y-high; bc: 0 periodic (both sides of a
 * direction), 1 outflow, 2 reflective wall (mirror image: the normal
 * momentum and the moment along the normal change sign), 3 inflow (ghost
 * averages = inflow_state[0..ncomp-1] in conservative variables, ghost
 * moments zero).  Sides are set one at a time, so the combination is
 * checked when a step, residual or OE next uses it: a periodic side whose
 * opposite side is not periodic gives FAM_E_INVAL there, and an inflow side
 * next to a reflective wall FAM_E_UNSUPPORTED (not built) unless the wall's
 * split part (fam_set_bc_split) covers their shared corner.  Errors here:
 * FAM_E_INVAL (side or bc out of range, y sides of a 1D grid, inflow
 * without a state). */
fam_status fam_set_bc(fam_t h, int side, int bc, const double* inflow_state);

/* Split side (2D; the double Mach reflection of Example 4.8 imposes the
 * post-shock state on the wall's part x < 1/6): the ghost cells of `side`
 * whose nearest interior cell along the side (row for sides 0/1, column for
 * sides 2/3) has its centre below `position` hold `state` (conservative
 * averages, zero moments); the rest of the side keeps the condition set by
 * fam_set_bc.  position at or below the side's start removes the split.
 * Kept when fam_set_bc changes the side's condition.  Errors: FAM_E_INVAL
 * (side out of range, a periodic side, no state), FAM_E_UNSUPPORTED (1D). */
fam_status fam_set_bc_split(fam_t h, int side, double position, const double* state);

/* Front condition of a y-side (2D; the top side of Example 4.8 follows the
 * exact motion of the incident shock): a ghost cell of `side` with centre
 * (x, y) holds `behind` if x < a + b y + c t and `ahead` otherwise
 * (conservative averages, zero moments), t the time of the state the kernel
 * reads: rewritten before every stage for its input's time (t, t + dt,
 * t + dt/2 in SSP-RK3; the OE reads the state at t + dt).  fam_residual and
 * fam_oe take the handle's current time.  The front side has no images
 * (code 4 in the side's condition).  The fused final stage + OE runs split
 * while a front side is set.  Errors: FAM_E_INVAL (a 1D grid, an x-side,
 * missing states). */
fam_status fam_set_bc_front(fam_t h, int side, double a, double b, double c, const double* behind,
                            const double* ahead);

/* Copy a state in (layout above).  on_device = 0: U is host memory;
 * 1: U is device memory of the handle's device.  Resets the clock to t = 0
 * and the step counter to 0.  Synchronous for host memory. */
fam_status fam_set_state(fam_t h, const void* U, int on_device);

/* Copy the current state out (layout above).  Synchronous for host memory;
 * for device memory the copy is ordered on the handle's stream. */
fam_status fam_get_state(fam_t h, void* U, int on_device);

/* Enqueue one time step (Alg. 1): the three SSP-RK3 stages of eq. (3)/(12)
 * and the end-of-step OE (eq. 9 / eq. 2dOE_sol, system forms of Sec. 2.3).
 * The step size follows the CFL rule of Sec. 4 from the maximum Rusanov
 * speed at the current cell averages, computed on the device (no host
 * synchronisation).  Asynchronous; call fam_sync() to wait and check. */
fam_status fam_step(fam_t h, double cfl);

/* Enqueue exactly nsteps steps as one CUDA graph launch (captured once per
 * distinct nsteps and replayed).  Asynchronous. */
fam_status fam_run_steps(fam_t h, long nsteps, double cfl);

/* Advance to time T (the last step is shortened to land on T), at most
 * max_steps steps if max_steps > 0.  Synchronous.  *nsteps_out (may be NULL)
 * receives the number of steps taken by this call. */
fam_status fam_run(fam_t h, double T, double cfl, long max_steps, long* nsteps_out);

/* Enqueue nsteps steps with prescribed step sizes dts[0..nsteps-1] (host
 * array) instead of the CFL rule -- e.g. to replay a recorded step-size
 * sequence.  Asynchronous.  With "pp_limiter", a step the safeguard rejects
 * (fam_rejected_steps) leaves state and clock as they were and the next
 * prescribed size follows: the rejected size is not retried. */
fam_status fam_run_fixed(fam_t h, long nsteps, const double* dts);

/* Autotuner (not in the paper): times probe_steps steps of each 2D tile
 * shape, with the final stage and OE split and fused (option "fused_oe";
 * split only for Type-I OE or with "pp_limiter"), on the handle's current
 * state (restored afterwards, clock included), keeps the fastest and
 * appends it to cache_path (if not NULL) keyed by GPU name, equation,
 * order, precision, grid and the safeguard; a cached entry is reused
 * without timing.  *choice (may be NULL)
 * receives tile2d + 3 * fused_oe (0..5).  1D handles have one shape and no
 * fused path (choice 0).  Synchronous. */
fam_status fam_tune(fam_t h, double cfl, int probe_steps, const char* cache_path, int* choice);

/* Wait for the handle's stream and report device-side status flags. */
fam_status fam_sync(fam_t h);

/* Current time, size of the next step and number of steps taken (any may be
 * NULL).  Synchronous. */
fam_status fam_time(fam_t h, double* t, double* dt_next, long* steps);

/* Per-kernel device time accumulated over the profiled fam_step() calls since
 * the option "profile" was last set: ms[0..2] = stage 1..3 kernels, ms[3] =
 * OE kernel (milliseconds, CUDA events on the handle's stream); with
 * "fused_oe", ms[2] holds the fused final stage + OE launch and ms[3] is 0;
 * *nsteps = number of profiled steps.  Synchronises the stream. */
fam_status fam_profile(fam_t h, double* ms, long* nsteps);

/* Steps discarded since the state was set (option "pp_limiter"): a step
 * whose stage output averages leave the admissible set (rho <= 0 or p <= 0)
 * is dropped -- the OE writes nothing, the clock and the step count stay --
 * and retried with the step size halved, again and again (at most 30
 * times, then FAM_E_NONPHYSICAL); an accepted step restores the CFL size.
 * The forward-Euler bound of the safeguard holds for the speeds of each
 * stage's input, which can exceed those of U^n the step size came from.
 * fam_run_steps counts attempts, fam_time and fam_run accepted steps. */
fam_status fam_rejected_steps(fam_t h, unsigned long long* count);

/* Number of face quadrature points (1D: faces) at which one of the two
 * traces entering the Rusanov flux had no spectral radius, summed over every
 * residual evaluation (the three stages of each step, fam_residual) since the
 * last fam_set_state.  A trace has none when it is not an admissible Euler
 * state in the sense gamma p / rho < 0 (rho <= 0 or p <= 0 at a face point,
 * which the paper's optional positivity limiter (Sec. 2.3 remarks, Alg. 1)
 * would prevent and this library does not build); the flux then takes the
 * other trace's radius (IEEE maxNum, Sec. 2.3 Rusanov flux).  Faces counted:
 * x-faces 0..nx of every row and y-faces 0..ny of every column, four Gauss
 * points each in 2D; a periodic grid counts its boundary face twice (both
 * images are evaluated).  Synchronous.  Errors: FAM_E_INVAL (null pointer). */
fam_status fam_nonphysical_traces(fam_t h, unsigned long long* count);

/* Semi-discrete right-hand side R(U) of eq. (1dSemi) / eq. (11) for the
 * state U (layout above), written to R (same layout).  Uses the handle's
 * scratch buffers; the handle's current state is not changed. */
fam_status fam_residual(fam_t h, const void* U, void* R, int on_device);

/* The OE operator alone with step size dt (eq. 9 / eq. 2dOE_sol with the
 * Type-II coefficient): Uout = F_OE(U).  Averages are copied unchanged.
 * The handle's current state is not changed. */
fam_status fam_oe(fam_t h, double dt, const void* U, void* Uout, int on_device);

/* Message of the last failing call on h (never NULL). */
const char* fam_last_error(fam_t h);

/* Name of a status code. */
const char* fam_status_string(fam_status s);

/* Release all resources of h (NULL is ignored). */
void fam_destroy(fam_t h);

/* Adjoint (not in the paper; the reverse sweep of the time step).  Runs
 * nsteps steps (eq. 12 + OE) from U0 with the CFL step sizes of Sec. 4, then
 * returns in dJdU0 the gradient of a terminal functional J(U^T) with respect
 * to all initial averages and moments, given dJdUT = dJ/dU^T (both in the
 * state layout above).  The step sizes of the forward run are held fixed in
 * the reverse sweep.  The forward states are checkpointed every ckpt_every
 * steps and each segment is recomputed once in the reverse sweep (memory:
 * nsteps/ckpt_every + 4*ckpt_every padded states).  Subgradients: |x| ->
 * sign(x), a maximum -> the first maximiser (left/bottom trace, lowest
 * component, row-major stencil order).  On return the handle's state is
 * U^T.  Built for 2D Euler, FP64, periodic grids (FAM_E_UNSUPPORTED
 * otherwise).  on_device as in fam_set_state.  Synchronous. */
fam_status fam_adjoint(fam_t h, long nsteps, double cfl, int ckpt_every, const void* U0, const void* dJdUT,
                       void* dJdU0, int on_device);

/* ------------------------------------------------------------------------
 * Batched problems (not in the paper: many independent instances in one
 * persistent launch).
 *
 * 1D: instance i has nx[i] cells on [x0, x1] and order k[i]; all share the
 * equation, bc (periodic or outflow), gamma (see fam_create) and precision.
 * 2D (fam_batch2d_create; 2D Euler): instance i has nx[i] x ny[i] cells on
 * [x0, x1] x [y0, y1] and order k[i].
 * State layout: the instances' states (1D U_i[c][m][i], 2D U_i[c][m][j][i])
 * concatenated in instance order.  Each instance takes its own CFL step
 * size (Sec. 4) from its own maximum Rusanov speed(s).  The per-tile
 * arithmetic is the single-problem code, so each instance evolves exactly
 * as fam_step would (in 2D: with the same tile shape, option "tile2d").
 * Type-I OE, inflow and reflective sides are not offered for batches.
 * ------------------------------------------------------------------------ */
typedef struct fam_batch* fam_batch_t;

/* Errors: FAM_E_INVAL (bad sizes/orders), FAM_E_NOMEM, FAM_E_CUDA. */
fam_status fam_batch_create(fam_batch_t* out, int n_inst, const int* nx, const int* k, double x0, double x1,
                            int equation, int bc, double gamma, int precision, void* stream);
/* 2D batch of the Euler equations (equation must be FAM_EULER, else
 * FAM_E_UNSUPPORTED).  nx, ny, k: arrays of n_inst (each nx, ny >= 4). */
fam_status fam_batch2d_create(fam_batch_t* out, int n_inst, const int* nx, const int* ny, const int* k, double x0,
                              double x1, double y0, double y1, int equation, int bc, double gamma, int precision,
                              void* stream);
/* Keys: "oe_type" (0 / 2), "gamma_k" (<= 0: defaults per order), "ax",
 * "tile_x" (1D: 64 / 128 / 256 cells per tile), "tile2d" (2D: 0 / 1 / 2 for
 * 32x8 / 32x4 / 16x8 cells per tile), "blocks_per_sm" (<= 0: the occupancy
 * maximum), "pp_limiter" (1D Euler: the BP/PP safeguard of fam_set_option,
 * in every instance, step rejection included: each instance discards and
 * retries its own steps, fam_batch_rejected_steps), "wait_limit_ns" (how long a block waits at the persistent
 * kernel's grid barrier before the launch gives up with FAM_E_TIMEOUT from
 * fam_batch_sync; 0 restores the default of 2 s; at most 60 s),
 * "test_barrier_extra" (test hook, 0 or 1: the grid barrier waits for one
 * arrival more than there are blocks, so every wait runs out after
 * "wait_limit_ns"; the kernel then exits and fam_batch_sync reports
 * FAM_E_TIMEOUT).  After a timeout the batch's state is undefined until the
 * next fam_batch_set_state, which also resets the barrier. */
fam_status fam_batch_set_option(fam_batch_t h, const char* key, double value);
/* Copy the concatenated state in / out (on_device as in fam_set_state);
 * set_state resets every instance's clock. */
fam_status fam_batch_set_state(fam_batch_t h, const void* U, int on_device);
fam_status fam_batch_get_state(fam_batch_t h, void* U, int on_device);
/* Advance every instance by nsteps steps (eq. 3/12 + OE) in ONE cooperative
 * persistent kernel launch (a tile work list walked pass by pass with
 * bounded grid barriers), captured in a CUDA graph per (nsteps, cfl).
 * With "pp_limiter", nsteps counts attempts: an instance whose attempt the
 * safeguard rejects keeps its state and clock and takes its next attempt
 * with half the step size, so it advances by fewer accepted steps
 * (fam_batch_times) than the others.
 * Asynchronous; fam_batch_sync() waits and reports device flags. */
fam_status fam_batch_run(fam_batch_t h, long nsteps, double cfl);
fam_status fam_batch_sync(fam_batch_t h);
/* Per-instance time, next step size and steps taken (arrays of n_inst; any
 * may be NULL).  Synchronous. */
fam_status fam_batch_times(fam_batch_t h, double* t, double* dt, long* steps);
/* Per-instance health (arrays of n_inst; any may be NULL): ntrace as
 * fam_nonphysical_traces for the instance; status FAM_OK or
 * FAM_E_NONPHYSICAL (a non-finite value, or averages with rho <= 0 or
 * p <= 0, after some step); bad_step the 1-based step whose output was first
 * flagged (0: none).  A flagged instance stops after that step (its state is
 * that step's output) while the other instances go on; fam_batch_sync then
 * reports FAM_E_NONPHYSICAL for the batch.  Synchronous. */
fam_status fam_batch_health(fam_batch_t h, unsigned long long* ntrace, int* status, long* bad_step);
/* Per-instance attempts discarded since the state was set (option
 * "pp_limiter"; array of n_inst): an attempt whose stage output averages
 * leave the admissible set (rho <= 0 or p <= 0) writes nothing -- the
 * instance's later stages and OE skip it, its clock and step count stay --
 * and the instance's next attempt takes half the step size, again and again
 * (at most 30 halvings; the 31st stops the instance with FAM_E_NONPHYSICAL,
 * bad_step = the step it could not take); an accepted step restores the CFL
 * size.  The same rule as fam_rejected_steps, per instance.  Synchronous. */
fam_status fam_batch_rejected_steps(fam_batch_t h, unsigned long long* count);
/* Launch shape: tile width (2D: the tile's x extent), blocks of the
 * persistent grid, tiles, cells. */
fam_status fam_batch_info(fam_batch_t h, int* tile_x, int* grid, long* ntiles, long* cells);
/* Tile extents in cells (1D: tile_y = 1).  Either pointer may be NULL. */
fam_status fam_batch_tile(fam_batch_t h, int* tile_x, int* tile_y);
/* Autotuner: times probe_steps steps for each tile shape (1D widths 64,
 * 128, 256; 2D 32x8, 32x4, 16x8) and blocks-per-SM choice on the handle's
 * current state (restored afterwards, clocks included), keeps the fastest, and appends it to
 * cache_path (if not NULL) keyed by GPU name, problem and the safeguard; a
 * cached entry is reused without timing.  *tile_x receives the tile's x
 * extent. */
fam_status fam_batch_tune(fam_batch_t h, double cfl, int probe_steps, const char* cache_path, int* tile_x,
                          int* blocks_per_sm);
const char* fam_batch_last_error(fam_batch_t h);
void fam_batch_destroy(fam_batch_t h);

/* ------------------------------------------------------------------------
 * Allocation-free step (the paper has no counterpart: this is a calling
 * convention for callers that cannot allocate device memory -- host
 * applications that own a fixed device-memory budget and do not let plug-ins
 * call cudaMalloc, and latency-critical loops where an allocation's cost and
 * failure mode are not acceptable).
 *
 * One time step (three SSP-RK3 stages and the OE, as fam_step) of a 1D
 * problem of nx <= FAM_NOALLOC_MAX_CELLS cells, from U_in to U_out, both
 * caller-owned device buffers in the state layout of this header (element
 * type per precision).  equation, bc, gamma, k, precision as in fam_create;
 * the step size follows the CFL rule from U_in.  No device memory is
 * allocated or freed: the intermediate states and the control block live in
 * one static device array of the library (sized for FAM_NOALLOC_MAX_CELLS
 * cells of 6 planes in FP64, about 2.4 MB), present on every GPU that loads
 * the library until the process exits.  The first call on a device looks up
 * that array's device address (once per device, with the device current), so
 * make the first call on each device before any stream capture.  Every call
 * reuses the same array: calls whose GPU work may overlap (other streams or
 * host threads) race and must be serialised by the caller.  stream: a
 * cudaStream_t or NULL for the legacy default stream.  Synchronous: the
 * call waits for its stream, then reports FAM_E_NONPHYSICAL (a non-finite
 * value or a non-physical average) or FAM_E_TIMEOUT (a bounded wait gave up)
 * from the device flags, and writes the step size taken to *dt_used if
 * dt_used is not NULL.  Errors: FAM_E_INVAL (including nx above the limit),
 * FAM_E_CUDA.
 * ------------------------------------------------------------------------ */
#define FAM_NOALLOC_MAX_CELLS 16384
fam_status fam_step1d_noalloc(const void* U_in, void* U_out, int nx, double x0, double x1, int k, int equation,
                              int bc, double gamma, int precision, double cfl, double* dt_used, void* stream);

/* Measured throughput of this GPU's FP64 (precision 64) or FP32 (32) fused
 * multiply-add pipe in FLOP/s, from a register-resident FMA loop timed with
 * CUDA events (a roofline denominator; not part of the method). */
fam_status fam_alu_peak(int precision, double* flops_per_s);

/* Diagnostics: the library's FP64 reciprocal, reciprocal square root and
 * square root (FP32 hardware approximation refined by one third-order
 * step) applied to n host values x (positive, within the FP32 normal
 * range); results are written to the three host arrays.  Test hook for
 * comparing against correctly rounded results. */
fam_status fam_selftest_math(const double* x, int n, double* rcp, double* rsqrt, double* sqrt_out);

/* Diagnostics: the library's binary64 multiply computed with integer
 * instructions (the FP64 kernels run part of their products on the integer
 * pipes, beside the FP64 unit), applied elementwise to the n host pairs
 * (a[i], b[i]); prod[i] = a[i] * b[i] is written to a host array.  The IEEE
 * 754 round-to-nearest-even product is expected bit for bit, for every
 * input including zeros, subnormals, infinities and NaNs.  FAM_E_INVAL for
 * null pointers or n <= 0, FAM_E_NOMEM / FAM_E_CUDA on device errors. */
fam_status fam_selftest_int_fp64(const double* a, const double* b, int n, double* prod);

#ifdef __cplusplus
}
#endif
#endif /* FAM_H */
