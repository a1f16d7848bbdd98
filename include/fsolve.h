/*
 * fsolve.h -- C ABI of the GB300 (sm_103a) 2D Fourier-space PDE solver.
 *
 * Method: arXiv:2412.12308.  A solve is a forward 2D DFT of a real field on a
 * periodic Nx x Ny grid (Sec. II.D, row transforms along x then column
 * transforms along y), a pointwise spectral operator (Sec. III), and the
 * inverse 2D DFT (the inverse formula after Eq. DFT2, 1/(Nx Ny) applied once).
 *
 * Conventions shared by every entry point
 *   Fields      real, row-major [ny][nx] (x fastest), element type given by
 *               the plan's dtype (float or double), owned by the caller, in
 *               device memory or in host memory mapped into the device's
 *               address space (pinned under unified addressing; the kernels
 *               then read/write it over the host link).  Complex fields
 *               (the *_c entry points) are interleaved (re, im).
 *               Sample x_j = j Lx/nx, y_k = k Ly/ny (Sec. II.D).
 *   Wavenumbers omega_x(a) = 2 pi a'/Lx, a' = a for a <= nx/2 else a - nx (the
 *               index shift of Sec. II.B); the Nyquist index is kept with
 *               |omega| = pi nx / Lx.  |omega|^2 = omega_x^2 + omega_y^2.
 *   Sizes       nx, ny even, 8 <= n <= 8192, n = 2^a * {1, 3, 5}; nx != ny and
 *               Lx != Ly allowed.  Anything else: FS_ERR_SIZE.
 *   Streams     fs_stream is a cudaStream_t (NULL = legacy default stream).
 *               The solve, advance and batch calls only enqueue work on that
 *               stream and return.  These wait: fs_batch_wait and
 *               fs_serve_poll (bounded by their timeouts), fs_state_save/load
 *               and fs_rk4_mean (the stream), fs_rk4_step (earlier work on the
 *               stream, before uploading its step table), and the *_destroy
 *               calls (the device).
 *   Workspace   a plan owns its device workspace (twiddle and wavenumber
 *               tables, one half-spectrum); calls on one plan (or on states of
 *               one plan) must be ordered on one stream.  Different plans are
 *               independent.
 *   Errors      every entry point returns fs_status; nothing is thrown across
 *               the ABI.  fs_last_error() returns a thread-local message for
 *               the last failing call on the calling thread.  A CUDA error
 *               raised while enqueuing returns FS_ERR_CUDA; asynchronous kernel
 *               faults surface at the caller's next synchronisation.
 *   Precision   FS_F32: float fields, FP32 butterflies with twiddles computed
 *               in FP64 and rounded once; Poisson factors evaluated in FP64
 *               and rounded once (a per-plan table built on the first
 *               Poisson solve, half a spectrum of floats); the other spectral
 *               factors combined in double-float (two-float) arithmetic and
 *               rounded once.
 *               Target: rel-L2 <= 1e-5 against an FP64 reference.
 *               FS_F64: everything in FP64, target rel-L2 <= 1e-12.
 */
#ifndef FSOLVE_H
#define FSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fs_plan_s *fs_plan;
typedef struct fs_state_s *fs_state;
typedef void *fs_stream;

typedef enum { FS_F32 = 0, FS_F64 = 1 } fs_dtype;

typedef enum {
  FS_OK = 0,
  FS_ERR_ARG = -1,     /* null handle/pointer, bad enum, negative time */
  FS_ERR_SIZE = -2,    /* unsupported grid size */
  FS_ERR_NOMEM = -3,   /* device or host allocation failed */
  FS_ERR_BUDGET = -4,  /* request does not fit the serving HBM budget */
  FS_ERR_CUDA = -5,    /* a CUDA runtime call failed */
  FS_ERR_TIMEOUT = -6, /* a bounded device wait or fs_serve_poll timed out */
  FS_ERR_BUSY = -7,    /* resource in use (e.g. serving queue full) */
  FS_ERR_NODEV = -8    /* no CUDA device visible */
} fs_status;

/* ---------------------------------------------------------------- plans
 * fs_plan_create: validate (nx, ny), build the radix factorisation of nx/2
 * and ny, the FP64-generated twiddle tables omega_N^m (Eq. DFT) rounded once to
 * the plan dtype, the per-axis |omega|^2 tables (Sec. II.D frequency grid with
 * the Sec. II.B shift), and allocate the plan's workspace on the current
 * device.  dtype is an fs_dtype.  *out receives the handle (library-owned;
 * release with fs_plan_destroy).  Errors: FS_ERR_ARG (out NULL, Lx/Ly <= 0,
 * bad dtype), FS_ERR_SIZE, FS_ERR_NOMEM, FS_ERR_NODEV, FS_ERR_CUDA.
 */
fs_status fs_plan_create(int nx, int ny, double lx, double ly, int dtype, fs_plan *out);
/* Frees the plan's device memory after synchronising the device. NULL is ok. */
fs_status fs_plan_destroy(fs_plan plan);
/* Query: grid and path of a plan. path: 0 = single-kernel shared-memory solve,
 * 1 = three-pass (row / fused column / row). Any out pointer may be NULL. */
fs_status fs_plan_info(fs_plan plan, int *nx, int *ny, int *dtype, int *path,
                       size_t *workspace_bytes);

/* ---------------------------------------------------------------- autotuning
 * fs_tune: time candidate configurations of a grid's standalone passes on the
 * current GPU (CUDA events, `reps` Poisson solves each after 2 warm-ups; reps
 * < 1 means 10) and keep the fastest: the register tile (hence the radix
 * split) of the row and of the column transforms, the row-tile height and the
 * column-group width.  Rows are tuned first, then columns with the best rows;
 * the result replaces the default only if it is faster.  The result is stored
 * in a process-wide cache keyed by (GPU name, nx, ny, dtype) that
 * fs_plan_create applies to later plans of that grid (a batch adapts the tile
 * heights to its CTA size), and written to the JSON-lines file named by the
 * environment variable FS_TUNE_CACHE when it is set (that file is also loaded
 * on first use).  Grids that run as one single-kernel solve are not tuned
 * (the default is returned).  Allocates two fields and a stream for the
 * duration of the call and synchronises them.  No counterpart in the paper.
 * fs_tune_cache_load/save: read/write the cache as JSON lines; they return
 * the number of entries, -1 if the file cannot be opened.
 * fs_tune_cache_clear: drop every entry (returns how many).
 * fs_plan_tiles: the configuration a plan uses. */
typedef struct {
  int e_row, e_col, rows, cols; /* the chosen configuration */
  double us_default, us_tuned;  /* one Poisson solve, default and chosen */
  int candidates;               /* configurations timed */
} fs_tune_result;
fs_status fs_tune(int nx, int ny, double lx, double ly, int dtype, int reps, fs_tune_result *out);
/* fs_tune_batch: the same for a grid run inside a batch: times `nprob`
 * Poisson solves of the grid in one fs_batch_submit (after two warm-ups) for
 * every pair of row / column register tiles, and stores the fastest pair
 * under the batch mode of the cache (tile heights in a batch follow its CTA
 * size).  fs_batch_submit applies it to problems of that grid that run as
 * units (not the single-CTA or standalone ones).  rows/cols of the result
 * are 0. */
fs_status fs_tune_batch(int nx, int ny, double lx, double ly, int dtype, int nprob, int reps,
                        fs_tune_result *out);
int fs_tune_cache_load(const char *path);
int fs_tune_cache_save(const char *path);
int fs_tune_cache_clear(void);
fs_status fs_plan_tiles(fs_plan plan, int *e_row, int *e_col, int *rows, int *cols);

/* ---------------------------------------------------------------- one-shot solves
 * fs_poisson_solve: u = the zero-mean solution of lap u = f - mean(f)
 * (Eq. Poisson2, Eq. SolutionPoisson): forward 2D DFT, multiply by
 * -1/|omega|^2 with the zero mode set to 0, inverse 2D DFT.  f and u are device
 * [ny][nx] arrays of the plan dtype; u may alias f.
 */
fs_status fs_poisson_solve(fs_plan plan, const void *f, void *u, fs_stream stream);

/* fs_diffusion_solve: u(t) of u_t = D lap u from u(0) = u0 (Eq. DiffusionIVPFS
 * with s = 0, Eq. solCalorFourier; D rescales time): multiplier
 * exp(-D |omega|^2 t).  D >= 0, t >= 0.  u may alias u0. */
fs_status fs_diffusion_solve(fs_plan plan, const void *u0, double D, double t, void *u,
                             fs_stream stream);

/* fs_wave_solve: u(t) of u_tt = c^2 lap u from u(0) = u0, u_t(0) = v0
 * (Eq. WaveEquationFourierSpace with s = 0; Eq. OmegaZero, Eq. OmegaNonZero
 * with t -> c t).  v0 may be NULL (zero initial velocity).  c > 0; t may be
 * negative (the solution operator is a group).  u may alias u0. */
fs_status fs_wave_solve(fs_plan plan, const void *u0, const void *v0, double c, double t,
                        void *u, fs_stream stream);

/* ---------------------------------------------------------------- slab passes
 * The steps of one solve split by slabs, for a grid shared by several GPUs
 * (Sec. II.D: the 2D DFT is the x transforms of every row followed by the y
 * transforms of every column, so a slab of rows and a slab of x frequencies
 * are each transformed locally; the exchange between the two layouts is the
 * caller's all-to-all).  `plan` is the plan of the WHOLE grid (its nx, ny,
 * Lx, Ly, dtype and tables); the calls only enqueue work on `stream` and use
 * the plan's factor tables, like the solves.
 *   fs_rows_forward: x transforms of `nrows` real rows f [nrows][nx] ->
 *     half spectrum spec [nx/2+1][nrows] (x-frequency-major: element (a, y)
 *     at a*nrows + y), unnormalised (Sec. II.D first step, real input packed
 *     as in the one-shot solves).  1 <= nrows <= ny.
 *   fs_columns_apply: for the x frequencies a0 .. a0+ncols-1 (0 <= a0,
 *     a0 + ncols <= nx/2 + 1), spec_cols [ncols][ny] holding their whole
 *     columns: forward y transform, the operator of `op` times 1/(nx ny)
 *     (FS_OP_POISSON, FS_OP_DIFFUSION with D, t >= 0, or FS_OP_WAVE with
 *     c > 0 and zero initial velocity; Sec. III), inverse y transform, in
 *     place.
 *   fs_rows_inverse: inverse x transforms (C2R) of spec [nx/2+1][nrows] ->
 *     real rows u [nrows][nx].
 * Buffers are device memory of the plan dtype (complex interleaved for the
 * spectra), owned by the caller.  Errors: FS_ERR_ARG (NULL, bad range, bad
 * op or parameters), FS_ERR_CUDA, FS_ERR_NOMEM (first Poisson call on an FP32
 * plan builds its factor table). */
fs_status fs_rows_forward(fs_plan plan, int nrows, const void *f, void *spec, fs_stream stream);
fs_status fs_columns_apply(fs_plan plan, int a0, int ncols, int op, double D, double c, double t,
                           void *spec_cols, fs_stream stream);
fs_status fs_rows_inverse(fs_plan plan, int nrows, const void *spec, void *u, fs_stream stream);

/* ---------------------------------------------------------------- operator factors
 * fs_operator_factors: the real multiplier the FP32 column pass applies to
 * every half-spectrum element (a, b) of `plan`'s grid (Sec. III: Poisson
 * -1/|omega|^2, diffusion exp(-D |omega|^2 t), wave cos(c |omega| t) -- the
 * factor of U0 --, each times 1/(nx ny)), written to out [nx/2+1][ny]
 * (float, x-frequency-major, device memory owned by the caller).
 * fp64 = 0: evaluated exactly as the column pass does (two-float, hardware
 * sine/cosine of the reduced phase); fp64 = 1: evaluated in FP64 and rounded
 * once.  For measuring the FP32 path's factor precision and the cost of FP64
 * evaluation; the solves never call it.  FP32 plans only; op is
 * FS_OP_POISSON, FS_OP_DIFFUSION (D, t >= 0) or FS_OP_WAVE (c > 0).
 * Errors: FS_ERR_ARG, FS_ERR_CUDA. */
fs_status fs_operator_factors(fs_plan plan, int op, double D, double c, double t, int fp64, void *out,
                              fs_stream stream);

/* ---------------------------------------------------------------- complex fields
 * The same three solves for complex fields (Sec. II.B: the samples p_jk may
 * be complex; the full spectrum is used, a = 0..nx-1).  Fields are
 * interleaved complex (re, im) of the plan dtype, [ny][nx], device memory
 * owned by the caller; outputs may alias inputs.  Operators, parameters and
 * errors as for the real solves (Poisson removes the complex mean).  The
 * first complex call allocates a full-spectrum workspace (nx ny complex; a
 * second one for the wave with v0) kept until fs_plan_destroy.  FS_ERR_SIZE
 * for FP64 plans with nx = 5 * 2^k, k >= 8 (no length-nx radix plan). */
fs_status fs_poisson_solve_c(fs_plan plan, const void *f, void *u, fs_stream stream);
fs_status fs_diffusion_solve_c(fs_plan plan, const void *u0, double D, double t, void *u,
                               fs_stream stream);
fs_status fs_wave_solve_c(fs_plan plan, const void *u0, const void *v0, double c, double t,
                          void *u, fs_stream stream);

/* ---------------------------------------------------------------- kept states
 * fs_state_create: forward-transform the initial data once and keep the
 * half-spectra U0 (and V0 when v0 != NULL) on the device (Sec. III.B/III.C:
 * the IVP in Fourier space is fixed by f-hat and g-hat).  u0, v0: device
 * [ny][nx] of the plan dtype, read during the call's stream work only.  The
 * state is library-owned; release with fs_state_destroy.
 */
fs_status fs_state_create(fs_plan plan, const void *u0, const void *v0, fs_stream stream,
                          fs_state *out);
fs_status fs_state_destroy(fs_state state);
/* fs_state_reset: forward-transform new initial data into an existing state
 * (same plan; v0 must be NULL iff the state was created without v0).  No
 * allocation; stream-ordered like fs_state_create. */
fs_status fs_state_reset(fs_state state, const void *u0, const void *v0, fs_stream stream);
/* fs_state_set_source: attach a time-independent source s (device [ny][nx] of
 * the plan dtype, read during the call's stream work only) to a state; its
 * forward transform S is kept beside U0/V0.  Every later advance of the state
 * (per call, batched or served) then solves the forced problem of
 * Eq. DiffusionIVPFS / Eq. WaveEquationFourierSpace with s != 0 mode by mode:
 *   diffusion  U = U0 E + S (1 - E)/(D|w|^2), E = exp(-D|w|^2 t); U0 + S t at D|w|^2 = 0
 *   wave       U = U0 cos th + V0 sin th/(c|w|) + S (1 - cos th)/(c|w|)^2,
 *              V = -c|w| U0 sin th + V0 cos th + S sin th/(c|w|),  th = c|w|t;
 *              U0 + V0 t + S t^2/2 and V0 + S t at w = 0
 * (the particular term S/(c|w|)^2 that the printed Eq. OmegaNonZero leaves out
 * of the non-zero modes is included).  s == NULL detaches the source (its
 * spectrum buffer is kept for reuse).  Allocates the source spectrum on first
 * use (FS_ERR_NOMEM / FS_ERR_CUDA on failure, state unchanged); a failed
 * transform leaves the state without a source.  Stream-ordered like
 * fs_state_reset. */
fs_status fs_state_set_source(fs_state state, const void *s, fs_stream stream);

/* Checkpoints of a kept state (the state is just its spectra: Sec. III.B/III.C
 * fix the solution at any t from f-hat, g-hat and s-hat).
 * fs_state_bytes: size of a checkpoint (a header plus U0, V0 when present and
 *   the source spectrum when attached).
 * fs_state_save: write the checkpoint into host memory dst (cap >= that size);
 *   synchronises the stream.  FS_ERR_ARG if dst is NULL or too small.
 * fs_state_load: restore a checkpoint into a state of a plan with the same
 *   grid, domain and dtype and the same v0 presence (FS_ERR_ARG otherwise, the
 *   state unchanged); attaches the saved source (allocating its buffer if
 *   needed) or detaches it.  Synchronises the stream.  Advances of the loaded
 *   state equal those of the saved one (absolute-time closed forms). */
fs_status fs_state_bytes(fs_state state, size_t *bytes);
fs_status fs_state_save(fs_state state, void *dst, size_t cap, fs_stream stream);
fs_status fs_state_load(fs_state state, const void *src, size_t bytes, fs_stream stream);

/* fs_diffusion_advance: u(t) from a kept state, t absolute (>= 0) from the
 * state's initial data: inverse 2D DFT of U0 exp(-D|omega|^2 t)
 * (Eq. solCalorFourier), plus the source term when one is attached
 * (fs_state_set_source).  u_out: device [ny][nx]. */
fs_status fs_diffusion_advance(fs_state state, double D, double t, void *u_out, fs_stream stream);

/* fs_wave_advance: u(t) (and v = u_t(t) when v_out != NULL) from a kept state:
 * U = U0 cos(c|omega|t) + V0 sin(c|omega|t)/(c|omega|), U = U0 + V0 t at
 * omega = 0 (Eq. OmegaZero/OmegaNonZero); V = -c|omega| U0 sin + V0 cos (the
 * first-order system, Eq. SystemOfODEsForWaveEquation); plus the source terms
 * when a source is attached (fs_state_set_source). */
fs_status fs_wave_advance(fs_state state, double c, double t, void *u_out, void *v_out,
                          fs_stream stream);

/* ---------------------------------------------------------------- RK4, moving source
 * The wave equation u_tt = c^2 lap u + s(t, x, y) with the orbiting Gaussian
 * source of Sec. III.C (example with source):
 *   s = A exp(-|x - x0(t)|^2 / sigma^2) cos(gamma t),
 *   x0(t) = radius (cos(Omega t), sin(Omega t)),
 * |x - x0| the minimum-image distance on the periodic domain, grid points
 * x_j = x_min + j Lx/nx, y_i = y_min + i Ly/ny.  Every mode of the half
 * spectrum is advanced with the classical fourth-order Runge-Kutta method on
 * the first-order system of Eq. SystemOfODEsForWaveEquation,
 *   dU/dt = V,  dV/dt = -c^2 |omega|^2 U + S(t),
 * S(t) the forward 2D DFT of the source sampled on the grid, evaluated at
 * t_k, t_k + dt/2 and t_k + dt for the step from t_k.  The paper's example:
 * A = 1, sigma = 0.1, Omega = 5, gamma = 10 on [-2, 2]^2, dt = h/4.
 */
typedef struct fs_rk4_s *fs_rk4;
typedef struct {
  double A, sigma, radius, Omega, gamma; /* sigma > 0; all finite */
  double x_min, y_min;                   /* grid origin */
} fs_orbit_source;

/* fs_rk4_create: integrator at time t0 from u(t0) = u0 and u_t(t0) = v0
 * (device [ny][nx] of the plan dtype, read during the call's stream work;
 * NULL = zero field).  Allocates five half spectra (U, V, S(t) and two
 * row-transform buffers) and a step table; FS_ERR_ARG on a NULL plan/src/out,
 * c <= 0, non-finite or sigma <= 0 parameters; FS_ERR_CUDA on allocation or
 * launch failure (nothing is leaked).  The plan must outlive the integrator. */
fs_status fs_rk4_create(fs_plan plan, double c, const fs_orbit_source *src, const void *u0,
                        const void *v0, double t0, fs_stream stream, fs_rk4 *out);
/* fs_rk4_step: nsteps RK4 steps of size dt (> 0, finite; nsteps >= 0), stream
 * ordered.  The per-step source table is uploaded from pageable memory (the
 * call waits for earlier work on the stream), then a CUDA graph of the
 * 2 x nsteps launches is replayed (captured on first use for each
 * (nsteps, dt)).  Explicit RK4 is stable for dt c |omega|_max <= 2.8 (the
 * paper's dt = h/4 gives ~1.1); larger steps are not rejected. */
fs_status fs_rk4_step(fs_rk4 rk, double dt, int nsteps, fs_stream stream);
/* fs_rk4_output: u (and u_t when v_out != NULL) at the current time, device
 * [ny][nx]: the inverse 2D DFT of U (and V). */
fs_status fs_rk4_output(fs_rk4 rk, void *u_out, void *v_out, fs_stream stream);
/* fs_rk4_mean: the grid mean of u at the current time (U's zero mode divided
 * by nx ny); synchronises the stream. */
fs_status fs_rk4_mean(fs_rk4 rk, double *mean_u, fs_stream stream);
/* fs_rk4_time: the integrator's current time t0 + (steps taken) dt. */
fs_status fs_rk4_time(fs_rk4 rk, double *t);
/* fs_rk4_destroy: synchronises the device, frees everything (NULL is a no-op). */
fs_status fs_rk4_destroy(fs_rk4 rk);

/* ---------------------------------------------------------------- batches
 * A request of a batch.  op: one of FS_OP_*.  The solve ops read `in_u`
 * (and `in_v` for FS_OP_WAVE, may be NULL) and write `out_u`; the advance ops
 * read `state` and write `out_u` (and `out_v` for FS_OP_WAVE_ADVANCE, may be
 * NULL).  `plan` gives the grid; every plan in a batch must have the same
 * dtype.  Pointers are owned by the caller and must be accessible from the
 * device: device memory, or host memory mapped into the device's address
 * space (pinned memory under unified addressing); output fields in host
 * memory are stored by the kernels directly (on GB300 over NVLink-C2C,
 * overlapped with the batch's compute).
 */
enum {
  FS_OP_POISSON = 0,
  FS_OP_DIFFUSION = 1,
  FS_OP_WAVE = 2,
  FS_OP_DIFFUSION_ADVANCE = 3,
  FS_OP_WAVE_ADVANCE = 4
};

typedef struct fs_request {
  int op;
  fs_plan plan;
  fs_state state;
  const void *in_u;
  const void *in_v;
  void *out_u;
  void *out_v;
  double D, c, t;
  /* serving only (ignored by fs_batch_submit): */
  int keep;        /* diffusion / zero-velocity wave solve: keep the forward
                      spectrum for this many follow-up requests */
  uint64_t parent; /* advance op: ticket of the request whose kept spectrum
                      to advance (instead of `state`) */
} fs_request;

/* fs_batch_submit: run n independent requests (any mix of sizes, operators
 * and kept states; Sec. III solves applied to many problems at once) as ONE
 * persistent kernel launch, captured in a CUDA graph and replayed when the
 * same batch shape repeats.  The launch's CTAs pull work units (diffusion
 * factor ranges, row tiles, column groups, C2R tiles, whole small problems)
 * from a device work table through an atomic counter; a unit waits (bounded:
 * 2 s per wait by default, env FS_BATCH_WAIT_NS; expiry sets FS_ERR_TIMEOUT in
 * the batch status and the kernel exits) only for units of its own problem
 * listed before it.  When a batch has both problems small enough to be
 * solved whole by one CTA and problems run as units, the small ones run as a
 * second launch in the same graph, beside the first (its own counter and
 * status; the batch status is the first error of the two).  Problems of
 * 4096^2 points or more (env FS_BATCH_DIRECT_MIN)
 * fill the GPU on their own and run as the standalone pass kernels, in order,
 * before that launch.  Workspace comes from a library-owned arena per in-flight
 * batch.  Each problem's result depends only on its own request (same tile
 * shapes and unit code alone or in any mix), so it is bit-identical across
 * batches.  The call enqueues on `stream` and returns; *ticket_out names the
 * batch for fs_batch_wait.  Errors: FS_ERR_ARG, FS_ERR_SIZE (mixed dtypes),
 * FS_ERR_NOMEM, FS_ERR_CUDA.
 */
fs_status fs_batch_submit(const fs_request *reqs, int n, uint64_t *ticket_out, fs_stream stream);
/* Block until batch `ticket` finished (bounded by timeout_us; <0 = no bound);
 * returns the batch's device status (FS_OK or FS_ERR_TIMEOUT) or a wait error. */
fs_status fs_batch_wait(uint64_t ticket, int timeout_us);

/* ---------------------------------------------------------------- serving
 * Continuous batching of solve and advance requests (Sec. III solves served
 * as a stream; the kept spectra realise the paper's observation that the IVP
 * in Fourier space is fixed by f-hat, so later times need only the inverse
 * transform).  A server thread forms batches from the queue in arrival order
 * whenever one of `slots` in-flight batches (each on its own stream) is free;
 * a request is admitted when its workspace plus the spectrum it keeps fits the
 * HBM budget next to everything in flight and kept; follow-ups wait until
 * their parent's spectrum is on the device.  One server per process.
 * fs_serve_start: budget (bytes, reserved on the current device), slots >= 2,
 *   max requests per batch.
 * fs_serve_enqueue: copy a request into the queue; *ticket_out names it.
 *   FS_ERR_BUDGET if it can never fit, FS_ERR_BUSY if the queue is full.
 *   A follow-up names its parent's ticket in `parent`; a parent that kept its
 *   spectrum with keep = k accepts at most k follow-ups (the spectrum is
 *   released once k have completed): a further one, or one whose parent kept
 *   nothing, is rejected with FS_ERR_ARG.  A queued follow-up whose parent's
 *   spectrum is gone finishes with latency -1 and fs_serve_poll reports
 *   FS_ERR_ARG.
 * fs_serve_replay: open-loop driver -- enqueue reqs[i] at arrival_s[i]
 *   seconds after the call (blocking until the last is enqueued); a
 *   follow-up's `parent` is given as (index of its parent in reqs) + 1.
 * fs_serve_poll: harvest up to `cap` finished tickets, waiting at most
 *   timeout_us (< 0: unbounded) for one; *n_done receives the count.
 * fs_serve_latency: enqueue -> observed completion, microseconds.
 * fs_serve_stats: batches, completed, max in flight, batches launched while
 *   another was in flight, peak bytes used, bytes used, queued, kept,
 *   failed (requests finished without running).
 * fs_serve_stop: drain the queue, wait for in-flight work, release memory. */
fs_status fs_serve_start(size_t hbm_budget_bytes, int slots, int max_batch);
fs_status fs_serve_enqueue(const fs_request *req, uint64_t *ticket_out);
fs_status fs_serve_replay(const fs_request *reqs, const double *arrival_s, int n, uint64_t *tickets_out);
fs_status fs_serve_poll(uint64_t *done_tickets, int cap, int *n_done, int timeout_us);
fs_status fs_serve_latency(uint64_t ticket, double *latency_us);
fs_status fs_serve_stats(uint64_t *out, int cap);
fs_status fs_serve_stop(void);


/* ---------------------------------------------------------------- no allocation
 * fs_poisson_solve_static: the same FP32 Poisson solve as fs_poisson_solve,
 * for callers that may not allocate device memory while they run (code
 * hosted in an application that owns the device memory pool, loops where an
 * allocation's implicit device synchronisation is not acceptable, programs
 * that size all device memory at start-up).  It needs no plan and allocates
 * nothing: its scratch (work spectrum and tables) is one fixed device array
 * inside the library, which every GPU that loads the library holds until the
 * process exits (about 4.2 MB).  The paper has no counterpart; this is a
 * deployment variant.
 *   f, u  device float [ny][nx] (u may alias f); Lx, Ly > 0.
 *   Sizes as for plans, and nx, ny <= 1024; larger grids: FS_ERR_SIZE.
 *   The first call on each device looks up the array's device address (with
 *   that device current); make that first call before any stream capture.
 *   All calls share the array and it keeps the last call's contents, so calls
 *   whose GPU work can overlap (different streams or host threads on one
 *   device) race; serialise them.  Nothing in it needs to start zeroed.
 *   Errors: FS_ERR_ARG, FS_ERR_SIZE, FS_ERR_CUDA, FS_ERR_NODEV. */
fs_status fs_poisson_solve_static(int nx, int ny, double lx, double ly, const void *f, void *u,
                                  fs_stream stream);

/* ---------------------------------------------------------------- misc */
const char *fs_last_error(void);
/* Size rule used by every entry point: 1 if n is supported, else 0. */
int fs_size_supported(int n);
/* Radix factorisation used for a length-L transform with `e` elements per
 * thread: writes up to `cap` radices into out, returns the count (0: none). */
int fs_radix_plan(int L, int e, int *out, int cap);
/* Device error word of the bounded waits inside the kernels (a TMA copy
 * that did not complete within 1 s makes the kernel record an error and
 * return instead of waiting forever).  Synchronises the device, writes the
 * code (0 = none) to *code when non-NULL, clears it, and returns
 * FS_ERR_TIMEOUT if it was set. */
fs_status fs_device_status(int *code);
/* Number of this library's kernels launched since load (all threads). */
uint64_t fs_kernel_launches(void);
/* Kernel timing: when enabled, every launch is bracketed by CUDA events on its
 * own stream (adds ~2 event records per launch).  fs_profile_report
 * synchronises the recorded events and writes, per kernel class, the launch
 * count and total device time in milliseconds; classes: 0 row R2C, 1 column,
 * 2 row C2R, 3 factor, 4 small, 5 batch.  Returns the number of classes
 * written (<= cap).  fs_profile_enable(0) stops recording and clears. */
fs_status fs_profile_enable(int on);
int fs_profile_report(uint64_t *counts, double *total_ms, int cap);

#ifdef __cplusplus
}
#endif

#endif /* FSOLVE_H */
