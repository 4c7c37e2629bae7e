/*
 * alweno.h -- C ABI of the GB300 arc-length WENO (WENO-L) solver for
 * Hamilton-Jacobi equations  phi_t + H(D phi) = 0  (paper: "Arc length based
 * WENO scheme for Hamilton-Jacobi Equations", Sec. 2, Steps 1-5).
 *
 * One call advances phi with the fifth-order WENO reconstruction of the
 * one-sided derivatives phi_x^-/+ (Steps 1-2), nonlinear weights from the
 * arc-length smoothness indicators (Step 4, Eq. newbeta/length) or the
 * Jiang-Peng indicators (the comparison scheme of Sec. 3), the
 * Lax-Friedrichs numerical Hamiltonian (Sec. 2, LF flux) and the TVD-RK3
 * time integrator (Step 5), in 1D or 2D (dimension by dimension, Sec. 2 Note).
 * Every RK stage is one CUDA kernel on the device.
 *
 * Conventions (all entry points):
 *  - Return an alw_status; nothing aborts or throws across the ABI.  On error,
 *    alw_last_error() returns a thread-local message.
 *  - Host pointers passed in are owned by the caller and only read (or
 *    written, for outputs) during the call.
 *  - Device memory is owned by the library.  It is obtained through the
 *    allocator installed with alw_set_allocator (default: the CUDA
 *    stream-ordered allocator on the solver's stream).
 *  - Arrays are row-major with x fastest: index j*nx + i for node (x_i, y_j);
 *    1D arrays have ny = 1.
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    needs one returns ALW_ECUDA.
 */
#ifndef ALWENO_H
#define ALWENO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ALW_OK = 0,
  ALW_EINVAL = 1,      /* bad argument (size mismatch, unknown enum, NULL) */
  ALW_ENOMEM = 2,      /* device or host allocation failed */
  ALW_ECUDA = 3,       /* CUDA runtime/driver error */
  ALW_ENONFINITE = 4,  /* a NaN/Inf appeared in dH/dp during a stage */
  ALW_ETIMEOUT = 5,    /* a bounded device wait gave up */
  ALW_EBUSY = 6,       /* object in use (e.g. server still running) */
  ALW_EBUDGET = 7,     /* request exceeds the device-memory budget */
  ALW_ENOTFOUND = 8    /* unknown instance / request id */
} alw_status;

/* Boundary conditions.  PERIODIC: n nodes on [lo, hi), dx = (hi-lo)/n.
 * LINEXTRAP: n nodes on [lo, hi] including both ends, dx = (hi-lo)/(n-1),
 * ghost values phi_{-m} = (1+m) phi_0 - m phi_1 (mirror image at the right). */
enum { ALW_BC_PERIODIC = 0, ALW_BC_LINEXTRAP = 1 };

/* Hamiltonians H(p, q), p = phi_x, q = phi_y (Sec. 3 examples). */
enum {
  ALW_H_BURGERS2D = 0, /* (p+q+1)^2/2     Example 3 */
  ALW_H_NEGCOS2D = 1,  /* -cos(p+q+1)     Example 4 */
  ALW_H_SIN2D = 2,     /* sin(p+q)        Example 10 */
  ALW_H_ADVECT1D = 3,  /* p               Example 1 */
  ALW_H_BURGERS1D = 4, /* (p+1)^2/2       Example 6 */
  ALW_H_NEGCOS1D = 5,  /* -cos(p+1)       Example 2 */
  ALW_H_EIKONAL2D = 6, /* sqrt(p^2+q^2+1) Example 12 */
  ALW_H_NONCONVEX1D = 7, /* (p^2-1)(p^2-4)/4 Example 8; non-convex: the node alpha is the
                            maximum of |H_p| over the interval between the one-sided derivatives */
  ALW_H_OPTCTRL2D = 8    /* sin(y)p + (sin(x)+sign q)q - sin^2(y)/2 - (1-cos x)   Example 11;
                            depends on the node position x_i = xlo + i dx, y_j = ylo + j dy;
                            alpha_x = |sin y|, alpha_y = max |sin x + s| over the signs s of the
                            interval between v^- and v^+ (both when it contains 0).  Single
                            solvers only (batches and the server reject it). */
};

/* Smoothness indicators of the nonlinear weights (Step 4). */
enum { ALW_W_ARCLEN = 0, ALW_W_JP = 1 };

/* alpha of the Lax-Friedrichs flux (LF flux, alpha = max |H_1|) and of the
 * CFL time step.  A "grid maximum" is the maximum over all nodes and over the
 * four (u^-/u^+, v^-/v^+) combinations of |dH/dp| (x) and |dH/dq| (y).
 *  LOCAL_*  : flux uses the node's own maximum over the four combinations.
 *  GLOBAL_* : flux uses a grid maximum.
 *  *_LAGGED : the grid maximum of the previous stage (one kernel per stage;
 *             a prime pass over phi^0 supplies the first).
 *  *_EXACT  : the grid maximum of the current stage (GLOBAL) / of phi^n for
 *             dt (both): an extra reduction pass, for validation.
 *  FIXED    : alpha_fixed for flux and dt.
 *  DEFAULT  : LOCAL_LAGGED in 1D, GLOBAL_LAGGED in 2D. */
enum {
  ALW_ALPHA_DEFAULT = -1,
  ALW_ALPHA_LOCAL_LAGGED = 0,
  ALW_ALPHA_LOCAL_EXACT = 1,
  ALW_ALPHA_GLOBAL_LAGGED = 2,
  ALW_ALPHA_GLOBAL_EXACT = 3,
  ALW_ALPHA_FIXED = 4
};

/* Time step (Sec. 3: CFL 0.6): dt = cfl / (alpha_x/lx + alpha_y/ly) with
 * lx = dx (CFL) or dx^{5/3} (DX53, for convergence studies); the last step is
 * clipped so that t reaches t_final exactly. */
enum { ALW_DT_CFL = 0, ALW_DT_DX53 = 1 };

/* Arithmetic.  FP64: all in double.  FP32: phi and all arithmetic in float.
 * MIXED: stencil arithmetic in float; phi^n is held as an unevaluated sum of
 * two floats (hi + lo, about 48 significant bits) and the RK stages store
 * float increments that carry the low part, lo + (phi_s - phi^n), so a stage
 * state is hi plus one float array and the accumulation of phi over long runs
 * keeps double-class precision; the CFL reduction is in double.  In FP32 and
 * MIXED the square roots, logarithms, reciprocals, sines and cosines of the
 * stencil and of the Hamiltonians are the GPU's hardware approximations
 * (relative error of a few units in the last float place; the logarithm's
 * absolute error is about 2^-22), so float results match the FP64 oracle to
 * float accuracy, not bit for bit. */
enum { ALW_PREC_FP64 = 0, ALW_PREC_FP32 = 1, ALW_PREC_MIXED = 2 };

typedef struct {
  int32_t dim;          /* 1 or 2 */
  int32_t nx, ny;       /* nodes per direction; ny = 1 when dim = 1 */
  int32_t bc;           /* ALW_BC_* (same on every side) */
  double xlo, xhi;      /* x extent */
  double ylo, yhi;      /* y extent (ignored when dim = 1) */
} alw_grid;

typedef struct {
  int32_t kind;         /* ALW_H_* */
  double param[4];      /* reserved, must be zero */
} alw_hamiltonian;

typedef struct {
  int32_t weights;      /* ALW_W_* */
  double eps;           /* epsilon of Eq. WLOC1 (paper: 1e-6) */
  double cfl;           /* CFL number (paper: 0.6) */
  int32_t dt_mode;      /* ALW_DT_* */
  int32_t alpha_mode;   /* ALW_ALPHA_* */
  double alpha_fixed[2];/* used by ALW_ALPHA_FIXED */
  int32_t precision;    /* ALW_PREC_* */
} alw_scheme;

/* Checkpoint: phi^n is transferred separately (alw_get_phi / alw_set_state). */
typedef struct {
  double t;             /* current time */
  int64_t steps;        /* RK3 steps taken */
  double alpha[2];      /* most recent grid-maximum reduction (lagged alpha) */
} alw_state;

typedef struct alw_solver alw_solver;

/* Device allocator hook (process-wide; no counterpart in the paper).  alloc
 * returns device memory of at least `bytes` usable in stream order on
 * `stream`, or NULL; free releases it.  Pass NULL to restore the default
 * (cudaMallocAsync/cudaFreeAsync: the C library depends on no framework; the
 * Python binding installs the PyTorch caching allocator through this hook). */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *ctx);
  void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
  void *ctx;
} alw_allocator;
alw_status alw_set_allocator(const alw_allocator *allocator);

/* Library version string and the thread-local message of the last error (no
 * counterpart in the paper). */
const char *alw_version(void);
const char *alw_last_error(void);

/* Create a solver on the current CUDA device; `cuda_stream` is a cudaStream_t
 * (NULL = the default stream) on which every later call enqueues its work.
 * Problem statement: Eq. HJ / HJ1.  Errors: ALW_EINVAL (bad grid/scheme, nx <
 * 1, LINEXTRAP with fewer than 2 nodes, 1D grid with a 2D Hamiltonian or the
 * reverse), ALW_ENOMEM, ALW_ECUDA. */
alw_status alw_create(const alw_grid *grid, const alw_hamiltonian *ham, const alw_scheme *scheme,
                      void *cuda_stream, alw_solver **out);
/* Release the solver and its device memory (no counterpart in the paper); NULL is ALW_EINVAL. */
alw_status alw_destroy(alw_solver *s);

/* Set the initial data phi(x, 0) = phi^0(x) of Eq. HJ from a host array of
 * n = nx*ny doubles (copied); resets t to 0, the step count and the lagged
 * alpha (a prime pass over phi^0 supplies the first, Step 5 with the LF flux).
 * ALW_EINVAL if n != nx*ny. */
alw_status alw_set_phi0(alw_solver *s, const double *host_phi, size_t n);

/* Same (initial data of Eq. HJ) from a device array (e.g. a torch tensor's data
 * pointer) of n values of `dtype` (0 = double, 1 = float), contiguous
 * row-major; copied on the stream.  ALW_EINVAL for another dtype or n. */
alw_status alw_set_phi0_device(alw_solver *s, const void *dev_phi, int32_t dtype, size_t n);

/* Advance to t_final with TVD-RK3 (Step 5): whole steps, the last one clipped.
 * Work is enqueued as CUDA-graph replays on the solver's stream; the call
 * returns after the device reports t >= t_final.  steps_out (nullable) gets
 * the number of steps taken by this call.  ALW_ENONFINITE if dH/dp became
 * non-finite (phi is left at the step where it was detected). */
alw_status alw_step_to(alw_solver *s, double t_final, int64_t *steps_out);

/* Advance exactly nsteps TVD-RK3 steps (Step 5) with the CFL time step of
 * Sec. 3 (no clipping; used for throughput measurement).  Asynchronous:
 * returns after enqueueing. */
alw_status alw_advance(alw_solver *s, int64_t nsteps);

/* Enqueue a single RK stage (1, 2 or 3) with the given dt (asynchronous; for
 * stage-level tests and per-stage timing).  Stage 1 reads phi^n and writes
 * stage 1's state, and so on; the state after stage 3 is phi^{n+1} (t and the
 * step count are not changed).  ALW_EINVAL for a stage outside 1..3 or a
 * non-finite dt. */
alw_status alw_run_stage(alw_solver *s, int32_t stage, double dt);

/* Wait for the solver's stream (no counterpart in the paper); returns
 * ALW_ENONFINITE if a stage flagged a non-finite dH/dp. */
alw_status alw_sync(alw_solver *s);

/* Copy the solution phi(x, t) of Eq. HJ at the solver's current time
 * (interior, n = nx*ny doubles) to a caller-owned host buffer; for MIXED the
 * two float parts are summed exactly in double.  alw_get_phi_device writes n
 * values of `dtype` (0 = double, 1 = float) to a caller-owned device array.
 * ALW_EINVAL if n != nx*ny. */
alw_status alw_get_phi(alw_solver *s, double *host_out, size_t n);
alw_status alw_get_phi_device(alw_solver *s, void *dev_out, int32_t dtype, size_t n);

/* Read the state of RK stage `stage` (1 or 2) after alw_run_stage (phi_1 or
 * phi_2 in the notation of Step 5), as doubles. */
alw_status alw_get_stage_phi(alw_solver *s, int32_t stage, double *host_out, size_t n);

/* Time, steps, lagged alpha; and restoring them with phi (checkpoint/resume,
 * no counterpart in the paper: resuming reproduces an uninterrupted run bit
 * for bit, to a tie in the hi/lo split of MIXED). */
alw_status alw_get_state(alw_solver *s, alw_state *state);
alw_status alw_set_state(alw_solver *s, const alw_state *state, const double *host_phi, size_t n);

/* Device bytes held by the solver (no counterpart in the paper). */
alw_status alw_memory_bytes(alw_solver *s, size_t *bytes);

/* ------------------------------------------------------------------------
 * Batches: many independent 2D periodic instances of uneven size (grids,
 * Hamiltonians, phase-shifted initial data and end times may all differ)
 * advanced together by one persistent launch per RK stage over a shared
 * work list of (instance, tile) pairs, replayed from a CUDA graph until every
 * instance has reached its own t_final.  Each instance follows exactly the
 * same arithmetic as a single solver with the same scheme (same dt rule,
 * alpha, weights), so its result does not depend on the other instances.
 * Precision must be FP32 or MIXED; alpha_mode DEFAULT, GLOBAL_LAGGED,
 * LOCAL_LAGGED or FIXED.  Not a construct of the paper: it serves many solves
 * per device. */
typedef struct alw_batch alw_batch;

/* Work-list orders the autotuner chooses from. */
enum { ALW_ORDER_INSTANCE = 0, ALW_ORDER_LARGEST_FIRST = 1, ALW_ORDER_INTERLEAVED = 2 };
typedef struct {
  int32_t order;            /* ALW_ORDER_* */
  int32_t steps_per_graph;  /* RK3 steps captured per graph replay (1..256) */
  int32_t grid_ctas;        /* persistent CTAs; 0 = as many as fit on the device (larger values are capped) */
  int32_t run;              /* entries of the ordered work list a persistent CTA takes in a row before
                               the next CTA's turn (0..64): 1 = consecutive entries side by side on
                               neighbouring CTAs; k > 1 = blocks of k, so a CTA changes instance (and
                               folds that instance's alpha) less often while neighbouring blocks
                               still run together; 0 = one contiguous stretch per CTA.  The
                               autotuner uses 4. */
  int32_t tile_w;           /* tile width in nodes: 64 (tiles 64 x 32) or 32 (tiles 32 x 32: twice the
                               tiles, each with 1.1x the halo reads per node); 0 = 64.  The
                               autotuner times both on the batch's own work list. */
  int32_t one_launch;       /* 1: one launch per RK stage over every instance, the kernel choosing
                               each tile's Hamiltonian at run time; 0: one launch per Hamiltonian
                               present, each with a kernel specialised for it.  The autotuner
                               times both when the batch mixes Hamiltonians. */
} alw_batch_tuning;

alw_status alw_batch_create(const alw_scheme *scheme, void *cuda_stream, alw_batch **out);
/* Add an instance (grid dim 2, periodic; host_phi0 of n = nx*ny doubles, copied to
 * device memory before the call returns, so the caller may reuse it).  id_out
 * receives its index.  ALW_EBUSY after the batch has been built or run. */
alw_status alw_batch_add(alw_batch *b, const alw_grid *grid, const alw_hamiltonian *ham, const double *host_phi0,
                         size_t n, double t_final, int32_t *id_out);
/* Fix the tuning (NULL: let the autotuner choose on the next run).  ALW_EINVAL
 * for a field outside its range (tile_w other than 0, 32, 64; one_launch other than 0, 1). */
alw_status alw_batch_set_tuning(alw_batch *b, const alw_batch_tuning *tuning);
alw_status alw_batch_get_tuning(alw_batch *b, alw_batch_tuning *tuning);
/* Lay out the device arena, upload every instance and tune the work list now
 * (alw_batch_run does this on its first call); instances cannot be added
 * afterwards.  Separates set-up from the time loop. */
alw_status alw_batch_build(alw_batch *b);
/* Advance every instance to its t_final; returns after all have arrived.
 * replays_out (nullable): graph replays used.  ALW_ENONFINITE if an instance
 * saw a non-finite dH/dp (the others still finish). */
alw_status alw_batch_run(alw_batch *b, int64_t *replays_out);
/* Instance id's phi at its current time (n = its nx*ny doubles, caller-owned host
 * buffer) and its state; ALW_ENOTFOUND for an unknown id, ALW_EINVAL before
 * the first run or for a wrong n.  Device bytes held; release everything. */
alw_status alw_batch_get_phi(alw_batch *b, int32_t id, double *host_out, size_t n);
alw_status alw_batch_get_state(alw_batch *b, int32_t id, alw_state *state);
alw_status alw_batch_memory_bytes(alw_batch *b, size_t *bytes);
alw_status alw_batch_destroy(alw_batch *b);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  Submitted solves (2D,
 * periodic, FP32 or MIXED, grid sides up to max_side) wait in a FIFO queue; a
 * host worker thread admits them at round boundaries while a slot and enough
 * of the device-memory budget are free (state stays resident on the device),
 * advances every resident instance by a few RK3 steps per round in shared
 * persistent launches (their stages interleave), and retires each instance
 * when it reaches its t_final.  Each result equals the single solve of the
 * same request.  Not a construct of the paper. */
typedef struct alw_server alw_server;

typedef struct {
  int32_t status;     /* ALW_OK or the request's error */
  int64_t steps;      /* RK3 steps taken */
  double queue_s;     /* submit -> admission */
  double latency_s;   /* submit -> result available */
} alw_request_info;

typedef struct {
  int64_t submitted, admitted, completed, queued, rounds;
  int64_t arena_rows, free_rows;  /* device arena rows in total / free now */
} alw_server_stats;

/* hbm_budget_bytes bounds all device memory the server holds (arena of
 * resident instances + tables + staging); ALW_EBUDGET if it cannot hold one
 * instance of max_side x max_side.  max_slots bounds resident instances. */
alw_status alw_server_create(const alw_scheme *scheme, size_t hbm_budget_bytes, int32_t max_slots, int32_t max_side,
                             void *cuda_stream, alw_server **out);
/* Minimum RK3 steps per round (admission granularity).  Rounds with no new
 * instance stretch to the fewest remaining steps among the active instances,
 * at most 16, so that a lone large solve is not slowed by round trips. */
alw_status alw_server_set_round_steps(alw_server *s, int32_t steps);
/* Round membership: the oldest resident instance always runs; the others join in
 * admission order while the round holds at most `tiles` tiles (64 x 32 nodes each)
 * in total, and instances of at most 32 tiles always join.  Large solves thus run
 * in arrival order with the small ones beside them.  0 = no limit (every resident
 * instance in every round).  Default: four waves of the persistent stage kernel.  Under load
 * the limit grows to half of the resident instances' tiles, so that many waiting instances
 * share fuller launches and fewer rounds. */
alw_status alw_server_set_round_tiles(alw_server *s, int32_t tiles);
/* Queue a solve (host_phi0 copied); req_id receives its id. */
alw_status alw_server_submit(alw_server *s, const alw_grid *grid, const alw_hamiltonian *ham, const double *host_phi0,
                             size_t n, double t_final, uint64_t *req_id);
/* Wait up to timeout_s (0: do not wait) for a request.  done = 1 when finished;
 * then info (nullable) is filled and, if host_out is given (n values), the
 * result is copied and the request is forgotten. */
alw_status alw_server_poll(alw_server *s, uint64_t req_id, double timeout_s, int32_t *done, double *host_out,
                           size_t n, alw_request_info *info);
/* Counters of the server (submitted, admitted, completed, queued, rounds, arena rows). */
alw_status alw_server_stats_get(alw_server *s, alw_server_stats *stats);
/* Stops the worker after its current round and frees everything. */
alw_status alw_server_destroy(alw_server *s);

/* ------------------------------------------------------------------------
 * No-allocation entry point (the paper has no counterpart; it serves callers
 * that cannot obtain device memory on demand, e.g. a framework whose pool
 * allocator owns all device memory, or a real-time loop that must not
 * allocate after start-up).
 *
 * Advances the caller's device array dev_phi_in (n = nx*ny doubles, row-major,
 * x fastest) by nsteps TVD-RK3 steps of fixed size dt with the FP64 stage
 * kernel and writes the result to dev_phi_out (may equal dev_phi_in).  The
 * scheme must have precision ALW_PREC_FP64.  The working storage is a fixed
 * 16 MiB device array inside this library (held by every GPU that loads it,
 * until the process exits); grids whose three padded FP64 copies do not fit
 * (about 800 x 800 in 2D) are rejected with ALW_EBUDGET.  No device memory is
 * allocated or freed.
 *
 * The first call on a device looks up the array's address and should be made
 * before any stream capture.  CUDA loads device code lazily by default, so
 * that first call also loads this library's device code on the device and
 * reserves the 16 MiB there (or fails with ALW_ECUDA if the device has no
 * room left): make it before a pool takes the device's memory or a real-time
 * phase begins, and check its status.  Every call clears the storage it uses; calls
 * whose GPU work overlaps (e.g. on two streams at once) race on the shared
 * storage and must be serialised by the caller.  Work is enqueued on
 * cuda_stream and the call returns after it completes; ALW_ENONFINITE if
 * dH/dp became non-finite. */
alw_status alw_step_noalloc(const alw_grid *grid, const alw_hamiltonian *ham, const alw_scheme *scheme,
                            const double *dev_phi_in, double *dev_phi_out, double dt, int32_t nsteps,
                            void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ALWENO_H */
