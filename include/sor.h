/*
 * sor.h -- C ABI of the GB300 red-black SOR library (libsorgb.so).
 *
 * The library solves the 2D steady heat-conduction / Poisson problem
 *     -Laplace(u) = f  on the unit square, Dirichlet data on the edges,
 * discretised with the 5-point stencil on an N x N interior (array side N+2,
 * h = 1/(N+1)), by red-black successive over-relaxation:
 *   - cell update: Eq. 1 of the paper (SOR extrapolation of the Gauss-Seidel
 *     value) with the 5-point stencil, Section 2.1 and Section 3.1:
 *       u_ij <- (1-w) u_ij + (w/4) (u_{i-1,j} + u_{i+1,j} + u_{i,j-1} + u_{i,j+1} + h^2 f_ij)
 *   - colouring: red <=> (i+j) even, black <=> (i+j) odd (Section 3.1,
 *     Figure 1); each iteration updates all red cells, then all black cells
 *     from the new red values (Section 3.1, Algorithm 1);
 *   - convergence: the largest change between successive iterates is
 *     compared with the tolerance every K iterations (Section 2.1,
 *     Section 3.3, Algorithm 1); a residual-based test is also offered.
 * Indices: row i = 0..N+1 (row 0 is the north edge), column j = 0..N+1;
 * arrays are row-major, (N+2)*(N+2) doubles, the outer ring holding the
 * Dirichlet data.  The ring is read, never written.
 *
 * Every entry point returns a sor_status; nothing throws, aborts or exits
 * across the ABI.  Non-convergence within the iteration cap is not an
 * error: the call returns SOR_OK with result.converged == 0 (Algorithm 1
 * reports whether SOR converged).
 *
 * Pointers to caller data may be host or device pointers (detected with
 * cudaPointerGetAttributes).  The library never frees caller memory.
 */
#ifndef SOR_H_
#define SOR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sor_ctx sor_ctx; /* opaque, owned by the library */

typedef enum {
  SOR_OK = 0,
  SOR_NOT_READY = 1,            /* sor_poll: the solve is still queued or running */
  SOR_ERR_INVALID_ARG = -1,     /* a NULL pointer, N < 1, w outside (0,2), ... */
  SOR_ERR_BUDGET = -2,          /* the request alone needs more than the context's HBM budget */
  SOR_ERR_OOM = -3,             /* a device or host allocation failed */
  SOR_ERR_CUDA = -4,            /* a CUDA runtime call failed (sor_last_error has the text) */
  SOR_ERR_TIMEOUT = -5,         /* sor_wait gave up, or a device-side wait ran past its limit */
  SOR_ERR_INTERNAL = -6,        /* a device-side consistency check failed */
  SOR_ERR_UNKNOWN_TICKET = -7,  /* sor_poll / sor_wait of a ticket this context never issued,
                                   or one whose result was already collected */
  SOR_ERR_CANCELLED = -8        /* the context was destroyed before the solve finished */
} sor_status;

/* Convergence quantity tested every check_every iterations (plain modes). */
typedef enum {
  SOR_STOP_MAXDELTA = 0,  /* max over the interior of |u_k - u_{k-1}| < tol (Section 2.1) */
  SOR_STOP_RESID_REL = 1  /* ||b - A u||_inf / ||b||_inf < tol, boundary moved into b
                             (||r||_inf alone when b == 0) */
} sor_stop;

typedef enum {
  SOR_FP64 = 0,        /* FP64 storage and arithmetic */
  SOR_FP32 = 1,        /* FP32 storage and arithmetic (reduced precision; error vs FP64 stated) */
  SOR_FP32_REFINE = 2  /* FP64 defect correction: r = b - A u and u += d in FP64, the
                          correction d from inner_sweeps FP32 red-black SOR sweeps on
                          A d = r starting from d = 0; stops on the relative residual */
} sor_precision;

/* Bit flags for sor_params.flags. */
#define SOR_FLAG_EXACT_ORDER 1 /* SOR_FP64: evaluate the update as
                                  (1-w)*u + (w/4)*(((N+S)+(W+E))+g) with every
                                  product and sum rounded separately (no fused
                                  multiply-add, no rescaling).  Slower on GB300,
                                  whose FP64 rate is low; results then equal a
                                  plain CPU evaluation bit for bit. */

typedef struct {
  int32_t n;            /* interior side N >= 1 (array side N+2) */
  int32_t precision;    /* sor_precision */
  double omega;         /* relaxation factor, 0 < w < 2; w <= 0 selects
                           w_opt = 2 / (1 + sin(pi / (N+1))) */
  double tol;           /* tolerance eps of the stopping test (strict <) */
  int32_t stop;         /* sor_stop; ignored by SOR_FP32_REFINE (always residual) */
  int32_t max_iters;    /* cap on red-black iterations (sweeps); >= 0 */
  int32_t check_every;  /* K >= 1: test only when the iteration count is a multiple of K
                           (Section 3.3).  SOR_FP32_REFINE tests after every correction. */
  int32_t inner_sweeps; /* SOR_FP32_REFINE: sweeps per correction (>= 1); 0 = 20 */
  int32_t flags;        /* SOR_FLAG_* */
  int32_t stall_window; /* > 0: residual tests only (SOR_FP32_REFINE, or SOR_STOP_RESID_REL): also
                           stop, with converged = 0, once this many residual tests in a row have
                           not produced a new smallest residual while staying within a factor 4
                           of it (a plateau: the tolerance is below what FP64 can reach for this
                           problem); a test further above ends the run.  0 = off.  Must be >= 0. */
} sor_params;

typedef struct {
  int32_t iterations;     /* red-black iterations (sweeps) carried out */
  int32_t converged;      /* 1 if the stopping test passed, 0 if the cap was hit */
  int32_t outer_steps;    /* SOR_FP32_REFINE: corrections applied; 0 otherwise */
  int32_t reserved;
  double final_maxdelta;  /* max |change| of the last iteration (plain modes; -1 if none) */
  double final_resid_rel; /* relative residual of the returned solution, in FP64 */
  double latency_s;       /* host wall time from the call (or submit) to the result */
  double device_s;        /* device time of the solve's kernels and copies (CUDA events) */
} sor_result;

/* Optional device-memory hooks: alloc(bytes, user) returns device memory or
 * NULL; free_(ptr, user) releases it.  Both NULL: cudaMalloc / cudaFree. */
typedef void *(*sor_alloc_fn)(size_t bytes, void *user);
typedef void (*sor_free_fn)(void *ptr, void *user);

/* Create a context on CUDA device `device`.
 *   hbm_budget_bytes: upper bound on the device memory the context holds for
 *     solves (0 = 90% of the free memory at creation).  A solve needing more
 *     than the whole budget fails with SOR_ERR_BUDGET; batch requests wait
 *     until enough of the budget is free.
 *   cuda_stream: cudaStream_t for sor_solve's work (NULL = a stream the
 *     library creates).  Batch work runs on a library-owned stream.
 * On success *out receives the context (free it with sor_destroy). */
sor_status sor_create(sor_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream,
                      sor_alloc_fn alloc, sor_free_fn free_, void *alloc_user);

/* Blocking solve of one problem.
 *   u0:    (N+2)^2 row-major initial profile; its ring is the Dirichlet data
 *          (Algorithm 1 input).  Host or device memory.
 *   f:     N*N row-major interior source of -Laplace(u) = f, or NULL for f = 0.
 *   u_out: (N+2)^2 row-major final profile (may equal u0).
 *   res:   optional result record.
 * Inputs are read before the call returns; u_out is written before it returns. */
sor_status sor_solve(sor_ctx *ctx, const sor_params *params, const double *u0, const double *f, double *u_out,
                     sor_result *res);

/* Blocking solve of one problem on a cube: the 3D grids the paper names as
 * the next step of its study (Section 5, Conclusion and Future Work), solved
 * by the same method -- Algorithm 1 with the update of Eq. 1, the
 * Gauss-Seidel value taken from the 7-point stencil:
 *   U <- (1-w) U + (w/6) ((((N + S) + (W + E)) + (D + U)) + h^2 f),
 * red = (i + j + k) even, red phase first.  FP32 (precision SOR_FP32), and
 * FP64 with SOR_FLAG_EXACT_ORDER, round every product and sum on its own in
 * that order; FP64 by default computes the same iteration with the neighbour
 * sums regrouped (in-plane pairs shared by two cells) and the unknowns
 * rescaled within each run of iterations between tests, one FMA per update
 * (within 1e-12 of the exact order in the tested solves).  The residual
 * r~ = (h^2 f + sum of the six neighbours) - 6 u is formed in FP64.
 * SOR_FP32_REFINE runs the defect correction on the cube: per outer step
 * the FP64 residual test (rho < tol), then inner_sweeps FP32 red-black sweeps
 * (exact order) on A d = (float)r~ from d = 0, then u += d in FP64; at most
 * max_iters / inner_sweeps corrections (results equal the CPU oracle's bit
 * for bit).
 *   params: n = interior side N (1 <= N <= 1200); omega <= 0 selects
 *           2 / (1 + sin(pi / (N+1))); stop, tol, max_iters, check_every as
 *           for sor_solve; precision SOR_FP64, SOR_FP32 or SOR_FP32_REFINE
 *           (inner_sweeps >= 0, 0 = 20); flags 0 or SOR_FLAG_EXACT_ORDER;
 *           stall_window >= 0 as for sor_solve.  Anything else returns
 *           SOR_ERR_INVALID_ARG.
 *   u0:    (N+2)^3 array indexed [k][i][j] (plane, row, column), its outer
 *          shell the Dirichlet data.  Host or device memory.
 *   f:     N^3 interior source of -Laplace(u) = f ([k][i][j]), or NULL.
 *   u_out: (N+2)^3 final values (may equal u0).  res: optional.
 * Device memory comes from the context's allocator and counts against its
 * budget (SOR_ERR_BUDGET when the solve does not fit). */
sor_status sor_solve3d(sor_ctx *ctx, const sor_params *params, const double *u0, const double *f, double *u_out,
                       sor_result *res);

/* Blocking solve of one problem with the compact 9-point stencil by
 * four-colour SOR (Section 3.1 names multi-colour SOR beside red-black SOR;
 * the diagonal couplings of the 9-point stencil need four colours,
 * c = 2 (i & 1) + (j & 1), updated in the order 0, 1, 2, 3).  Cell equation
 * 20 u = 4 (N + S + W + E) + (NW + NE + SW + SE) + 6 h^2 f, update
 *   U <- (1-w) U + (w/20) ((4 ((N + S) + (W + E)) + ((NW + NE) + (SW + SE))) + 6 h^2 f),
 * every product and sum rounded on its own in that order in FP32 and in FP64
 * with SOR_FLAG_EXACT_ORDER; FP64 by default regroups the sum as
 * (NW + 4 N + NE) + (SW + 4 S + SE) + 4 (W + E), the south triple of a cell
 * serving as the north triple of the cell two rows down, with fused
 * multiply-adds (within 1e-12 of the exact order in the tested solves).  The
 * residual r~ = (6 h^2 f + (4 s4 + sd)) - 20 u is formed in FP64 and b~
 * weighs the ring's edge neighbours by 4 and its diagonal ones by 1.
 * SOR_FP32_REFINE runs the defect correction with these sweeps: per outer
 * step the FP64 residual test (rho < tol), inner_sweeps FP32 four-colour
 * iterations (exact order) on A d = (float)r~ from d = 0, then u += d in
 * FP64; at most max_iters / inner_sweeps corrections (results equal the CPU
 * oracle's bit for bit).
 *   params: as for sor_solve with precision SOR_FP64, SOR_FP32 or
 *           SOR_FP32_REFINE (inner_sweeps >= 0, 0 = 20), flags 0 or
 *           SOR_FLAG_EXACT_ORDER, stall_window >= 0 as for sor_solve (else
 *           SOR_ERR_INVALID_ARG);
 *           omega <= 0 selects 2 / (1 + sin(pi / (N+1))).
 *   u0, f, u_out: as for sor_solve ((N+2)^2, N^2, (N+2)^2; host or device);
 *          the 9-point stencil also reads the ring's corners.
 * Device memory counts against the context's budget. */
sor_status sor_solve9(sor_ctx *ctx, const sor_params *params, const double *u0, const double *f, double *u_out,
                      sor_result *res);

/* Blocking solve of one plate by block two-colour SOR, the reading taken
 * here of the block-parallel SOR that Section 3.1 names beside red-black and
 * multi-colour SOR (it gives no definition of its own):
 *   - the interior is tiled into blocks of block_rows x block_cols cells,
 *     block (I, J) holding rows 1 + I*block_rows .. and columns
 *     1 + J*block_cols .. (the last blocks clipped at N);
 *   - block (I, J) has colour (I + J) mod 2; an iteration updates every
 *     colour-0 block, then every colour-1 block;
 *   - inside a block the cells are updated one at a time in row-major order
 *     with the update of Eq. 1 (5-point Gauss-Seidel value), each reading the
 *     newest value of every neighbour:
 *       U <- (1-w) U + (w/4) (((N + S) + (W + E)) + h^2 f),
 *     every product and sum rounded on its own in that order, in FP64, or in
 *     FP32 (precision SOR_FP32: u0 and h^2 f rounded once to FP32, the
 *     coefficients (float)(1-w) and (float)(w/4), the result widened).
 * Blocks of one colour share no edge, so they are updated at once, one warp
 * per block (the lanes take the block's rows as a wavefront, which reads the
 * same values as the row-major order).  1 x 1 blocks are red-black SOR with
 * red = (i + j) even first; one block covering the interior is SOR in
 * natural order.  Results equal the CPU reference bit for bit.
 *   params: n (1 <= N <= 60000), omega (<= 0 selects 2 / (1 + sin(pi / (N+1)))),
 *           stop (SOR_STOP_MAXDELTA or SOR_STOP_RESID_REL, tested when the
 *           iteration count is a multiple of check_every), tol, max_iters,
 *           check_every as for sor_solve; precision SOR_FP64 or SOR_FP32 (FP32
 *           stops on max|change| only, and stages each block with its halo
 *           in shared memory: (32 / s) (block_rows + 2) (block_cols + 2)
 *           floats, s the smallest power of two >= block_rows, at most
 *           200 KB); flags 0 or SOR_FLAG_EXACT_ORDER (the same: the order is
 *           always exact); stall_window must be 0.  Anything else returns
 *           SOR_ERR_INVALID_ARG.
 *   block_rows: 1 .. 32; block_cols: >= 1 (else SOR_ERR_INVALID_ARG).
 *   u0, f, u_out: as for sor_solve ((N+2)^2, N^2 or NULL, (N+2)^2; host or
 *          device memory; u_out may equal u0).  A device u_out holds the
 *          iterate during the solve.  res: optional (final_resid_rel is the
 *          scaled residual of the returned iterate, in FP64).
 * Device memory counts against the context's budget (SOR_ERR_BUDGET when
 * the solve does not fit). */
sor_status sor_solve_block(sor_ctx *ctx, const sor_params *params, int32_t block_rows, int32_t block_cols,
                           const double *u0, const double *f, double *u_out, sor_result *res);

/* Diagnostic of the failure path of the data-flow kernels (sor_solve3d and
 * sor_solve9 in FP64).  Their device-side waits are bounded: a warp whose
 * neighbours do not report progress gives up after a fixed number of polls,
 * records an error that the solve returns as SOR_ERR_INTERNAL, and the
 * context stays usable.  This call runs that wait, in one warp, on a progress
 * counter preset to 0 (nothing advances it, so the wait must give up) or to
 * 1 (complete: it must not), polling at most `polls` times (1 .. 2^21, about
 * 0.1 us each).  *timed_out = 1 when the wait gave up, 0 when it saw the
 * counter complete.  No GPU fault or hang is involved.
 * Returns SOR_ERR_INVALID_ARG for arguments out of range. */
sor_status sor_diag_flow_wait(sor_ctx *ctx, int polls, int preset, int *timed_out);

/* Measured FP64 rate of the context's GPU: the peak that bounds the FP64
 * colour phases (Eq. 1 evaluated in FP64, Section 3.1) on GB300, whose HBM
 * could feed them faster than its FP64 units compute.  A full-occupancy
 * grid runs independent chains of FP64 fused multiply-adds (kind 0) or
 * additions (kind 1) on the context's stream, timed with CUDA events (one
 * warm-up launch, then one timed launch of about 70 ms); *ops_per_s receives
 * the FP64 lane operations per second of the whole GPU (an FMA counts once;
 * its flops are twice that).  Blocks until done; allocates and frees a
 * 2.5 MB output buffer.  SOR_ERR_INVALID_ARG for another kind or a NULL
 * output. */
sor_status sor_diag_fp64_rate(sor_ctx *ctx, int kind, double *ops_per_s);

/* Diagnostic of the debug build's device-side index checks (no counterpart
 * in the paper: a test aid).  A library compiled with SOR_DEBUG_BOUNDS
 * checks, before a kernel touches a tile of a plate (pack, the colour-phase
 * sweeps, the fused FP32 sweeps, the residual and correction passes), that
 * the rows and columns it will read and write lie inside the slot's arrays;
 * a tile that does not is skipped and the solve returns SOR_ERR_INTERNAL
 * ("device-side index check failed") instead of touching memory outside
 * them.  This call sends one index below a one-element range through the
 * check (no memory is accessed at it) and sets *fired = 1 when the check
 * refused it and recorded the error, 0 in release builds, where the checks
 * are compiled away.  SOR_ERR_INVALID_ARG for a NULL output. */
sor_status sor_diag_bounds(sor_ctx *ctx, int *fired);

/* Non-blocking submission to the context's continuous-batching scheduler.
 * u0 and f are copied before the call returns.  u_out must stay valid until
 * sor_poll / sor_wait reports SOR_OK for the ticket; it is written then.
 * Requests are admitted in arrival order while their device memory fits the
 * budget, and every admitted request is stepped together with the others. */
sor_status sor_batch_submit(sor_ctx *ctx, const sor_params *params, const double *u0, const double *f,
                            double *u_out, uint64_t *ticket);

/* Non-blocking submission of a cube solve (the 3D 7-point red-black SOR of
 * sor_solve3d, with the same parameters, FP64 / FP32 / FP32_REFINE) to the
 * context's scheduler.  u0 ((N+2)^3) and f (N^3 or NULL) are copied before
 * the call returns; u_out must stay valid until sor_poll / sor_wait report
 * SOR_OK for the ticket.  Cube requests are solved whole, in arrival order,
 * by up to four worker threads, each on its own CUDA stream, concurrently
 * with the plates the scheduler steps and with each other; each waits for
 * device memory under the context's budget (SOR_ERR_BUDGET at submit only
 * when it needs more than the whole budget).  The result equals
 * sor_solve3d's for the same arguments, bit for bit.  Tickets are shared with
 * sor_batch_submit.  sor_destroy cancels queued cube requests and stops
 * running ones at their next chunk boundary (SOR_ERR_CANCELLED). */
sor_status sor_batch_submit3d(sor_ctx *ctx, const sor_params *params, const double *u0, const double *f,
                              double *u_out, uint64_t *ticket);

/* SOR_NOT_READY while the ticket is queued or running; SOR_OK (and *res)
 * once u_out holds the result -- the ticket is then retired; the solve's own
 * error status if it failed; SOR_ERR_UNKNOWN_TICKET otherwise. */
sor_status sor_poll(sor_ctx *ctx, uint64_t ticket, sor_result *res);

/* sor_poll, blocking up to timeout_s seconds (< 0: no limit); SOR_ERR_TIMEOUT
 * if the ticket is still pending then (it stays valid). */
sor_status sor_wait(sor_ctx *ctx, uint64_t ticket, double timeout_s, sor_result *res);

/* Cancel queued and running batch work (their tickets report
 * SOR_ERR_CANCELLED to nobody: the context is gone), release every device
 * buffer and stream the library created, and free the context. */
sor_status sor_destroy(sor_ctx *ctx);

/* Tuning and instrumentation knobs (sor_set_option / sor_get_option). */
typedef enum {
  SOR_OPT_TIMING = 1,          /* 1: time the sweep kernels with CUDA events (sor_get_stats) */
  SOR_OPT_GRAPHS = 2,          /* 1 (default): replay launch sequences as CUDA graphs */
  SOR_OPT_CHUNK = 3,           /* iterations per launched chunk between convergence polls (0 = auto) */
  SOR_OPT_TEMPORAL_DEPTH = 4,  /* FP32 sweeps: iterations fused per launch (0 = autotuned when
                                  SOR_OPT_AUTOTUNE is 1, else 6 with the tile kernels, 4 with the
                                  wavefront kernels; supported: 1 (unfused), tile 2, 3, 4, 6, 8,
                                  wavefront 2 .. 5; others round down) */
  SOR_OPT_AUTOTUNE = 5,        /* 1: on the first FP32 or defect-correction solve of a size bucket,
                                  time the fused-sweep kernel family, depth and rows per tile, and
                                  the corrections per graph, and keep the fastest (results are the
                                  same bit for bit whichever is chosen) */
  SOR_OPT_BATCH_MAX_SLOTS = 6, /* cap on concurrently admitted batch requests (0 = no cap) */
  SOR_OPT_CLUSTER = 7,         /* plain solves of small plates (N <= 384 in FP64, N <= 768 in FP32) in a
                                  single launch, exact operation order: 1 (default) = on a cooperative
                                  grid of many SMs when the stop test is max|change| (neighbouring bands
                                  exchange edge rows point to point, the stop test is decided behind the
                                  sweeps), else in one thread-block cluster; 3 = the same grid with a
                                  grid-wide barrier per colour phase; 2 = always the cluster; 0 = never.
                                  Results are identical in every form */
  SOR_OPT_FAST_CHAIN = 8,      /* 1 (default): the FP64 default path runs each chunk of iterations in one
                                  cooperative launch with neighbour-to-neighbour progress counters; 0: one
                                  launch per colour phase.  Results are identical either way */
  SOR_OPT_FUSED_KERNEL = 9,    /* FP32 sweeps: 0 (default) = chosen by grid size (tile kernels up to
                                  N = 6144 for SOR_FP32 and N = 12288 for the inner sweeps of
                                  SOR_FP32_REFINE, wavefront kernels above) or by the autotuner; 1 = tile
                                  kernels (a shared-memory tile pass per launch); 2 = wavefront kernels
                                  (a register wavefront per warp).  Results are identical either way */
  SOR_OPT_BATCH_PLAIN_STEP = 10, /* iterations per scheduler step of plain (FP64 / FP32) batch slots:
                                   0 (default) = tuned online over the scheduler's first rounds with
                                   plain slots (8, 16, 32, 64 tried, the highest update rate kept);
                                   > 0 = that many.  Results are identical either way: every slot
                                   stops on the device at its own tested iteration */
  SOR_OPT_CUBE_DEPTH = 11,      /* FP32 sweeps on cubes (sor_solve3d, SOR_FP32): 0 (default) = one
                                   data-flow launch per run of iterations, one colour phase at a time;
                                   1 or 2 = that many iterations fused per blocked launch, each tile of
                                   rows x packed columns x planes streamed through its planes with the
                                   colour phases run as a wavefront in shared memory (slower on GB300 at
                                   the sizes measured).  Results are identical */
  SOR_OPT_BLOCK_CHAIN = 12      /* sor_solve_block: blocks of one block row that a warp segment runs
                                   back to back, its wavefront carried from one into the next so it
                                   ramps up and down once per run: 0 (default) = enough blocks for
                                   about 128 columns per run; k > 0 = k blocks.  Results are identical */
} sor_option;

sor_status sor_set_option(sor_ctx *ctx, int32_t option, int64_t value);
sor_status sor_get_option(sor_ctx *ctx, int32_t option, int64_t *value);

/* Counters accumulated since sor_create or the last sor_reset_stats. */
typedef struct {
  uint64_t solves;            /* sor_solve calls completed */
  uint64_t batch_completed;   /* batch tickets completed */
  uint64_t sweep_launches;    /* colour half-sweep (or fused sweep) kernel launches issued */
  uint64_t lattice_updates;   /* interior cell updates performed (sweeps x N^2) */
  double sweep_ms;            /* CUDA-event time of the timed sweep chunks (SOR_OPT_TIMING) */
  uint64_t timed_launches;    /* sweep launches inside those timed chunks */
  uint64_t timed_updates;     /* lattice updates inside those timed chunks */
  uint64_t bytes_reserved;    /* device bytes currently held for solves */
  uint64_t bytes_peak;        /* high-water mark of bytes_reserved */
  uint64_t kernel_launches;   /* kernel launches of sor_solve calls, every kind (graph replays included) */
  uint64_t batch_plain_step;  /* iterations per scheduler step of plain batch slots in use (0 = none yet) */
} sor_stats;

sor_status sor_get_stats(sor_ctx *ctx, sor_stats *out);
sor_status sor_reset_stats(sor_ctx *ctx);

/* Text of the last error recorded on this context (thread-safe copy). */
sor_status sor_last_error(sor_ctx *ctx, char *buf, size_t len);
const char *sor_status_string(int32_t status);

/* w_opt = 2 / (1 + sin(pi / (N+1))) for the 5-point Laplacian (Young). */
double sor_omega_opt(int32_t n);

/* Blocking FP64 solve that allocates no memory (no counterpart in the paper:
 * it exists for library integration only).
 *
 * For callers that must not allocate device memory while they run: hosts
 * with a fixed memory plan (real-time or embedded code that reserves every
 * buffer up front), plug-ins whose framework owns the device allocator, and
 * code that may not call cudaMalloc at all.  sor_solve allocates its working
 * buffers; this call instead keeps them in one fixed array of about 4.8 MB of
 * device memory built into the library, which every GPU that loads the
 * library holds until the process exits.
 *
 *   params: as for sor_solve, restricted to precision SOR_FP64 and
 *           1 <= n <= 512; larger grids or other precisions return
 *           SOR_ERR_INVALID_ARG.  The update is evaluated in exact order
 *           (the SOR_FLAG_EXACT_ORDER path of sor_solve, whose results it
 *           equals bit for bit) whatever the flag says.
 *   u0, f, u_out: DEVICE pointers on the current device (f may be NULL);
 *           host pointers and pointers on another device return
 *           SOR_ERR_INVALID_ARG.
 *   res:    optional; device_s is 0 (no events are created).
 *   cuda_stream: stream for the work (NULL = the legacy default stream).
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  Every call
 * shares the one array and it keeps the previous call's contents, so each call
 * clears what it reads first.  Calls that overlapped on the GPU would race on
 * the array: the library serialises callers and each call returns only after
 * its work on the stream has finished, on error returns too.  Allocates nothing: no cudaMalloc,
 * cudaFree or allocating library call. */
sor_status sor_solve_static(const sor_params *params, const double *u0, const double *f, double *u_out,
                            sor_result *res, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SOR_H_ */
