/*
 * srfmg.h -- C ABI of the GB300 (sm_103a) segmental-refinement full multigrid
 * solver for the cell-centred 7-point Poisson problem on the unit cube.
 *
 * Method: Adams, Brown, Knepley, Samtaney, "Segmental Refinement: A Multigrid
 * Technique for Data Locality".
 *   problem        Sec. 2, Eq. (eq:eq), Eq. (eq:deq): -Delta u = f in (0,1)^3,
 *                  u = 0 on the boundary, N^3 cells, cell centres (i + 1/2)/N.
 *                  The library solves A u = f with A = -Delta_h,
 *                  (A u)_i = (6 u_i - sum of the 6 neighbours) N^2, ghost cells
 *                  outside the domain holding minus their mirror cell (Sec. 3.3).
 *   FMG            Sec. 3.2, Fig. "Full multigrid": F(alpha, nu1, nu2) cycles
 *                  built on the FAS V-cycle of Sec. 3.1, Fig. "FAS multigrid
 *                  V-cycle", Eq. (eq:cresid2).
 *   SR-FMG         Sec. 4, Figs. "FMG segmental refinement" and "FAS V-cycle
 *                  segmental refinement": the K finest levels are split into
 *                  segments of seg^3 genuine cells (on the finest level) plus
 *                  J_k buffer cells per side, Eq. (eq:nb); levels 0 and below
 *                  are solved globally.
 *   components     Sec. 5.1: Chebyshev smoothers (degree nu1/nu2 around the
 *                  V-cycle, alpha before it), 8-child average restriction,
 *                  cell-centred trilinear prolongation.
 *
 * Conventions for every entry point:
 *   - grids are contiguous float64 arrays of n^3 values (of nx ny nz values,
 *     nx = n len[0], ny = n len[1], nz = n len[2], on a rectangular domain),
 *     index [z][y][x], x fastest, owned by the caller; below "n^3 doubles"
 *     stands for nx ny nz;
 *   - "device" pointers must be CUDA device memory of the device that was
 *     current when the handle was created; "host" pointers are host memory;
 *   - stream is a cudaStream_t (NULL = the legacy default stream);
 *   - return value: SR_OK (0) or a negative SR_ERR_* code; no entry point
 *     aborts the process or prints.
 */
#ifndef SRFMG_H
#define SRFMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SR_FMG_MAXK 12

/* status codes */
#define SR_OK 0
#define SR_ERR_INVALID (-1)          /* bad argument or inconsistent configuration */
#define SR_ERR_UNSUPPORTED_SIZE (-2) /* grid size the solver does not handle */
#define SR_ERR_OOM (-3)              /* device or host allocation failed */
#define SR_ERR_CUDA (-4)             /* a CUDA call failed (launch, copy, sync) */
#define SR_ERR_TIMEOUT (-5)          /* a bounded device-side wait gave up */
#define SR_ERR_NONFINITE (-6)        /* the right-hand side holds a NaN or Inf */
#define SR_ERR_NO_DEVICE (-7)        /* no usable CUDA device */

/* precision modes */
#define SR_FP64 0   /* every step in float64 */
#define SR_MIXED 1  /* float32 smoothing, residuals and transfers inside a float64
                       defect-correction loop; coarse right-hand sides (tau) and
                       the coarsest solve in float64 arithmetic */

typedef struct sr_fmg_s* sr_fmg_t;

/*
 * Solver configuration.  sr_fmg_default_config fills it for a given n.
 *   n         fine cells per unit length (h = 1/n); the fine grid has
 *             n len[0] x n len[1] x n len[2] cells, fewer than 2^31.  n must
 *             halve down to the coarsest grid.
 *   n_coarse  cells per unit length of the coarsest grid, solved exactly
 *             (Sec. 3.1, the "else" branch of FASMGV); 0 = keep halving until
 *             2 or 3 remain.  At most 16.  Grids of up to 512 cells use a
 *             dense inverse; larger ones, with at most 32 cells per axis, the
 *             separable sine-transform solve (about 2 (nx + ny + nz) float64
 *             operations per cell); other coarsest grids of up to 4096 cells
 *             the dense inverse again, and anything larger is
 *             SR_ERR_UNSUPPORTED_SIZE.  A deeper exact solve (16) lets FMG
 *             reach an algebraic error well below the discretisation error
 *             (Sec. 3.2: FMG is asymptotically exact once the coarsest
 *             solve and the V-cycle are accurate enough).
 *   seg       genuine segment edge on the finest level (segments are cubes);
 *             0 = plain FMG (no segmental refinement).  n % seg == 0 and
 *             seg % 2^K == 0.
 *   K         number of SR levels (the K finest levels); 0 = plain FMG.
 *   A, B      buffer schedule J_k = 2 floor((A + B (K - k)) / 2), Eq. (eq:nb),
 *             used when use_J == 0.
 *   use_J, J  when use_J != 0, J[k-1] is the buffer width J_k, k = 1..K;
 *             every J_k must be even and J_{k-1} >= J_k / 2.
 *   alpha, nu1, nu2   Chebyshev degrees of the F(alpha, nu1, nu2) cycle (1, 2, 2).
 *   cheb_lo, cheb_hi  Chebyshev interval as fractions of lambda_max(D^-1 A)
 *             (D = w0 n^2 the diagonal; lambda_max = 2 for the 7-point
 *             operator, the largest corner value of the symbol / w0 for a
 *             27-point one); defaults 1/6 and 1.
 *   precision SR_FP64, or SR_MIXED: the whole FMG / SR-FMG solve S32 runs in
 *             float32 storage and arithmetic (tau right-hand sides and the
 *             coarsest solve in float64 arithmetic) inside float64 defect
 *             correction: u = S32(f), then n_outer - 1 times
 *             u += S32(f - A u) with the defect in float64 (no counterpart in
 *             the paper, which states no precision).
 *   n_outer   SR_MIXED passes, 1..16 (0 = 2).
 *   mbs       maximum buffer schedule (Sec. 5.2.1): J_1 = A (even) and
 *             J_k = 2^(k-1) J_1, so every coarser compute region is exactly
 *             the support of the next finer one; overrides A, B and J.
 *   len       the domain [0, len[0]] x [0, len[1]] x [0, len[2]] in unit
 *             lengths, each 1..64 (0 reads as 1); the paper's experiments
 *             use (2, 1, 1) with 4 x 2 x 2 segments (Sec. 5.1).
 *   stencil   7 (0 reads as 7): A u = n^2 (6 u - sum of the 6 face
 *             neighbours), Eq. (eq:deq) with L = -Delta; or 27:
 *             A u = n^2 (w0 u - w[0] sum_faces - w[1] sum_edges
 *             - w[2] sum_corners), w0 = 6 w[0] + 12 w[1] + 8 w[2], the
 *             paper's "27-point finite volume stencil" (Sec. 5.1).  The
 *             weights must be consistent with -Delta (w[0] + 4 w[1] + 4 w[2]
 *             = 1) and give a positive definite operator; 27 requires
 *             SR_FP64.
 *   graph     1: sr_fmg_solve_async (and sr_fmg_solve, sr_fmg_solve_host)
 *             queue the whole solve as one CUDA graph, captured on the
 *             first call for an (f, u) pair -- and again when the pair
 *             changes -- and relaunched afterwards (same kernels, same
 *             results, fewer launch gaps); solves made while the per-kernel
 *             profiler is on launch kernel by kernel.  Not for use inside
 *             the caller's own stream capture.  0 (default): kernel by
 *             kernel.
 *   seg_first, seg_count  segment range (SR_FP64 with seg > 0, K > 0): the
 *             handle holds and processes only segments seg_first ..
 *             seg_first + seg_count - 1, numbered x fastest over the grid of
 *             segments (n len[0] / seg of them along x), and solves through
 *             the stage entry points below, one handle per process or GPU
 *             sharing the segments of one problem; the global levels (the
 *             transition level and below) are solved redundantly by every
 *             handle (Sec. 7: redundant coarse-grid solves instead of idle
 *             processes).  seg_count = 0 (default): all segments.
 */
typedef struct {
  int n;
  int n_coarse;
  int seg;
  int K;
  int A, B;
  int use_J;
  int J[SR_FMG_MAXK];
  int alpha, nu1, nu2;
  double cheb_lo, cheb_hi;
  int precision;
  int n_outer;
  int mbs;
  int len[3];
  int stencil;
  double w[3];
  int graph;
  int seg_first, seg_count;
} sr_fmg_config;

/* Fill cfg with the defaults for an n^3 grid: unit cube, 7-point operator,
 * plain FMG, F(1,2,2), Chebyshev interval [1/6, 1] * lambda_max, coarsest
 * grid 2^3 or 3^3, buffers A = 8, B = 0, SR_FP64, n_outer = 2. */
void sr_fmg_default_config(sr_fmg_config* cfg, int n);

/* Validate cfg, build the level and segment plan and allocate the device
 * workspace on the current device.  *out receives the handle (NULL on error).
 * Errors: SR_ERR_INVALID, SR_ERR_UNSUPPORTED_SIZE, SR_ERR_OOM, SR_ERR_CUDA,
 * SR_ERR_NO_DEVICE. */
int sr_fmg_create(sr_fmg_t* out, const sr_fmg_config* cfg);

/* Release the workspace and the handle (NULL is accepted). */
int sr_fmg_destroy(sr_fmg_t h);

/* Bytes of device memory the handle holds. */
int sr_fmg_workspace_bytes(sr_fmg_t h, size_t* bytes);

/* Solve A u = f by FMG or SR-FMG.  f_dev, u_dev: device arrays of n^3
 * doubles; u_dev receives the solution (its prior content is ignored).  The
 * work is queued on stream; the call then waits for the stream and returns
 * the solve's status (SR_ERR_NONFINITE if f holds a NaN or Inf, in which case
 * u_dev is undefined).  f_dev and u_dev must not overlap. */
int sr_fmg_solve(sr_fmg_t h, const double* f_dev, double* u_dev, void* stream);

/* As sr_fmg_solve, but only queues the work and returns launch errors; the
 * solve's own status is read later by sr_fmg_check.  Calls on one handle must
 * not run concurrently (they share the workspace). */
int sr_fmg_solve_async(sr_fmg_t h, const double* f_dev, double* u_dev, void* stream);

/* Wait for stream and return the status of the solves queued on h since the
 * previous check (SR_OK, SR_ERR_NONFINITE, SR_ERR_TIMEOUT); the status is
 * then cleared. */
int sr_fmg_check(sr_fmg_t h, void* stream);

/* End-to-end solve from host memory: copies f_host (n^3 doubles) to the
 * device, solves, copies the solution to u_host, waits for stream.  Page-
 * locked host buffers give the fastest copies; pageable memory also works. */
int sr_fmg_solve_host(sr_fmg_t h, const double* f_host, double* u_host, void* stream);

/*
 * Iterative V-cycle solver, the comparison solver of Sec. 5.3 (V-cycles to
 * a relative residual tolerance; Fig. "Errors of all solvers"): starting
 * from the values in u_dev (zero them for the paper's setting), apply the
 * FAS V-cycle of Fig. "FAS multigrid V-cycle" on the global grid until
 *   ||f - A u||_inf <= rtol * ||f||_inf      or      max_cycles cycles ran.
 * h must be a plain float64 handle (seg == 0 or K == 0, SR_FP64), else
 * SR_ERR_INVALID.  f_dev, u_dev: device arrays of n^3 doubles, C order
 * [z][y][x], not overlapping; the caller owns them.  rtol >= 0,
 * max_cycles >= 0.  On return *cycles = V-cycles applied and *rel_resid =
 * the final ||f - A u||_inf / ||f||_inf (0 when both are 0, HUGE_VAL when
 * only f is 0); SR_OK also when max_cycles ran out before rtol was met
 * (compare *rel_resid with rtol).  Synchronous: it reads the residual norm
 * back after every cycle.  SR_ERR_NONFINITE if f or a residual is not finite.
 */
int sr_fmg_vsolve(sr_fmg_t h, const double* f_dev, double* u_dev, double rtol, int max_cycles,
                  int* cycles, double* rel_resid, void* stream);

/*
 * Pipelined end-to-end solves from host memory.  Each call queues: the copy
 * of f_host (n^3 doubles) into one of two device staging slots on an internal
 * stream, the solve on `stream`, and the copy of the solution to u_host on a
 * second internal stream; consecutive calls alternate slots, so one call's
 * copies overlap its neighbours' solves.  The host buffers must stay valid
 * and unchanged until sr_fmg_check_host returns (page-locked memory lets
 * the copies run asynchronously).  sr_fmg_check_host waits for every copy
 * out and returns the accumulated status of the solves (as sr_fmg_check).
 */
int sr_fmg_solve_host_async(sr_fmg_t h, const double* f_host, double* u_host, void* stream);
int sr_fmg_check_host(sr_fmg_t h);

/*
 * Stage-by-stage SR-FMG solve, for sharing the segments of one problem among
 * several handles (segment ranges; any FP64 SR handle works, one handle then
 * solving alone).  Each SR stage k = 1..K (Fig. "FMG segmental refinement")
 * is split at the transition level, the one step of the method where
 * segments exchange data (Sec. 4):
 *   sr_fmg_stage_down(h, f, k)   k = 1 first runs the f hierarchy and the
 *                       global FMG up to the transition level; then the FMG
 *                       prolongation onto level k, S^alpha, and the down-leg
 *                       of the SR V-cycle on the handle's segments, which
 *                       owner-write their genuine transition-level cells of
 *                       \hat I u_1 and of the restricted residual into the
 *                       two exchange arrays (all other cells zero).
 *   sr_fmg_stage_buffers(h, &uhat0, &rho0, &count)   device pointers of the
 *                       two exchange arrays, count doubles each (the
 *                       transition level's cells, C order); owned by h.
 *   (the caller)        replaces both arrays, on every handle, by their sum
 *                       over all handles of the problem (an all-reduce): as
 *                       every cell has one owner the sum is exact, and every
 *                       handle then holds the whole transition level.
 *   sr_fmg_stage_up(h, f, k, u)  the transition-level right-hand side, the
 *                       global V-cycle (redundant on every handle) and the
 *                       up-leg on the handle's segments; after k = K the
 *                       genuine finest cells of the handle's segments go to
 *                       u (n^3 doubles; the other cells are not written).
 * f: the whole right-hand side on every handle (device, n^3 doubles).  The
 * calls queue work on stream and return launch errors; sr_fmg_check reports
 * a non-finite f.  Handles with a segment range refuse sr_fmg_solve and the
 * other whole-solve entry points (SR_ERR_INVALID).  SR_MIXED handles and
 * plain FMG handles are refused too.  Stage calls on one handle run in
 * order: down(1), exchange, up(1), down(2), ..., up(K).
 */
int sr_fmg_stage_down(sr_fmg_t h, const double* f_dev, int k, void* stream);
int sr_fmg_stage_buffers(sr_fmg_t h, double** uhat0, double** rho0, size_t* count);
int sr_fmg_stage_up(sr_fmg_t h, const double* f_dev, int k, double* u_dev, void* stream);

/*
 * Launch shape of the handle's kernels (results do not depend on it, bit
 * for bit): zchunk = cells in z that a thread of the z-column kernels walks
 * (1..256, default 16; the float32 prolongation walks twice that, the
 * float32 residual + restriction a quarter of it in coarse cells, at least
 * one), cells_per_thread = cells a thread of the per-cell kernels takes
 * (1..16, default 2).  Drops the handle's captured graphs;
 * batches holding the handle re-capture theirs at their next solve.  The
 * batch autotuner (paper_1406_7808_gb300/autotune.py) picks both per grid
 * size by timing.  The paper has no counterpart.
 */
int sr_fmg_set_launch_shape(sr_fmg_t h, int zchunk, int cells_per_thread);
int sr_fmg_launch_shape(sr_fmg_t h, int* zchunk, int* cells_per_thread);

/* Number of kernel launches the handle's last queued solve made. */
int sr_fmg_launches_per_solve(sr_fmg_t h, int* launches);

/*
 * Per-kernel profile.  sr_fmg_profile(h, 1) clears the counters and starts
 * bracketing every kernel launch of later solves on h with CUDA events (a few
 * microseconds of overhead per launch); sr_fmg_profile(h, 0) stops.  Both
 * wait for the device.  sr_fmg_profile_read waits for the recorded launches
 * and returns, for one kernel kind (0 <= kind < sr_fmg_profile_kinds()), its
 * name (static string), launch count, summed device time in milliseconds, and
 * the summed algorithmic floating-point operations (each add, multiply or
 * fused multiply-add counts one) and bytes (each array element read or
 * written once) of those launches.  Kind names ending in "_f32" are float32
 * storage and arithmetic, "_mixed" float32 storage with float64 arithmetic,
 * the others float64.
 */
int sr_fmg_profile(sr_fmg_t h, int enable);
int sr_fmg_profile_kinds(void);
int sr_fmg_profile_read(sr_fmg_t h, int kind, const char** name, long long* launches,
                        double* ms, double* ops, double* bytes);

/*
 * Measured peak fused multiply-add rate of the current device: bits = 64
 * (float64) or 32 (float32).  *lane_ops_per_s receives the lane operations
 * per second (one FMA on one lane counts one) of a kernel that keeps every
 * SM's pipe busy with independent FMA chains, best of three event-timed
 * launches on stream after one warm-up; the call waits for them.  It
 * allocates and frees a small output buffer.  The solver's float64 kernels
 * are bound by this rate, not by HBM (the roofline denominator of the
 * stencil passes; the paper, which reports CPU results, has no
 * counterpart).  Errors: SR_ERR_INVALID (bits, null output), SR_ERR_OOM,
 * SR_ERR_CUDA, SR_ERR_NO_DEVICE.
 */
int sr_probe_fma_rate(int bits, double* lane_ops_per_s, void* stream);

/*
 * Allocation-failure injection and bookkeeping, for testing the error paths
 * (the paper has no counterpart).  Every device allocation the library makes
 * for a handle (workspace, plan, staging buffers) is counted.
 *   sr_debug_fail_alloc(n)  n > 0: the n-th such allocation from now fails
 *                           as if the device had run out of memory (the
 *                           entry point that made it returns SR_ERR_OOM and
 *                           releases what it had allocated); 0 turns the
 *                           injection off.  SR_ERR_INVALID for n < 0.
 *   sr_debug_alloc_count()  allocations attempted since the library loaded
 *   sr_debug_live_bytes()   bytes of device memory the library's handles
 *                           hold now
 * Process-wide; not meant for concurrent use with other threads creating
 * handles.
 */
int sr_debug_fail_alloc(int nth);
long long sr_debug_alloc_count(void);
long long sr_debug_live_bytes(void);

/*
 * Last-stage trimming switch, for testing (the paper has no counterpart).
 * By default (enable = 1) the last stage's correction, residual and update
 * on every SR level run only on the cells the finest genuine cells still
 * depend on; every value kept is computed by the same arithmetic as on the
 * full box, so the result is bitwise the same either way.  enable = 0 runs
 * them on the full regions.  Drops the handle's captured graphs.
 */
int sr_debug_last_stage_trim(sr_fmg_t h, int enable);

/*
 * Segment-resident legs (the float32 inner solver of SR_MIXED, 7-point,
 * degree-2 smoothers): on every SR level below a stage's top level whose
 * boxes fit, the down-leg (coarse right-hand side, pre-smoother, residual and
 * restriction) and the up-leg (correction, post-smoother, w - t) of each
 * segment run as one launch of a thread-block cluster per segment that
 * holds the segment's box in shared memory (Sec. 4; the near-memory
 * residency of a segment, Sec. 6), with the same results bit for bit as the
 * separate kernels.  sr_debug_segment_legs(h, 1, ...) runs the legs;
 * 0 (the default) the separate kernels, which are faster on GB300 (the
 * mixed 512^3 solve: 24.2 ms against 30 to 32 ms with the legs).  *levels (may
 * be NULL) receives a bit mask of the SR levels j (bit j) that have a leg.
 * Drops the handle's captured graphs.
 *
 * sr_debug_force_wait_timeout(h, 1) makes every bounded device-side wait of
 * the legs (when they run) expect data that never arrives, so each wait
 * runs out (after about a second) and the solve reports SR_ERR_TIMEOUT; 0
 * turns it off.
 * For testing that path: nothing faults or hangs, the handle stays usable.
 */
int sr_debug_segment_legs(sr_fmg_t h, int enable, int* levels);
int sr_debug_force_wait_timeout(sr_fmg_t h, int enable);

/*
 * The global V-cycle in one persistent launch (float64 handles, 7-point
 * operator, degree-2 smoothers; Sec. 3.1, Fig. "FAS multigrid V-cycle"):
 * from the first global level of at most 64^3 cells down to the coarsest
 * grid, every pass of the cycle runs inside one cooperative launch whose
 * blocks meet at a grid barrier between passes, with the same results bit
 * for bit as the separate kernels.  Its barrier waits are bounded (about a
 * second each; SR_ERR_TIMEOUT on expiry; sr_debug_force_wait_timeout makes
 * them run out).  sr_debug_persistent_vcycle(h, 0, ...) runs the separate
 * kernels instead (for comparisons); 1 (the default) the persistent cycle.
 * *available (may be NULL) receives 1 if the handle can use it.  Drops the
 * handle's captured graphs.
 */
int sr_debug_persistent_vcycle(sr_fmg_t h, int enable, int* available);

/*
 * Testing hook for the float64 -> float32 rounding the mixed mode's
 * float64-arithmetic kernels store their results with (a round-to-nearest-
 * even conversion on the integer pipe): out[i] = in[i] rounded, device
 * arrays of n values; waits for stream.  Results must equal the IEEE 754
 * conversion bit for bit.
 */
int sr_debug_narrow(const double* in, float* out, long long n, void* stream);

/* Human-readable name of a status code (static string). */
const char* sr_fmg_status_string(int status);

/*
 * Single components on a whole n^3 grid, device arrays, for testing each
 * step against a reference.  Each call allocates and frees its own
 * temporaries and waits for stream before returning.
 *   sr_op_apply        out = A u                                  (Eq. eq:deq)
 *   sr_op_residual     r = f - A u                                (Fig. "FAS multigrid V-cycle")
 *   sr_op_smooth       u <- S^nu(A, u, f), Chebyshev on D^-1 A over
 *                      [cheb_lo, cheb_hi] * 2                     (Sec. 5.1)
 *   sr_op_restrict     ac = 8-child average of a, (n/2)^3 result  (Sec. 5.1)
 *   sr_op_prolong      af = trilinear interpolation of the nc^3 grid ac onto
 *                      (2 nc)^3                                  (Sec. 5.1)
 *   sr_op_coarse_solve u = A^-1 f exactly, n <= 32                (Sec. 3.1)
 *   sr_op_vcycle       one FAS V-cycle on u with right-hand side f, using
 *                      cfg's cycle parameters (seg and K ignored)  (Sec. 3.1)
 */
int sr_op_apply(int n, const double* u, double* out, void* stream);
int sr_op_residual(int n, const double* f, const double* u, double* r, void* stream);
int sr_op_smooth(int n, int nu, double cheb_lo, double cheb_hi, const double* f, double* u,
                 void* stream);
int sr_op_restrict(int n, const double* a, double* ac, void* stream);
int sr_op_prolong(int nc, const double* ac, double* af, void* stream);
int sr_op_coarse_solve(int n, const double* f, double* u, void* stream);
int sr_op_vcycle(const sr_fmg_config* cfg, const double* f, double* u, void* stream);

/*
 * The same components on any grid and operator of the configuration: the
 * grid has n len[0] x n len[1] x n len[2] cells (cfg->n per unit length),
 * the operator is cfg->stencil / cfg->w, the smoother interval
 * cfg->cheb_lo / cfg->cheb_hi.  For restrict cfg describes the fine grid,
 * for prolong the coarse grid (the output has twice the cells per
 * dimension).  Arrays unpadded, C order [z][y][x], device memory.
 */
int sr_op_apply_ex(const sr_fmg_config* cfg, const double* u, double* out, void* stream);
int sr_op_residual_ex(const sr_fmg_config* cfg, const double* f, const double* u, double* r,
                      void* stream);
int sr_op_smooth_ex(const sr_fmg_config* cfg, int nu, const double* f, double* u, void* stream);
int sr_op_restrict_ex(const sr_fmg_config* cfg, const double* a, double* ac, void* stream);
int sr_op_prolong_ex(const sr_fmg_config* cfg, const double* ac, double* af, void* stream);
int sr_op_coarse_solve_ex(const sr_fmg_config* cfg, const double* f, double* u, void* stream);

/*
 * Batched solves (many right-hand sides on grids of any sizes and
 * configurations).  A batch groups existing handles (not owned: destroy the
 * batch before its handles); problem i is solved by hs[i].  The first solve
 * for a set of f / u device pointers captures every problem's solve into one
 * CUDA graph whose branches run on capture streams forked from stream
 * (biggest problems first, each to the least loaded branch); later solves
 * with the same pointers relaunch that graph with one cudaGraphLaunch.  The
 * first batch solve must not itself be issued during a stream capture.
 *   sr_fmg_batch_solve        blocking; returns the first failing status
 *   sr_fmg_batch_solve_async  queue only; sr_fmg_batch_check waits and reports
 *   sr_fmg_batch_autotune     times the graph with 1, 2, 4, ... 32 branches
 *                             (at most count) and keeps the fastest; results
 *                             do not depend on the choice
 *   sr_fmg_solve_batched      one-shot: batch, solve, release
 * Errors: SR_ERR_INVALID for null or non-device pointers, repeated handles or
 * outputs, f overlapping its u; SR_ERR_CUDA for failed capture or launch.
 */
typedef struct sr_fmg_batch_s* sr_fmg_batch_t;
int sr_fmg_batch_create(sr_fmg_batch_t* out, const sr_fmg_t* hs, int count);
int sr_fmg_batch_destroy(sr_fmg_batch_t b);
int sr_fmg_batch_solve(sr_fmg_batch_t b, const double* const* f, double* const* u, void* stream);
int sr_fmg_batch_solve_async(sr_fmg_batch_t b, const double* const* f, double* const* u,
                             void* stream);
int sr_fmg_batch_check(sr_fmg_batch_t b, void* stream);
int sr_fmg_batch_autotune(sr_fmg_batch_t b, const double* const* f, double* const* u,
                          void* stream, int* streams_out, float* ms_out);
int sr_fmg_batch_set_streams(sr_fmg_batch_t b, int streams);
int sr_fmg_solve_batched(sr_fmg_t* hs, const double* const* f, double* const* u, int count,
                         void* stream);

/*
 * Chebyshev smoother that allocates nothing (the paper has no counterpart:
 * this is a service for callers that cannot allocate device memory where they
 * smooth, e.g. when all device memory is handed out by another allocator or
 * when cudaMalloc's implicit synchronisation is not acceptable).
 * Same operation and arguments as sr_op_smooth on device arrays f and u of
 * n^3 doubles, but the scratch (two n^3 arrays and a grid descriptor) lives in
 * one fixed device array of this library, sized for n <= SR_NOALLOC_MAX_N
 * (4 MiB + 256 bytes; every GPU that loads the library holds it until the
 * process exits).  No cudaMalloc, cudaFree or allocating library call is made.
 *   - n > SR_NOALLOC_MAX_N returns SR_ERR_UNSUPPORTED_SIZE; bad arguments
 *     return SR_ERR_INVALID.
 *   - The work is queued on stream and the call returns without waiting.
 *   - The first call on a device looks up the device address of the scratch
 *     array (once per device, with that device current); make that first call
 *     before any stream capture.
 *   - All calls share the one scratch array, which keeps the last call's
 *     contents: calls that overlap on the GPU (other streams or threads, or
 *     another solver using this entry point at the same time) race and give
 *     wrong results.  Nothing in the scratch needs to start at zero.
 */
#define SR_NOALLOC_MAX_N 64
int sr_op_smooth_noalloc(int n, int nu, double cheb_lo, double cheb_hi, const double* f,
                         double* u, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SRFMG_H */
