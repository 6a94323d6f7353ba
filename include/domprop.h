/*
 * domprop.h -- C ABI of the GB300 domain-propagation library (libdomprop.so).
 *
 * The library tightens variable bounds of a system of linear constraints
 *
 *     lhs <= A x <= rhs,      lb <= x <= ub,      x_j integer for some j
 *
 * (Eq. 1 of Sofranac, Gleixner, Pokutta, "Accelerating Domain Propagation:
 * an Efficient GPU-Parallel Algorithm over Sparse Matrices", arXiv 2009.07785)
 * by round-synchronous domain propagation (Alg. 2 of that paper): every
 * round computes each row's minimum and maximum activity (Def. 1, Eq. 2a/2b)
 * with infinite contributions counted apart (Sec. 3.4), derives a bound
 * candidate for every nonzero from the row's residual activity (Eq. 3a/3b in
 * the residual form of Eq. 5a/5b), rounds integer candidates (Step 3), and
 * applies candidates that improve a bound by more than a threshold
 * (Sec. 1.1, last paragraph; Sec. 3.5) with atomic min/max.  Rounds repeat on
 * the device, with no host synchronisation between rounds, until a round
 * changes nothing, detects infeasibility (Step 2, or crossing bounds), or a
 * round cap is reached (Sec. 4.1 uses 100).
 *
 * Conventions shared by every entry point
 *   - Return value: >= 0 on success (see each function), a negative DP_ERR_*
 *     code on failure.  No C++ exception crosses this boundary.
 *   - Infinite bounds and sides: IEEE +-inf, or any value whose magnitude is
 *     >= params.inf_threshold.
 *   - All floating-point data is IEEE binary64; all arithmetic on the device
 *     is binary64 as well.
 *   - Pointers documented as "host or device" may point to host memory
 *     (pageable or pinned) or to device memory of the context's GPU; the
 *     library detects which with cudaPointerGetAttributes.
 *   - The library never frees or retains caller memory.
 *   - Calls on one dp_ctx are not thread-safe: serialise them.
 */
#ifndef DOMPROP_H
#define DOMPROP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------- */
#define DP_OK 0
#define DP_CAP_HIT 1             /* success, but the round cap was hit    */
#define DP_ERR_INVALID_ARG (-1)  /* null pointer, bad size, bad params     */
#define DP_ERR_BAD_CSR (-2)      /* malformed CSR, column out of range,
                                    zero / NaN / infinite coefficient      */
#define DP_ERR_NAN_INPUT (-3)    /* NaN in lb, ub, lhs or rhs, or lb=+inf,
                                    ub=-inf, lhs=+inf, rhs=-inf            */
#define DP_ERR_OOM (-4)          /* device or host allocation failed       */
#define DP_ERR_CUDA (-5)         /* a CUDA runtime call failed             */
#define DP_ERR_TIMEOUT (-6)      /* a bounded device wait gave up          */

typedef struct dp_ctx dp_ctx;       /* one GPU + one stream + scratch      */
typedef struct dp_matrix dp_matrix; /* a constraint matrix resident on GPU */

/*
 * Tolerances and limits.  The paper fixes only the round cap (100, Sec. 4.1);
 * the other values are readings of passages that name a threshold without a
 * value (Sec. 1.1 last paragraph: improvement threshold; Step 3: rounding of
 * integer bounds).  dp_params_default() fills in:
 *   max_rounds    = 100
 *   eps_int       = 1e-6   integer candidates: ceil(c - eps_int) for lower,
 *                          floor(c + eps_int) for upper bounds
 *   tau_rel       = 1e-6   a continuous candidate c is applied to a lower
 *                          bound l iff l == -inf or c > l + tau_rel*max(1,|l|)
 *                          (upper bounds mirrored); integer candidates must
 *                          be strictly better
 *   eps_feas      = 1e-6   Step 2 / crossing tolerance eps_feas*max(1,|v|)
 *   inf_threshold = 1e20   |v| >= inf_threshold means infinite
 */
typedef struct {
  int32_t max_rounds;
  int32_t reserved0;
  double eps_int;
  double tau_rel;
  double eps_feas;
  double inf_threshold;
} dp_params;

/* Fills *out with the defaults above.  Returns DP_OK or DP_ERR_INVALID_ARG
 * if out is NULL. */
int dp_params_default(dp_params *out);

/* Human-readable text for a return code; never NULL, static storage. */
const char *dp_strerror(int code);

/*
 * Creates a context on CUDA device `device` that issues all work on
 * `cuda_stream` (a cudaStream_t; NULL means the context creates and owns a
 * non-blocking stream).  The caller keeps ownership of a stream it passes
 * and must keep it alive until dp_destroy.
 * Returns DP_OK, DP_ERR_INVALID_ARG, DP_ERR_CUDA or DP_ERR_OOM.
 */
int dp_create(dp_ctx **out, int device, void *cuda_stream);

/* Destroys a context (and its stream, if the context created it).  Every
 * matrix loaded through it must have been freed first.  NULL is a no-op. */
void dp_destroy(dp_ctx *ctx);

/*
 * Copies a CSR matrix (Sec. 3: row_ptr / col_idx / val) to the GPU and
 * builds the device layout (the one-time preprocessing that Sec. 4.3
 * excludes from timing: rows cut into chunks, chunks sorted by length and
 * stored as 32-wide slices).  All three arrays are HOST pointers:
 *   row_ptr[m+1]  int64, row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz
 *   col_idx[nnz]  int32 in [0, n)
 *   val[nnz]      finite, nonzero binary64 coefficients
 * Limits: 0 <= m, n < 2^31; 0 <= nnz < 2^31.
 * `chunk` is the longest row piece one thread reduces (0 = default 256;
 * otherwise 8..4096).  Longer rows are split across threads and combined in
 * a second pass.
 * On success *out owns device memory until dp_matrix_free.
 * Returns DP_OK, DP_ERR_INVALID_ARG, DP_ERR_BAD_CSR, DP_ERR_OOM, DP_ERR_CUDA.
 */
int dp_matrix_load(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz,
                   const int64_t *row_ptr, const int32_t *col_idx,
                   const double *val, int32_t chunk, dp_matrix **out);

/*
 * dp_matrix_load with the row sides known at load time (HOST lhs[m],
 * rhs[m]; not kept).  They only order rows of equal length by which sides
 * are finite (|side| < 1e20), so that the 32 rows of a warp tend to share
 * a side pattern and a warp whose rows all have an infinite side skips that
 * side's activity (its binary64 work halves for one-sided rows).  Any
 * dp_propagate call on the matrix stays valid with any sides: the kernels
 * test the actual sides.  The paper has no counterpart (its rows are
 * grouped by length only, Sec. 3.2).
 */
int dp_matrix_load_sides(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz,
                         const int64_t *row_ptr, const int32_t *col_idx,
                         const double *val, int32_t chunk, const double *lhs,
                         const double *rhs, dp_matrix **out);

/*
 * dp_matrix_load_sides with the merge-path layout instead of row chunks:
 * rows (grouped by the finiteness of their sides when lhs/rhs are given,
 * else in CSR order) stay in CSR, and the merged sequence of the m row
 * ends and nnz nonzeros is cut into segments of `items_per_thread` items
 * (4..4096), one per thread of the activity pass, so that every thread
 * does the same work whatever the row lengths.  A row that lies within one
 * segment is summed in CSR order (results bit-identical to the oracle's);
 * a row that crosses segment boundaries is summed in pieces, combined in a
 * fixed order by a second pass (results within the documented tolerance).
 * This is the merge-based SpMV balancing that the paper's Conclusions and
 * Outlook name as a direction beyond CSR-adaptive (Sec. 3.2).  Only
 * dp_propagate and dp_propagate_hostloop accept such a matrix (the other
 * entry points return DP_ERR_INVALID_ARG); dp_matrix_set_launch applies to
 * its activity pass.  Limits as dp_matrix_load, and m + nnz must be below
 * 2^30 * items_per_thread.  Returns as dp_matrix_load.
 */
int dp_matrix_load_merge(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz,
                         const int64_t *row_ptr, const int32_t *col_idx,
                         const double *val, int32_t items_per_thread,
                         const double *lhs, const double *rhs, dp_matrix **out);

/*
 * Loads `count` independent problems as one matrix: problem k has m[k]
 * rows, n[k] variables and the CSR arrays row_ptr[k], col_idx[k], val[k]
 * (host, as in dp_matrix_load, columns local to the problem); lhs/rhs
 * (arrays of count host pointers, or both NULL) are the optional side hints
 * of dp_matrix_load_sides.  The result is their block-diagonal union: rows
 * and variables are concatenated in problem order (dp_matrix_set_offsets
 * gives each problem's first row and variable), and it is propagated with
 * dp_propagate_set, which stops and counts rounds per problem -- many
 * matrices of uneven size in one device-side round loop, every problem
 * reaching exactly its own dp_propagate result.  The paper propagates one
 * problem per call; this is the batched-matrices form.
 * Returns DP_OK, DP_ERR_INVALID_ARG, DP_ERR_BAD_CSR, DP_ERR_OOM or
 * DP_ERR_CUDA.
 */
int dp_matrix_load_set(dp_ctx *ctx, int32_t count, const int32_t *m,
                       const int32_t *n, const int64_t *const *row_ptr,
                       const int32_t *const *col_idx, const double *const *val,
                       int32_t chunk, const double *const *lhs,
                       const double *const *rhs, dp_matrix **out);

/* Problems of a set: *count, and (if not NULL) row_off[count+1] and
 * var_off[count+1], the first row and variable of each problem in the
 * union (the last entries are the totals).  For a plain matrix *count = 0. */
int dp_matrix_set_offsets(const dp_matrix *set, int32_t *count,
                          int32_t *row_off, int32_t *var_off);

/* Warps per block of the round kernels (4 or 8; the default is 8): a launch
 * shape the autotuner chooses.  Waits for the matrix's pending work. */
int dp_matrix_set_launch(dp_matrix *mat, int32_t round_warps);

/* Lossless value compression: when every coefficient of a loaded matrix is
 * an integer in [-127, 127] the library also keeps the values as int8, and
 * with on = 1 the single-instance round kernels read those (1 byte per
 * value instead of 8; the binary64 value is rebuilt exactly on the integer
 * pipe); on = 0 (the default) reads the binary64 values.  *active (may be
 * NULL) tells whether the kernels now read the int8 copy.  Results are
 * identical either way.  On GB300 the round kernel is bound by gathers and
 * instruction issue rather than by the value stream, and the conversion
 * made it slower, hence off by default.  Waits for the matrix's pending
 * work. */
int dp_matrix_set_compression(dp_matrix *mat, int32_t on, int32_t *active);

typedef struct {
  int32_t chunk;        /* row split length (dp_matrix_load's `chunk`) */
  int32_t round_warps;  /* warps per block (dp_matrix_set_launch) */
  float us_per_round;   /* measured device time of one round, microseconds */
  int32_t reserved;
} dp_tune_entry;

/*
 * Autotuner: times `rounds` rounds (from the given bounds; rounds <= 0: the
 * whole propagation, to the fixed point or params' cap) of the problem
 * for every row split length in {64, 128, 256, 512, 1024} that gives a
 * distinct layout (the long-row threshold of the paper's row bins,
 * Sec. 3.2: longer rows are split and combined in a second pass) and every
 * block shape {4, 8} warps, with CUDA events on each round kernel (the
 * host-driven loop; the best of three timed calls; value compression off).
 * Arguments as
 * dp_matrix_load_sides plus the problem of
 * dp_propagate; lhs/rhs order the rows when they are host arrays.
 * entries[max_entries] (may be NULL if 0) receive the measurements, *count
 * their number, *best the fastest.  Loads and frees one matrix per
 * distinct layout, so it costs several layout builds: run it once per
 * matrix family and load with the best chunk and launch shape.
 */
int dp_autotune(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz,
                const int64_t *row_ptr, const int32_t *col_idx,
                const double *val, const double *lb, const double *ub,
                const uint8_t *vartype, const double *lhs, const double *rhs,
                const dp_params *params, int32_t rounds,
                dp_tune_entry *entries, int32_t max_entries, int32_t *count,
                dp_tune_entry *best);

/*
 * Autotuner of the batched-node path (dp_propagate_nodes): times the whole
 * batched propagation of `nodes` node bound vectors (lb/ub [nodes*n],
 * node-major, host or device, as in dp_propagate_nodes; nodes >= 1) for
 * every row split length in {32, 64, 128, 256, 512} that gives a distinct
 * layout, with the host-driven loop's CUDA-event stage times (the best of
 * three timed calls).  In the batched kernels a warp walks a chunk for 32
 * node lanes, so the split length bounds the serial chain of each work item:
 * short pieces suit batches with few live nodes (a server's lanes), long
 * ones batches of many nodes.  entries[].round_warps is 0 (the batched
 * kernels have one launch shape); us_per_round is the batch's kernel time
 * divided by its rounds.  Other arguments and results as dp_autotune.
 */
int dp_autotune_nodes(dp_ctx *ctx, int32_t m, int32_t n, int64_t nnz,
                      const int64_t *row_ptr, const int32_t *col_idx,
                      const double *val, int32_t nodes, const double *lb,
                      const double *ub, const uint8_t *vartype, const double *lhs,
                      const double *rhs, const dp_params *params,
                      dp_tune_entry *entries, int32_t max_entries, int32_t *count,
                      dp_tune_entry *best);

/* Frees a matrix; NULL is a no-op. */
void dp_matrix_free(dp_matrix *mat);

/* Shape of a loaded matrix (any pointer may be NULL). */
int dp_matrix_info(const dp_matrix *mat, int32_t *m, int32_t *n,
                   int64_t *nnz, int64_t *padded_slots, int32_t *split_rows);

/*
 * Measurement, not propagation (the paper's roofline analysis, Sec. 4.4,
 * asks what bounds a round; this measures it on the loaded matrix): times
 * `reps` launches (after one warm-up) of a kernel that makes the memory
 * accesses of one round's activity pass on this matrix's layout and launch
 * shape -- every value and column streamed, every nonzero's 32-byte
 * variable record gathered -- and does none of its arithmetic.  *us gets the
 * fastest launch in microseconds: the floor that the round's memory traffic
 * sets.  The records need not hold bounds (their contents are not used).
 * Synchronises the context's stream.  Sliced layout only.  Returns DP_OK,
 * DP_ERR_INVALID_ARG or DP_ERR_CUDA.
 */
int dp_matrix_access_floor(dp_ctx *ctx, const dp_matrix *mat, int32_t reps, float *us);

/*
 * Propagates one problem over a loaded matrix (Alg. 2, round-synchronous).
 * Inputs (host or device, all binary64 unless noted; not modified):
 *   lb[n], ub[n]      variable bounds
 *   vartype[n]        uint8: 0 = continuous, nonzero = integer
 *   lhs[m], rhs[m]    row sides
 *   params            NULL = dp_params_default()
 * Outputs (host or device, caller-allocated, written on success and on
 * infeasibility; never aliased with inputs):
 *   lb_out[n], ub_out[n]  bounds after the last executed round
 *   infeasible            HOST int32: 1 if Step 2 or crossing bounds
 *                         detected infeasibility (the run stops after the
 *                         detecting round), else 0
 *   rounds                HOST int32: executed rounds, counting the final
 *                         round that found no change
 * Integer variables' input bounds are rounded (ceil(lb-eps_int),
 * floor(ub+eps_int)) before round 1.
 * Blocks until results are available (the stream is synchronised once, at
 * the end).  Returns DP_OK (converged, or infeasible), DP_CAP_HIT (the last
 * round still changed a bound when max_rounds rounds had run), or an error.
 */
int dp_propagate(dp_ctx *ctx, const dp_matrix *mat, const double *lb,
                 const double *ub, const uint8_t *vartype, const double *lhs,
                 const double *rhs, const dp_params *params, double *lb_out,
                 double *ub_out, int32_t *infeasible, int32_t *rounds);

/*
 * dp_propagate with the whole round loop in one persistent kernel: a
 * cooperative launch (all blocks resident) whose blocks separate the round's
 * phases by grid barriers and read the loop condition after the last one --
 * the device-driven loop of Sec. 3.7 without any per-round launch.  Same
 * arguments, results and status as dp_propagate (single problems only;
 * DP_ERR_INVALID_ARG for a problem set).  Its barrier waits are bounded:
 * DP_ERR_TIMEOUT would report a barrier that did not complete (it cannot
 * happen when the launch succeeds).
 */
int dp_propagate_persistent(dp_ctx *ctx, const dp_matrix *mat,
                            const double *lb, const double *ub,
                            const uint8_t *vartype, const double *lhs,
                            const double *rhs, const dp_params *params,
                            double *lb_out, double *ub_out,
                            int32_t *infeasible, int32_t *rounds);

/*
 * Propagates every problem of a set (dp_matrix_load_set) in one device-side
 * round loop.  lb, ub, vartype (length: total variables) and lhs, rhs
 * (total rows) are the problems' arrays concatenated in problem order
 * (host or device); lb_out/ub_out likewise.  Each problem stops on its own
 * (no change, infeasibility, or the cap) and keeps its bounds from then on:
 * its results equal dp_propagate on that problem alone.  infeasible[count],
 * rounds[count] and status[count] (HOST int32; status may be NULL: 1 = the
 * cap stopped it with a change in its last round) are per problem.
 * Returns DP_OK, DP_CAP_HIT (some problem hit the cap), or an error as
 * dp_propagate (DP_ERR_INVALID_ARG for a matrix that is not a set).
 */
int dp_propagate_set(dp_ctx *ctx, const dp_matrix *set, const double *lb,
                     const double *ub, const uint8_t *vartype,
                     const double *lhs, const double *rhs,
                     const dp_params *params, double *lb_out, double *ub_out,
                     int32_t *infeasible, int32_t *rounds, int32_t *status);

/*
 * dp_propagate_set with the whole round loop in one persistent cooperative
 * kernel (Sec. 3.7, Appendix C): every phase of every round runs in one
 * launch, with a bounded grid barrier between phases (see
 * dp_ctx_set_wait_limit).  Same arguments, results and return values as
 * dp_propagate_set, plus DP_ERR_TIMEOUT if a barrier wait runs out (the
 * context stays usable) and DP_ERR_CUDA if the device cannot launch
 * cooperative kernels; DP_ERR_INVALID_ARG for a set loaded in the merge
 * layout.
 */
int dp_propagate_set_persistent(dp_ctx *ctx, const dp_matrix *set,
                                const double *lb, const double *ub,
                                const uint8_t *vartype, const double *lhs,
                                const double *rhs, const dp_params *params,
                                double *lb_out, double *ub_out,
                                int32_t *infeasible, int32_t *rounds,
                                int32_t *status);

/*
 * The same propagation with the round loop driven from the host: after each
 * round the control block is copied back and the stream synchronised, and
 * the host decides whether to launch the next round (the cpu_loop variant
 * of Sec. 3.7, which the paper uses for its main results).  Results are
 * identical to dp_propagate; it exists to measure the cost of the host
 * round trip and to time the round's kernels one by one.
 * kernel_ms (nullable, 5 floats): total milliseconds, measured with CUDA
 *   events on the context's stream around each launch, of the five round
 *   kernels in this order: activities and screen of every chunk (whole rows
 *   also queue their candidates), combine of split rows, screen of split
 *   rows' chunks, evaluation of the queued candidates, per-variable finish.
 * kernel_launches (nullable, 5 int32): how many times each was launched.
 * Arguments and return values are otherwise those of dp_propagate.
 */
int dp_propagate_hostloop(dp_ctx *ctx, const dp_matrix *mat, const double *lb,
                          const double *ub, const uint8_t *vartype,
                          const double *lhs, const double *rhs,
                          const dp_params *params, double *lb_out,
                          double *ub_out, int32_t *infeasible, int32_t *rounds,
                          float *kernel_ms, int32_t *kernel_launches);

/*
 * Failure detection and test hooks.  The paper has no counterpart; these
 * exist so that the library's bounded waits and its clean-up after a
 * failed allocation can be tested without faulting a GPU.
 *
 * dp_ctx_set_wait_limit: a block of a persistent round loop
 * (dp_propagate_persistent, dp_propagate_nodes_persistent,
 * dp_propagate_set_persistent) waits at a grid barrier for at most `sleeps`
 * sleeps of about 64 ns before it records DP_ERR_TIMEOUT and every block
 * leaves the kernel; the call then returns DP_ERR_TIMEOUT and the context
 * stays usable.  0 restores the default (2^25 sleeps, about 2 s).  Under a
 * cooperative launch every block is resident, so the default is never
 * reached unless something is wrong; a test sets a few sleeps to make the
 * wait run out.  Returns DP_OK or DP_ERR_INVALID_ARG (ctx NULL, sleeps < 0).
 *
 * dp_debug_fail_alloc: the k-th device allocation the library makes from
 * now on (k >= 1, process-wide, counted over every context) fails as if the
 * device were out of memory, so that the caller sees DP_ERR_OOM; k = 0
 * disarms.  Returns DP_OK or DP_ERR_INVALID_ARG (k < 0).
 *
 * dp_debug_live_allocs: the number of device allocations the library holds
 * at this moment (process-wide), to check that a failed call leaked none.
 */
int dp_ctx_set_wait_limit(dp_ctx *ctx, int64_t sleeps);
int dp_debug_fail_alloc(int32_t k);
int64_t dp_debug_live_allocs(void);

/*
 * Allocation-free propagation.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory -- a solver
 * whose device memory belongs to a pool allocator (a framework's caching
 * allocator, the solver's own arena) that a stray cudaMalloc would fragment
 * or exhaust, or a latency-critical pipeline in which cudaMalloc/cudaFree
 * would synchronise the device.  It calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 * It propagates one problem given entirely in DEVICE memory of `device`:
 * the CSR matrix (row_ptr[m+1] int64, col_idx[nnz] int32, val[nnz] binary64,
 * same rules as dp_matrix_load), lb, ub, vartype, lhs, rhs, and the outputs
 * lb_out, ub_out (which also hold the round state).  infeasible and rounds
 * are HOST pointers; params as for dp_propagate (NULL = defaults).  Work is
 * issued on `cuda_stream` (NULL = the legacy default stream); the host waits
 * for the stream after every round (one thread per row, no screen), so this
 * path is for callers that cannot allocate, not the fast path.
 *
 * Its only scratch -- the next-state bound keys and a control block -- is a
 * file-scope device array sized for n <= DP_NOALLOC_MAX_VARS variables
 * (16 MiB plus 256 bytes), which every GPU that loads the library holds
 * until the process exits.  Larger n is rejected with DP_ERR_INVALID_ARG, as
 * are host pointers where device pointers are required.  A malformed matrix
 * returns DP_ERR_BAD_CSR and bad bounds or sides DP_ERR_NAN_INPUT; nothing
 * is read out of range.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array and each call
 * re-initialises what it uses; calls whose GPU work can overlap (several
 * streams or host threads) race on it and must be serialised by the caller.
 * Results equal dp_propagate's.  Returns DP_OK, DP_CAP_HIT or an error.
 */
#define DP_NOALLOC_MAX_VARS (1 << 20)
int dp_propagate_noalloc(int device, void *cuda_stream, int32_t m, int32_t n,
                         int64_t nnz, const int64_t *row_ptr,
                         const int32_t *col_idx, const double *val,
                         const double *lb, const double *ub,
                         const uint8_t *vartype, const double *lhs,
                         const double *rhs, const dp_params *params,
                         double *lb_out, double *ub_out, int32_t *infeasible,
                         int32_t *rounds);

/*
 * Propagates `count` branch-and-bound nodes over one loaded matrix: each
 * node is its own bound vector, and each is propagated exactly as
 * dp_propagate would propagate it alone (same rounds, same results), with
 * all nodes of a launch sharing the device-side round loop.  The paper
 * (Sec. 5) points at propagation after branching -- many nodes, each a few
 * bound changes away from a propagated state -- as the solver use that
 * needs new parent methods on a GPU; its constraint marking (Alg. 1,
 * Sec. 2.1) is applied per node: after round 1 a row is processed for a
 * node only when one of its variables changed for that node.
 * Inputs (host or device; not modified):
 *   lb[count*n], ub[count*n]  binary64 bounds, node-major: node k's vector
 *                             is lb[k*n .. k*n+n-1]
 *   vartype[n], lhs[m], rhs[m], params   shared by all nodes, as in
 *                             dp_propagate
 * Outputs (host or device, caller-allocated, node-major like the inputs):
 *   lb_out[count*n], ub_out[count*n]  bounds after each node's last round
 *   infeasible[count], rounds[count]  HOST int32, per node, as in dp_propagate
 *   status[count]     HOST int32 or NULL: 1 if the node stopped at the round
 *                     cap with its last round still changing a bound
 * Nodes run in launches of up to 1024 (fewer when n is large: entry
 * indices node + j*nodes stay below 2^30); 32 nodes share each warp, so
 * counts that are multiples of 32 use the device best.  The first call
 * allocates a workspace of about 80 bytes per (variable, node) pair kept
 * with the matrix (freed by dp_matrix_free); host inputs are staged.
 * Returns DP_OK, DP_CAP_HIT (some node hit the cap), DP_ERR_INVALID_ARG,
 * DP_ERR_NAN_INPUT (any node), DP_ERR_OOM or DP_ERR_CUDA.
 */
int dp_propagate_nodes(dp_ctx *ctx, const dp_matrix *mat, int32_t count,
                       const double *lb, const double *ub,
                       const uint8_t *vartype, const double *lhs,
                       const double *rhs, const dp_params *params,
                       double *lb_out, double *ub_out, int32_t *infeasible,
                       int32_t *rounds, int32_t *status);

/*
 * dp_propagate_nodes with the round loop driven from the host (one stream
 * synchronisation per round) so that each stage of a round can be timed;
 * same results.  kernel_ms[6] (HOST, may be NULL) receives the summed
 * CUDA-event time of each stage over all rounds and launches, in the order
 * mark, mark_split, act, combine, cand_split, finish; kernel_launches[6]
 * (HOST, may be NULL) how often each ran (stages 1, 3, 4 run only for
 * matrices with split rows).  A measuring aid: the paper has no
 * counterpart.
 */
int dp_propagate_nodes_hostloop(dp_ctx *ctx, const dp_matrix *mat,
                                int32_t count, const double *lb,
                                const double *ub, const uint8_t *vartype,
                                const double *lhs, const double *rhs,
                                const dp_params *params, double *lb_out,
                                double *ub_out, int32_t *infeasible,
                                int32_t *rounds, int32_t *status,
                                float *kernel_ms, int32_t *kernel_launches);

/*
 * dp_propagate_nodes with the whole round loop in one persistent kernel (the
 * single-kernel loop of Sec. 3.7 and Appendix C, for a batch): a
 * cooperative launch of as many blocks as fit on the GPU at once runs every
 * phase of every round, with a bounded grid barrier between phases (see
 * dp_ctx_set_wait_limit) instead of kernel boundaries and no graph.  Same
 * arguments, results and return values as dp_propagate_nodes, plus
 * DP_ERR_TIMEOUT if a barrier wait runs out (the context stays usable) and
 * DP_ERR_CUDA if the device cannot launch cooperative kernels.
 */
int dp_propagate_nodes_persistent(dp_ctx *ctx, const dp_matrix *mat,
                                  int32_t count, const double *lb,
                                  const double *ub, const uint8_t *vartype,
                                  const double *lhs, const double *rhs,
                                  const dp_params *params, double *lb_out,
                                  double *ub_out, int32_t *infeasible,
                                  int32_t *rounds, int32_t *status);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  The paper has no
 * counterpart (it propagates one problem per call); this is how a solver
 * service keeps a GPU busy with many small propagations (Sec. 5: nodes a
 * few bound changes away from a propagated state).
 *
 * A server keeps matrices resident (dp_server_add_matrix) and answers
 * requests (dp_server_submit): one node bound vector of a resident matrix,
 * propagated exactly as dp_propagate would propagate it alone.  Each
 * resident matrix runs a batch of `slots` node slots on its own stream,
 * round by round; between two rounds, finished nodes are read out and
 * their slots are given to waiting requests, which join the running batch
 * (continuous batching).  A matrix's device workspace is allocated when it
 * first has work, within `mem_budget` bytes for all matrices (admission by
 * device memory; idle matrices give theirs back when another needs room).
 * Requests beyond the free slots and memory wait in arrival order.
 * All functions are thread-safe; a worker thread owned by the server does
 * all device work.
 * ---------------------------------------------------------------------- */
typedef struct dp_server dp_server;

typedef struct {
  int32_t slots;        /* node slots per resident matrix: a multiple of 32,
                           32..1024 (0 = 64) */
  int32_t reserved0;
  int64_t mem_budget;   /* device bytes for all matrices' workspaces
                           (<= 0: half of the free device memory at
                           creation) */
  dp_params params;     /* shared by every request (max_rounds >= 1) */
} dp_server_config;

typedef struct {
  uint64_t tag;         /* the tag given to dp_server_submit */
  int32_t status;       /* DP_OK or DP_CAP_HIT */
  int32_t infeasible;   /* as in dp_propagate */
  int32_t rounds;       /* as in dp_propagate */
  int32_t matrix;       /* matrix id */
  double arrival_us;    /* arrival time (dp_server_clock_us scale) */
  double done_us;       /* time the result was written to lb_out/ub_out */
} dp_completion;

typedef struct {
  int64_t submitted, completed, in_system;
  int64_t rounds;            /* batched rounds launched (all matrices) */
  int64_t slot_rounds;       /* sum over rounds of the propagating nodes */
  int64_t admissions;        /* requests placed into slots */
  int64_t max_active_slots;  /* largest number of propagating nodes of a round */
  int64_t workspaces_allocated, evictions;
  int64_t device_bytes;      /* workspace bytes currently held */
} dp_server_stats;

/* Creates a server on ctx's device (cfg NULL: 64 slots, half of the free
 * memory, dp_params_default()).  Returns DP_OK, DP_ERR_INVALID_ARG,
 * DP_ERR_OOM or DP_ERR_CUDA. */
int dp_server_create(dp_ctx *ctx, const dp_server_config *cfg,
                     dp_server **out);

/* Makes a loaded matrix (of the server's context) resident with its
 * variable types and sides (host or device; copied).  The matrix must
 * outlive the server.  *matrix_id receives its id (0, 1, ...). */
int dp_server_add_matrix(dp_server *s, const dp_matrix *mat,
                         const uint8_t *vartype, const double *lhs,
                         const double *rhs, int32_t *matrix_id);

/* Queues one request: lb[n], ub[n] (HOST memory, read when the request is
 * admitted) and lb_out[n], ub_out[n] (HOST memory, written when it
 * completes) must stay valid until its completion is polled.  arrival_us is
 * the request's arrival time on the dp_server_clock_us scale (<= 0: now);
 * latency is measured from it.  The bounds are checked here: NaN, lb >=
 * inf_threshold or ub <= -inf_threshold return DP_ERR_NAN_INPUT and queue
 * nothing. */
int dp_server_submit(dp_server *s, int32_t matrix_id, const double *lb,
                     const double *ub, double *lb_out, double *ub_out,
                     uint64_t tag, double arrival_us);

/* Moves up to max completions into out[] (*count of them), waiting up to
 * wait_us microseconds for the first one when none is ready.  Returns
 * DP_OK, or DP_ERR_CUDA once the worker has seen a device error. */
int dp_server_poll(dp_server *s, dp_completion *out, int32_t max,
                   int32_t *count, int32_t wait_us);

/* Counters since creation. */
int dp_server_stats_get(dp_server *s, dp_server_stats *out);

/* Microseconds on the steady clock the server time-stamps with. */
double dp_server_clock_us(void);

/* Completes every submitted request, stops the worker and frees the
 * server (not the matrices).  Returns DP_OK or the worker's error. */
int dp_server_destroy(dp_server *s);

#ifdef __cplusplus
}
#endif

#endif /* DOMPROP_H */
