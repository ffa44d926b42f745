/*
 * sptrsv.h -- C ABI of the GB300 (sm_103a) sparse triangular solver.
 *
 * Solves the sparse triangular systems of Li, "On Parallel Solution of Sparse
 * Triangular Linear Systems in CUDA" (arXiv:1710.04985), eq. (1):
 *
 *      (L + D) x = f      or      (U + D) x = f,
 *
 * with the matrix in CSR (Sec. 3).  A setup phase (Sec. 4.4) validates the
 * pattern and computes the level of every unknown and the level sets
 * (Sec. 4.1); a solve phase then runs either the level-scheduled solve
 * (Alg. 1, one launch per level) or the self-scheduled solve (Alg. 3, one
 * launch, each row starting as soon as its dependencies are published).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - The matrix is square, n x n, CSR: rowptr int32[n+1], colidx int32[nnz],
 *    vals float64 or float32 [nnz], 0-based, column indices strictly
 *    increasing within a row, every entry in the declared triangle.  Unlike
 *    Sec. 3 (which keeps D apart in a vector d) the diagonal is stored in its
 *    row: the last entry of a lower row, the first entry of an upper row.
 *    With SPTRSV_UNIT the diagonal is taken to be 1 and a stored diagonal
 *    entry, if present, is ignored.
 *  - All array arguments named d_* are DEVICE pointers on the device that
 *    was current when the plan was made.  Sizes are element counts.
 *  - Right-hand sides and solutions are row-major [n][ld] with nrhs <= ld
 *    columns in use (a torch (n, nrhs) tensor has ld = nrhs).  d_x == d_b
 *    (an in-place solve, as in Sec. 3.1 where x starts as f) is allowed.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *    solve is enqueued on it and returns without synchronising.
 *  - Nothing throws across the ABI; every call returns a status.
 *
 * Ownership
 * ---------
 *  The caller owns every array it passes.  The plan BORROWS d_rowptr,
 *  d_colidx and d_vals: they must stay valid, with the same pattern, until
 *  sptrsv_free.  Values may change between solves without re-analysis (the
 *  ILU refactorisation case of Sec. 1); the plan's copies of the values (the
 *  FP32 copy of the refined solve, the level-ordered copy of
 *  SPTRSV_ALGO_SELF_PERMUTED and the part-ordered copy of
 *  SPTRSV_ALGO_SELF_PARTITIONED) are brought up to date by
 *  sptrsv_refresh_values.  The plan OWNS its level arrays, the
 *  transposed pattern, its counters, its status word and its scratch.
 *  Solves on one plan must be serialised (one stream at a time): they share
 *  the plan's counters and scratch.
 *
 * Errors
 * ------
 *  Structural errors are found by sptrsv_analyze, which synchronises its
 *  stream once.  Device-side failures of a solve (a dependency wait that ran
 *  past its limit) are recorded in the plan's status word and returned by
 *  sptrsv_status.
 */
#ifndef SPTRSV_H
#define SPTRSV_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SPTRSV_API __attribute__((visibility("default")))
#else
#define SPTRSV_API
#endif

typedef struct sptrsv_plan_s *sptrsv_plan_t;

typedef enum {
    SPTRSV_OK = 0,
    SPTRSV_ERR_INVALID_ARG = 1,   /* bad size, null pointer, bad enum, ld < nrhs, ...   */
    SPTRSV_ERR_STRUCTURE = 2,     /* unsorted/duplicate column, entry outside triangle,
                                     column out of range, bad rowptr                     */
    SPTRSV_ERR_ZERO_PIVOT = 3,    /* missing or zero diagonal (Sec. 3 assumes none)      */
    SPTRSV_ERR_CUDA = 4,          /* a CUDA runtime call failed                          */
    SPTRSV_ERR_OOM = 5,           /* device allocation failed                            */
    SPTRSV_ERR_TIMEOUT = 6,       /* a dependency wait ran past the spin limit           */
    SPTRSV_ERR_NOT_SUPPORTED = 7, /* e.g. a call that must allocate while capturing      */
    SPTRSV_ERR_INTERNAL = 8       /* a self-check of the setup failed (a library bug);
                                     the plan is not created                             */
} sptrsv_status_t;

typedef enum { SPTRSV_F64 = 0, SPTRSV_F32 = 1 } sptrsv_dtype_t;
typedef enum { SPTRSV_LOWER = 0, SPTRSV_UPPER = 1 } sptrsv_uplo_t;
typedef enum { SPTRSV_NON_UNIT = 0, SPTRSV_UNIT = 1 } sptrsv_diag_t;
typedef enum {
    SPTRSV_ALGO_LEVEL = 0,        /* Alg. 1 (LEVR): one launch per level                 */
    SPTRSV_ALGO_SELF = 1,         /* Alg. 3 (SLFR): one launch, rows self-scheduled in
                                     level order                                         */
    SPTRSV_ALGO_SELF_TILED = 2,   /* Alg. 3 over tiles of consecutive rows: a block owns a
                                     tile and serves in-tile dependencies from shared
                                     memory (Sec. 4.3 remark 2); one right-hand side,
                                     more columns fall back to SPTRSV_ALGO_SELF          */
    SPTRSV_ALGO_SELF_CHAINS = 3   /* Alg. 3 with a warp's ticket = 32/lanes consecutive
                                     rows of the substitution order (segments taken in
                                     the level order of the segment graph); a
                                     dependency inside the segment passes between lanes
                                     without a memory round trip.  The first use per
                                     direction and lanes runs a segment analysis
                                     (allocates, synchronises the stream, refused with
                                     SPTRSV_ERR_NOT_SUPPORTED during graph capture);
                                     one right-hand side, more columns fall back to
                                     SPTRSV_ALGO_SELF                                    */,
    SPTRSV_ALGO_SELF_PERMUTED = 4 /* Alg. 3 on a level-ordered copy of the matrix: row k
                                     of the copy is row jlev[k], columns renumbered to
                                     positions in jlev, values copied (the preordering
                                     of Sec. 4.3 remark 2), so a warp's rows and the
                                     unknowns it waits on are contiguous.  Same
                                     arithmetic in the same order as SPTRSV_ALGO_SELF
                                     (bitwise equal results for equal tuning).  The
                                     first use per direction builds the copy
                                     (allocates ~12 B per entry + 12 B per row in FP64,
                                     synchronises the stream, refused with
                                     SPTRSV_ERR_NOT_SUPPORTED during graph capture).
                                     The copy is a SNAPSHOT of the values (pre-scaled
                                     by 1/d(i) for a non-unit matrix): after changing
                                     d_vals in place call sptrsv_refresh_values
                                     (sptrsv_set_values does it).  More right-hand
                                     sides run the multi-RHS kernel on the same copy,
                                     with a position-ordered [n][nrhs] publication
                                     buffer (allocated on first use of each larger
                                     nrhs)                                               */,
    SPTRSV_ALGO_SELF_COLUMN = 5   /* Alg. 4 (SLFC): column-wise self-scheduled solve.
                                     Unknowns in level order wait on a dependency
                                     counter, then push a(r,i) x(i) into every
                                     dependent x(r) with FP atomic adds and decrement
                                     its counter.  The order of the adds is not fixed:
                                     results agree with the row-wise forms to rounding
                                     but are not bitwise reproducible.  x must not
                                     alias b except in place (x == b).  The first use
                                     per direction builds the counters (and the
                                     transposed pattern, which holds the columns of a
                                     lower/upper matrix): allocates, synchronises the
                                     stream, refused with SPTRSV_ERR_NOT_SUPPORTED
                                     during graph capture.  One right-hand side; more
                                     columns fall back to SPTRSV_ALGO_SELF               */,
    SPTRSV_ALGO_SELF_BLOCKED = 6  /* Alg. 3 on the level-ordered copy (as
                                     SPTRSV_ALGO_SELF_PERMUTED, same first-use build
                                     and value snapshot), a thread block per tile of
                                     tile_rows consecutive level-order positions
                                     (sptrsv_set_tiling; level_order is ignored):
                                     dependencies inside the tile pass through shared
                                     memory, warps take row groups dynamically, the
                                     tile's rows are prefetched into L2.  For narrow
                                     levels.  Bitwise equal to SPTRSV_ALGO_SELF for
                                     equal lanes.  More right-hand sides run as with
                                     SPTRSV_ALGO_SELF_PERMUTED                           */,
    SPTRSV_ALGO_SELF_PARTITIONED = 7  /* the blocked solve of SPTRSV_ALGO_SELF_BLOCKED
                                     on a part-ordered copy: the substitution order is
                                     split where the matrix decouples (every system
                                     boundary of a block-diagonal batch), long blocks
                                     are cut into parts of at most part_rows
                                     consecutive rows (sptrsv_set_partition), short
                                     ones packed together; parts are listed in the
                                     order they are handed out (see
                                     sptrsv_partition_info) and by level (Sec. 4.1)
                                     inside a part, and a thread block takes one part
                                     per tile, so a dependency inside the part passes
                                     through shared memory and only dependencies on
                                     earlier parts wait on published values in L2
                                     (Alg. 3).  On a grid in natural order a part is a
                                     slab of grid lines.  Built on first use (a copy of
                                     the pattern and values, same value snapshot as
                                     SPTRSV_ALGO_SELF_PERMUTED, allocates and
                                     synchronises; not during graph capture) and again
                                     when the part size changes.  Bitwise equal to
                                     SPTRSV_ALGO_SELF for equal lanes.  More right-hand
                                     sides run as with SPTRSV_ALGO_SELF_PERMUTED         */,
    SPTRSV_ALGO_AUTO = 8          /* the plan's default form (sptrsv_set_default_algo;
                                     SPTRSV_ALGO_SELF until one is set), e.g. the one an
                                     autotuner measured fastest                          */
} sptrsv_algo_t;

/* How sptrsv_solve_refined runs the refinement of one right-hand side
 * (several right-hand sides always use the staged form). */
typedef enum {
    SPTRSV_REFINE_STAGED = 0,    /* default: one FP32 solve pass (the plan's default form)
                                    and one FP64 residual pass per refinement step, the
                                    residual norm read by the host after each step      */
    SPTRSV_REFINE_ONE_PASS = 1   /* every step in one self-scheduled sweep over the
                                    level-ordered copy: a row computes its residual and
                                    correction for step m as soon as its dependencies
                                    have published step m (faster on deep, narrow
                                    matrices, slower on wide ones)                       */
} sptrsv_refine_t;

/* Level-analysis methods (sptrsv_reanalyze).  All give the same levels and
 * level sets (levels are unique); they differ in cost. */
typedef enum {
    SPTRSV_ANALYSIS_SWEEP = 0,            /* default: one persistent sync-free sweep
                                             in substitution order, lev(i) = 1 + max
                                             lev(j) computed as a (max,+) solve      */
    SPTRSV_ANALYSIS_KAHN_HOST_LOOP = 1,   /* Kahn's algorithm as in Sec. 4.4.1: one
                                             launch and one device-to-host copy per
                                             level                                  */
    SPTRSV_ANALYSIS_KAHN_PERSISTENT = 2,  /* Kahn's algorithm in one cooperative
                                             launch, levels separated by a bounded
                                             grid-wide barrier                      */
    SPTRSV_ANALYSIS_AUTO = 3              /* what sptrsv_analyze does: the persistent
                                             Kahn launch, which gives up after 256
                                             levels if they hold fewer than 112 rows
                                             on average (a deep, narrow graph; if the
                                             levels are still widening it looks again
                                             at level 1024 and asks for 168), and
                                             then the sweep                         */
} sptrsv_analysis_t;

/* ------------------------------------------------------------------ setup */

/* Largest matrix order and number of stored entries: 2^31 - 256.  A solve
 * kernel's cursor over a row's entries may run up to 128 entries past the
 * row's end and stays a 32-bit int. */
#define SPTRSV_MAX_SIZE 2147483392

/* Setup phase (Sec. 4.4, Table 1): validates the CSR (Sec. 3), builds the
 * CSR of the transpose (pattern and value map, Table 1's TRANS_GPU), computes
 * the 0-based level of every row, lev(i) = 1 + max lev(j) over the
 * off-diagonal entries j of row i (Sec. 4.1; roots get 0) with
 * SPTRSV_ANALYSIS_AUTO, and the level sets (nlev, ilev[nlev+1], jlev[n])
 * with rows in ascending index order inside a level.  An upper triangle is
 * swept in reverse (Sec. 4.1).
 *   n, nnz        matrix order and stored entries, 0 <= n, nnz <= SPTRSV_MAX_SIZE
 *                 (SPTRSV_ERR_INVALID_ARG beyond)
 *   d_rowptr ...  device CSR, borrowed until sptrsv_free (see above)
 *   dtype         element type of d_vals
 *   uplo, diag    triangle and diagonal kind
 *   stream        the setup runs on it and synchronises it once
 *   plan          out: the new plan, or NULL on error
 * Returns SPTRSV_ERR_STRUCTURE / SPTRSV_ERR_ZERO_PIVOT for an invalid matrix;
 * sptrsv_last_error_row() then gives the first offending row. */
SPTRSV_API sptrsv_status_t sptrsv_analyze(int n, int nnz, const int *d_rowptr,
                               const int *d_colidx, const void *d_vals,
                               sptrsv_dtype_t dtype, sptrsv_uplo_t uplo,
                               sptrsv_diag_t diag, void *stream,
                               sptrsv_plan_t *plan);

/* Recomputes the levels and level sets of the forward (transpose = 0) or
 * transposed (transpose = 1) system with `method` (Sec. 4.4: the setup
 * phase; Sec. 4.4.1: Kahn's algorithm on the GPU), replacing the plan's.  The
 * result is identical for every method; the wall time of this call, from
 * after a first synchronisation of `stream` to the end, including a
 * transposed pattern it had to build (Table 1's TRANS_GPU, which Kahn's
 * algorithm needs for the forward system), is what sptrsv_analysis_ms then
 * returns.  Allocates and synchronises; refused with
 * SPTRSV_ERR_NOT_SUPPORTED during graph capture. */
SPTRSV_API sptrsv_status_t sptrsv_reanalyze(sptrsv_plan_t plan, int transpose,
                                            sptrsv_analysis_t method, void *stream);

/* The analysis method that produced the forward (transpose = 0) or
 * transposed (transpose = 1) levels: SWEEP, KAHN_HOST_LOOP or
 * KAHN_PERSISTENT (AUTO resolves to one of them). */
SPTRSV_API sptrsv_status_t sptrsv_analysis_method(sptrsv_plan_t plan, int transpose,
                                                  int *method);

/* Releases everything the plan owns (synchronises the device first). */
SPTRSV_API sptrsv_status_t sptrsv_free(sptrsv_plan_t plan);

/* ------------------------------------------------------------------ solve */

/* Solves op(A) x = b with op = identity: forward substitution for a lower
 * plan, backward for an upper one (Sec. 3.1), by Alg. 1 (SPTRSV_ALGO_LEVEL)
 * or Alg. 3 (SPTRSV_ALGO_SELF and its other forms).  The level-ordered,
 * blocked and partitioned forms solve from the plan's SNAPSHOT of the values
 * (a copy made on first use): after changing d_vals in place call
 * sptrsv_refresh_values before solving again; the other forms read d_vals
 * at every solve.
 *   d_b, d_x  device [n][ld], element type of the plan, nrhs >= 1 columns
 *   ld        leading dimension of both, ld >= nrhs
 * With the self-scheduled algorithms, x is overwritten with a "not yet solved" marker
 * before the solve kernel runs, so x must not alias anything else the solve
 * reads except b itself (x == b is handled with plan scratch).
 * Asynchronous; device-side failures go to sptrsv_status.  Graph capturable
 * (an in-place SELF solve allocates its scratch on first use: make that
 * first call outside capture). */
SPTRSV_API sptrsv_status_t sptrsv_solve(sptrsv_plan_t plan, const void *d_b, void *d_x,
                             int nrhs, int ld, sptrsv_algo_t algo,
                             void *stream);

/* Solves A^T y = g (the adjoint solve used by the backward pass).  Sec. 3.2
 * reads a CSR matrix as the CSC of its transpose; the plan builds the CSR of
 * A^T (pattern plus a map into d_vals, so values are never copied) and its
 * levels, swept in the opposite direction (Sec. 4.1), on first use.  That
 * first call synchronises `stream` and allocates: make it outside capture.
 * Arguments as for sptrsv_solve. */
SPTRSV_API sptrsv_status_t sptrsv_solve_transpose(sptrsv_plan_t plan, const void *d_b,
                                       void *d_x, int nrhs, int ld,
                                       sptrsv_algo_t algo, void *stream);

/* Builds the transposed pattern (the CSC view of Sec. 3.2) and its levels
 * (Sec. 4.1, swept in the opposite direction) now, as the first
 * sptrsv_solve_transpose would; synchronises `stream`. */
SPTRSV_API sptrsv_status_t sptrsv_prepare_transpose(sptrsv_plan_t plan, void *stream);

/* Builds now whatever the first solve of `algo` (SPTRSV_ALGO_AUTO: the
 * plan's default form) in the forward (transpose = 0) or transposed
 * (transpose = 1) direction would build on first use: the transposed pattern
 * and its levels, the level- or part-ordered copy, the segment order of the
 * chained form or the counters of the column-wise form.  Allocates and
 * synchronises `stream` (refused with SPTRSV_ERR_NOT_SUPPORTED during
 * capture), so that later solves can be captured in a CUDA graph, and so
 * that this part of the setup (Sec. 4.4) can be timed on its own. */
SPTRSV_API sptrsv_status_t sptrsv_prepare(sptrsv_plan_t plan, int transpose,
                                          sptrsv_algo_t algo, void *stream);

/* ------------------------------------------------------- differentiation */

/* Gradient of a loss through x = A^{-1} b with respect to the stored values:
 * from eq. (1), dx = -A^{-1} (dA) x, so for every stored (i, j)
 *     d_gvals[p] = - sum_c d_y[i][c] * d_x[j][c]
 * where y = A^{-T} (dloss/dx) comes from sptrsv_solve_transpose.  Entries on
 * the diagonal of a SPTRSV_UNIT plan get 0.  d_y, d_x: [n][ld] device arrays
 * of the plan's type; d_gvals: [nnz] device array of the plan's type, on the
 * plan's pattern.  Asynchronous. */
SPTRSV_API sptrsv_status_t sptrsv_grad_vals(sptrsv_plan_t plan, const void *d_y,
                                 const void *d_x, int nrhs, int ld,
                                 void *d_gvals, void *stream);

/* --------------------------------------------------------------- precision */

/* FP64 residual r = b - A x of system (1), eq. (1) (diagonal taken as 1 for
 * a unit plan).  F64 plans only.  All three arrays [n][ld], device.  Asynchronous. */
SPTRSV_API sptrsv_status_t sptrsv_residual(sptrsv_plan_t plan, const double *d_b,
                                const double *d_x, double *d_r, int nrhs,
                                int ld, void *stream);

/* Mixed-precision solve with iterative refinement (F64 plans only; the
 * motivation is the refinement use of Sec. 1).  The bulk triangular solves
 * run in FP32 (an FP32 copy of the values, FP32 vectors and accumulation);
 * the residual r = b - A x, the correction update x += d and the solution
 * are FP64.  Two forms (sptrsv_set_refine_mode):
 *  - staged: FP32 solves of the plan's default form (sptrsv_set_default_algo)
 *    in that form's launch shape; the in-place, level-ordered, blocked and
 *    partitioned forms add every correction into x as they publish it (no
 *    separate update pass); each residual pass also writes the FP32
 *    right-hand side of the next correction;
 *  - one pass (one right-hand side): every step in one self-scheduled sweep
 *    over the level-ordered copy, in the level-ordered form's launch shape;
 *    a first pass applies three corrections (the residual it measures last
 *    is that of its next-to-last iterate), later passes start from the
 *    current x.
 * Stops when max|r| / (max|b| + ||A||_inf max|x|) <= tol or after max_iter
 * corrections.
 *   d_b, d_x     device FP64 [n][ld]; x is overwritten (no initial guess)
 *   iters        out (nullable): corrections applied after the first solve
 *                (at least one when max_iter >= 1 in the staged form:
 *                an FP32 solve alone does not meet an FP64 stop rule,
 *                so the first correction is taken without reading the norm)
 *   rel_resid    out (nullable): the last relative residual measured
 * Synchronises `stream` once per iteration to read the residual norm; the
 * first call allocates the FP32 copy of the values, FP32 copies of the
 * level- or part-ordered copy its form uses, and scratch.  Not graph
 * capturable.  Refresh the FP32 copies after changing the values with
 * sptrsv_refresh_values. */
SPTRSV_API sptrsv_status_t sptrsv_solve_refined(sptrsv_plan_t plan, const double *d_b,
                                     double *d_x, int nrhs, int ld,
                                     int max_iter, double tol, int *iters,
                                     double *rel_resid, void *stream);

/* The refinement form of sptrsv_solve_refined for one right-hand side
 * (SPTRSV_REFINE_STAGED by default); the getter returns it as an int. */
SPTRSV_API sptrsv_status_t sptrsv_set_refine_mode(sptrsv_plan_t plan, sptrsv_refine_t mode);
SPTRSV_API sptrsv_status_t sptrsv_get_refine_mode(sptrsv_plan_t plan, int *mode);

/* The form SPTRSV_ALGO_AUTO and the FP32 solves of sptrsv_solve_refined
 * run (any algorithm but SPTRSV_ALGO_AUTO; SPTRSV_ALGO_SELF by default).
 * The getter returns it as an int. */
SPTRSV_API sptrsv_status_t sptrsv_set_default_algo(sptrsv_plan_t plan, sptrsv_algo_t algo);
SPTRSV_API sptrsv_status_t sptrsv_get_default_algo(sptrsv_plan_t plan, int *algo);

/* Points the plan at a new values array with the same pattern and element
 * type (for example a new parameter tensor); borrowed like the first one.
 * The plan's copies of the values (FP32, level-ordered), if any, are
 * refreshed on `stream`.  The diagonal is not
 * re-checked: it must stay nonzero.  Asynchronous. */
SPTRSV_API sptrsv_status_t sptrsv_set_values(sptrsv_plan_t plan, const void *d_vals,
                                             void *stream);

/* Re-reads d_vals into every copy of the values the plan holds: the FP32
 * copy of sptrsv_solve_refined, the level-ordered copy of
 * SPTRSV_ALGO_SELF_PERMUTED / _BLOCKED (and of their multi-RHS solves), the
 * part-ordered copy of SPTRSV_ALGO_SELF_PARTITIONED, and the FP32 versions of
 * both copies that refined solves use.  Solves of those forms read the copies,
 * not d_vals: after changing d_vals in place, call this (on the solves'
 * stream, or synchronise) before the next solve.  Async. */
SPTRSV_API sptrsv_status_t sptrsv_refresh_values(sptrsv_plan_t plan, void *stream);

/* ----------------------------------------------------------------- tuning */

/* Launch shape of the solve kernels.  lanes_per_row in {1,2,4,8,16,32}: a
 * row is reduced by a sub-warp of that many lanes, so one warp holds
 * 32 / lanes_per_row rows; block_size a multiple of 32 in [32, 1024];
 * max_blocks caps the persistent grid of the self-scheduled solve (0 = as
 * many as fit on the device at once; the default is 2 blocks per SM, which
 * keeps enough rows waiting ahead of the dependency frontier without
 * flooding L2 with polls).  Applies to the forward and the transposed
 * solves.  Sets the shape of every algorithm (clearing the shapes set for
 * single algorithms by sptrsv_set_algo_tuning).  Multi-RHS solves have their
 * own launch shape (sptrsv_set_mrhs_tuning), by default this block size and
 * grid cap. */
SPTRSV_API sptrsv_status_t sptrsv_set_tuning(sptrsv_plan_t plan, int lanes_per_row,
                                  int block_size, int max_blocks);
/* Launch shape of one algorithm's single-RHS solves, overriding the plan's
 * shape for it (same ranges as sptrsv_set_tuning; lanes_per_row 0 clears it,
 * so the algorithm uses the plan's shape again).  Lets an autotuner keep the
 * best shape of every form it measured: solves that always run one form
 * (the FP32 solves inside sptrsv_solve_refined run SPTRSV_ALGO_SELF) keep
 * that form's shape whichever form won overall. */
SPTRSV_API sptrsv_status_t sptrsv_set_algo_tuning(sptrsv_plan_t plan, sptrsv_algo_t algo,
                                                  int lanes_per_row, int block_size,
                                                  int max_blocks);
SPTRSV_API sptrsv_status_t sptrsv_get_tuning(sptrsv_plan_t plan, int *lanes_per_row,
                                  int *block_size, int *max_blocks);

/* Launch shape of multi-RHS solves (nrhs > 1, Sec. 1's many right-hand
 * sides), kept apart from the single-RHS one: a group of lanes_per_row lanes
 * in {4, 8, 16, 32} owns a row, lane l handling columns l, l + lanes_per_row,
 * ...; every column is folded in the same order (farthest dependency
 * first), so the width does not change the results.  lanes_per_row 0 (the default) picks one lane per column up to 16
 * lanes; block_size 0 and max_blocks -1 (the defaults) use the single-RHS
 * values of sptrsv_set_tuning. */
SPTRSV_API sptrsv_status_t sptrsv_set_mrhs_tuning(sptrsv_plan_t plan, int lanes_per_row,
                                                  int block_size, int max_blocks);

/* Tiles of SPTRSV_ALGO_SELF_TILED: tile_rows consecutive positions of the
 * substitution order (level_order = 0: natural row order, reversed for an
 * upper plan; suits banded and chain-like matrices) or of the level order
 * jlev (level_order = 1: a tile spans many consecutive narrow levels).
 * 32 <= tile_rows, tile_rows * element size <= 48 KB - 256 B (6112 rows in
 * FP64, 12224 in FP32).  Default 2048 rows, substitution order. */
SPTRSV_API sptrsv_status_t sptrsv_set_tiling(sptrsv_plan_t plan, int tile_rows,
                                             int level_order);

/* Parts of SPTRSV_ALGO_SELF_PARTITIONED.  part_rows: rows per part (0:
 * automatic, the rows divided evenly over the GPU's SMs).  A part's unknowns
 * must fit one thread block's shared memory: larger values are reduced to the
 * largest part that fits (29,024 rows in FP64 and 58,048 in FP32 with 227 KB
 * per block).  cluster_blocks in {0, 1, 2, 4, 8}: with 2 or more, thread-block
 * clusters of that many blocks take consecutive parts together and read the
 * values of the cluster's earlier parts from those blocks' shared memory
 * (distributed shared memory) instead of waiting on L2; 0 and 1 use no
 * clusters (the default).  The part-ordered copy is rebuilt on the next
 * partitioned solve when part_rows changes.  Other values are
 * SPTRSV_ERR_INVALID_ARG. */
SPTRSV_API sptrsv_status_t sptrsv_set_partition(sptrsv_plan_t plan, int part_rows,
                                                int cluster_blocks);

/* The part size the next partitioned solve uses (after the automatic choice
 * and the shared-memory limit) and its cluster size (1: no clusters). */
SPTRSV_API sptrsv_status_t sptrsv_get_partition(sptrsv_plan_t plan, int *part_rows,
                                                int *cluster_blocks);

/* Layout of the part-ordered copy of the forward (transpose = 0) or
 * transposed (transpose = 1) system, as the last partitioned solve in that
 * direction built it (SPTRSV_ERR_NOT_SUPPORTED before the first).  The
 * substitution order is split where the matrix decouples (no row at or after
 * a position depends on a row before it; a block-diagonal batch decouples at
 * every system boundary) into *nblocks independent blocks; a block longer
 * than half the part size is cut into balanced parts of at most part_rows
 * rows, shorter neighbouring blocks share a part; the *nparts parts are
 * handed out to thread blocks latest start first: by the block's slack (the
 * deepest level of the matrix minus the block's own depth, Sec. 4.1) plus
 * the piece's share of the block's levels (piece index times the block's
 * level count / its number of parts, rounded down), in order of
 * substitution among equals.  *max_part_rows is the
 * longest part.  All outputs nullable; the device arrays are owned by the
 * plan and valid until the copy is rebuilt or the plan freed:
 *   d_part_ptr  int[nparts + 1]: first position of each part, in hand-out
 *               order (position k of the copy holds row d_order[k])
 *   d_order     int[n]: the row at each position of the copy */
SPTRSV_API sptrsv_status_t sptrsv_partition_info(sptrsv_plan_t plan, int transpose,
                                                 int *nparts, int *nblocks,
                                                 int *max_part_rows,
                                                 const int **d_part_ptr,
                                                 const int **d_order);

/* Upper bound on the polling rounds of one dependency wait before the wait
 * gives up, records SPTRSV_ERR_TIMEOUT with its row and goes on with NaN so
 * that every later row still finishes.  Default 2^24 rounds (several
 * seconds); the environment variable SPTRSV_SPIN_LIMIT overrides the
 * default for new plans. */
SPTRSV_API sptrsv_status_t sptrsv_set_spin_limit(sptrsv_plan_t plan, long long polls);

/* -------------------------------------------------------------- inspection */

/* Level data (Sec. 4.1) of the forward (transpose = 0) or transposed
 * (transpose = 1) system: nlev, and device pointers (owned by the plan) to
 * lev[n], ilev[nlev+1] and jlev[n].  The transposed data exist only after
 * sptrsv_prepare_transpose or a transposed solve. */
SPTRSV_API sptrsv_status_t sptrsv_levels(sptrsv_plan_t plan, int transpose, int *nlev,
                              const int **d_lev, const int **d_ilev,
                              const int **d_jlev);

/* Transposed pattern (CSR of A^T, the CSC view of Sec. 3.2): tptr[n+1],
 * tidx[nnz] and tmap[nnz], device pointers owned by the plan, with (A^T)
 * entry q equal to d_vals[tmap[q]]. */
SPTRSV_API sptrsv_status_t sptrsv_transpose_pattern(sptrsv_plan_t plan,
                                         const int **d_tptr,
                                         const int **d_tidx,
                                         const int **d_tmap);

/* Synchronises `stream`, then returns and clears the first device-side
 * failure recorded since the last call (SPTRSV_OK if none); *error_row
 * (nullable) receives its row, or -1. */
SPTRSV_API sptrsv_status_t sptrsv_status(sptrsv_plan_t plan, void *stream,
                              int *error_row);

/* Row of the last STRUCTURE / ZERO_PIVOT error of sptrsv_analyze on this
 * host thread, or -1. */
SPTRSV_API int sptrsv_last_error_row(void);

/* Human-readable name of a status, and the text of the last CUDA error seen
 * on this host thread. */
SPTRSV_API const char *sptrsv_status_string(sptrsv_status_t status);
SPTRSV_API const char *sptrsv_last_cuda_error(void);

/* Wall time of the last sptrsv_analyze or sptrsv_reanalyze of this plan
 * (ms, host clock around the synchronised setup). */
SPTRSV_API sptrsv_status_t sptrsv_analysis_ms(sptrsv_plan_t plan, double *ms);

/* Kernel timing.  While enabled, every solve records a pair of CUDA events
 * around its main kernel work (for the self-scheduled solve: the solve
 * kernel alone; for the level-scheduled solve: the whole per-level launch
 * sequence) on the solve's stream.  sptrsv_profile_read synchronises those
 * events and returns the summed milliseconds and the number of solves timed
 * since the last read, then clears them.  Not for use under graph capture. */
SPTRSV_API sptrsv_status_t sptrsv_profile_enable(sptrsv_plan_t plan, int enable);
SPTRSV_API sptrsv_status_t sptrsv_profile_read(sptrsv_plan_t plan, double *total_ms,
                                    int *count);

/* Kernels enqueued by the last solve call on this plan (for launch
 * accounting). */
SPTRSV_API int sptrsv_last_launch_count(sptrsv_plan_t plan);

/* ------------------------------------------------------------ no allocation */

/* Largest n that sptrsv_solve_noalloc accepts.  Its working memory is one
 * fixed array inside the library: 256 bytes plus 4 bytes per row, i.e.
 * 16 MiB + 256 B per GPU.  With CUDA's lazy module loading (the default
 * since CUDA 12) the array is reserved on a device when the library's code
 * is first used there, often by the first sptrsv_solve_noalloc call, and
 * then held until the process exits.  A caller whose own pool takes all
 * device memory should make one warm-up call per device before the pool
 * claims it (and before any stream capture, see below). */
#define SPTRSV_NOALLOC_MAX_ROWS 4194304

/* Solves A x = b for one right-hand side without a plan and without any
 * device allocation (the paper has no counterpart to this call).  It is for
 * callers that may not call cudaMalloc or cudaFree: code running inside an
 * application that owns all device memory through its own pool, or a
 * latency-critical loop that must not touch the device allocator (which can
 * take global locks and synchronise the device).  Such callers cannot make a
 * plan either, since the analysis allocates its level sets.
 *
 * What it does, all enqueued on `stream`: clears its working memory,
 * validates the CSR as sptrsv_analyze does, then runs the self-scheduled
 * solve of Alg. 3 with rows handed out in substitution order instead of
 * level order (rows wait for per-row ready flags; no level sets).
 *   n, nnz, d_rowptr, d_colidx, d_vals, dtype, uplo, diag: as sptrsv_analyze
 *   d_b, d_x   device vectors of n elements, contiguous; d_x == d_b allowed
 *   error_row  NULL: return right after enqueueing; SPTRSV_OK then only
 *              means "enqueued", and device-side errors are not reported.
 *              Non-NULL: wait for `stream`, then return the device-side
 *              result -- SPTRSV_ERR_STRUCTURE or SPTRSV_ERR_ZERO_PIVOT from
 *              validation (x untouched) or SPTRSV_ERR_TIMEOUT -- with its
 *              row in *error_row (-1 if none).
 * A dependency wait gives up after SPTRSV_SPIN_LIMIT polls (environment
 * variable, read at every call; 2^24 by default), reports
 * SPTRSV_ERR_TIMEOUT for its row and goes on with NaN.
 * Returns SPTRSV_ERR_INVALID_ARG for n > SPTRSV_NOALLOC_MAX_ROWS or
 * nnz > SPTRSV_MAX_SIZE.
 * Working memory: one array declared at file scope in the library, shared by
 * every call; each call clears the parts it uses before reading them, and
 * the array keeps the last call's contents afterwards.  Calls whose GPU work
 * overlaps (other streams, other host threads) race on it: serialise them.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (that device current); make that first call before
 * any stream capture. */
SPTRSV_API sptrsv_status_t sptrsv_solve_noalloc(int n, int nnz, const int *d_rowptr,
                                                const int *d_colidx, const void *d_vals,
                                                sptrsv_dtype_t dtype, sptrsv_uplo_t uplo,
                                                sptrsv_diag_t diag, const void *d_b,
                                                void *d_x, void *stream, int *error_row);

/* Test hook: the self-scheduled solve skips publishing this row (-1 = off),
 * so that every row depending on it exercises the bounded wait and the
 * SPTRSV_ERR_TIMEOUT path.  Faults nothing: the waits end at the limit. */
SPTRSV_API sptrsv_status_t sptrsv_debug_withhold_row(sptrsv_plan_t plan, int row);

#ifdef __cplusplus
}
#endif

#endif /* SPTRSV_H */
