/*
 * sptrsv.h - C ABI of a GB300 (sm_103a) sparse triangular solver that
 * executes forward (and backward) substitution according to a superstep
 * schedule of the factor's dependency DAG: wavefronts, GrowLocal, its
 * block-parallel form or GrowLocal on the Funnel-coarsened DAG; analysis on
 * the host or (wavefronts) on the device; plans saved to and loaded from
 * files; single, batched and served solves.
 *
 * Method: arXiv:2503.05408, "Efficient parallel scheduling for sparse
 * triangular solvers".  Citations below name the paper's sections,
 * equations, definitions and algorithms.
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status: SPTRSV_OK (0) or a negative
 *    SPTRSV_ERR_* code.  No exception crosses the ABI and nothing calls
 *    exit().  sptrsv_status_string() names a code; sptrsv_last_error()
 *    returns a thread-local message describing the last failure.
 *  - Host arrays passed in are owned by the caller and only read during the
 *    call (analyze copies what it needs).
 *  - Device vectors (b, x) are caller-owned device pointers on the plan's
 *    device; they must stay valid until the work enqueued on `stream`
 *    finishes.  Multi-RHS blocks are column-major with leading dimension ld.
 *  - Opaque handles (sptrsv_plan, sptrsv_batch, sptrsv_server) are owned by
 *    the library and released by the matching *_destroy call.
 *  - `stream` is a cudaStream_t passed as an opaque pointer (NULL = the
 *    legacy default stream).
 */
#ifndef SPTRSV_H
#define SPTRSV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef struct CUstream_st *sptrsv_stream;          /* == cudaStream_t */
typedef struct sptrsv_plan sptrsv_plan;

/* ---------------------------------------------------------------- status */
enum {
    SPTRSV_OK = 0,
    SPTRSV_ERR_ARG = -1,             /* null pointer, bad size, bad option          */
    SPTRSV_ERR_NOT_LOWER = -2,       /* an entry above the diagonal / out of range  */
    SPTRSV_ERR_UNSORTED_OR_DUP = -3, /* columns not strictly increasing in a row    */
    SPTRSV_ERR_ZERO_DIAG = -4,       /* diagonal missing, not last, or zero (Sec. 2.2 assumes
                                        a non-singular factor)                      */
    SPTRSV_ERR_OOM = -5,             /* host or device allocation failed            */
    SPTRSV_ERR_BUDGET = -6,          /* request can never fit the serving budget    */
    SPTRSV_ERR_CUDA = -7,            /* a CUDA runtime call failed                  */
    SPTRSV_ERR_LAUNCH = -8,          /* persistent grid cannot be co-resident       */
    SPTRSV_ERR_TIMEOUT = -9,         /* a bounded device wait expired; x is invalid */
    SPTRSV_ERR_NOT_CONVERGED = -10,  /* refinement hit max_iters (x still returned) */
    SPTRSV_ERR_PENDING = -11,        /* serving request not finished yet            */
    SPTRSV_ERR_NO_DEVICE = -12,      /* plan was analysed host-only (device = -1)   */
    SPTRSV_ERR_IO = -13              /* a saved plan could not be written or read   */
};

/* Name of a status code (static string). */
const char *sptrsv_status_string(int status);
/* Message of the last failure on the calling thread ("" if none). */
const char *sptrsv_last_error(void);
/* Library version as major*10000 + minor*100 + patch. */
int sptrsv_version(void);

/* ---------------------------------------------------------------- input */
/* Square lower-triangular factor in CSR, host memory, 0-based, int32 indices.
 * Each row lists its columns strictly increasing with the diagonal last
 * (Sec. 2.2: edge (j,i) of the DAG iff A_ij != 0, so the structural entries
 * define the DAG; the generators never store explicit zeros). */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int32_t *rowptr;   /* n + 1 */
    const int32_t *col;      /* nnz   */
    const double *val;       /* nnz   */
} sptrsv_csr;

/* ------------------------------------------------------------- analysis */
enum {
    SPTRSV_SCHED_LEVELS = 0,     /* wavefront schedule: superstep = wavefront (Sec. 1) */
    SPTRSV_SCHED_GROWLOCAL = 1   /* GrowLocal (Sec. 3, Algorithm 3.1)                  */
};
enum {                           /* value copies kept on the device (bit mask)        */
    SPTRSV_VALUES_F64 = 1,       /* FP64 values: plain FP64 solve                     */
    SPTRSV_VALUES_F32 = 2        /* FP32 hi + FP32 lo split: FP32 sweeps with FP64
                                    residual refinement, and FP32 solves              */
};

typedef struct {
    int32_t mode;      /* SPTRSV_SCHED_*                                                  */
    int32_t k;         /* GrowLocal cores; 0 = number of SMs of `device` (1 if host-only)  */
    double alpha0;     /* first superstep length (20, Sec. 3)                              */
    double growth;     /* alpha growth per attempt (1.5, Sec. 3)                           */
    double L;          /* barrier cost in Eq. 3.1 (500, Sec. 3 footnote)                   */
    double accept;     /* worthy iff beta >= accept * best beta (0.97, App. B)             */
    int32_t values;    /* SPTRSV_VALUES_* mask; 0 = F64 | F32                              */
    int32_t device;    /* CUDA device ordinal, or -1: analyse on the host only (no upload;
                          sptrsv_solve then returns SPTRSV_ERR_NO_DEVICE)                  */
    int32_t triangle;  /* SPTRSV_TRI_*: which system the plan solves (default LOWER)      */
    int32_t sched_blocks;  /* GROWLOCAL only.  0 or 1: one schedule over the whole DAG.
                          B > 1: block-parallel scheduling (Sec. 3.1): rows are cut into B
                          diagonal blocks, block b = rows floor(b n / B) .. floor((b+1) n / B)
                          - 1; GrowLocal runs on each block's sub-DAG (edges from earlier
                          blocks dropped, vertex weight = the full row's entry count) and
                          the block schedules are concatenated: a vertex of block b gets
                          its block superstep plus the supersteps of blocks 0..b-1.  The
                          result does not depend on sched_threads.                        */
    int32_t sched_threads; /* host threads for the schedule blocks (never more than B) and for
                          Funnel's triangle reduction; 0 = one per hardware thread.  The
                          schedule never depends on it.                                    */
    int32_t coarsen;   /* GROWLOCAL only, SPTRSV_COARSEN_*: FUNNEL schedules the DAG coarsened
                          by in-funnels (Sec. 4, Algorithm 4.1) after dropping the long edge of
                          every triangle u->v->w; each row takes its part's superstep and core.
                          Not combined with sched_blocks > 1.                             */
    double coarsen_max_weight;  /* largest part weight (stored entries of its rows) a part may
                          grow to, the size constraint of Sec. 4.2; <= 0: 500 (= L)         */
    int32_t analyze_on_device; /* 1: LEVELS schedule analysed on `device` (any triangle; UPPER and
                          LOWER_TRANSPOSED are reversed on the host first):
                          wavefronts by a polled kernel, the Sec. 5 order by a stable radix
                          sort, the device layout by gathers, from one upload of the CSR;
                          the plan equals the host analysis bit for bit (validation and the
                          one-block ring test stay on the host).  0: host analysis.          */
} sptrsv_analyze_opts;
enum { SPTRSV_COARSEN_NONE = 0, SPTRSV_COARSEN_FUNNEL = 1 };

/* The system a plan solves.  The method covers both substitution directions
 * (Sec. 2, Eq. 2.1 and its backward counterpart): an upper factor's DAG is the
 * lower one reversed, so UPPER and LOWER_TRANSPOSED are analysed as the lower
 * factor L' with rows and columns numbered backwards (row i of the system is
 * row n-1-i of L') and solved by the same kernels; b, x and sptrsv_plan_export
 * stay in the caller's numbering.
 *   LOWER            : L x = b, CSR of L, diagonal last in every row
 *   UPPER            : U x = b, CSR of U, columns increasing, diagonal FIRST
 *   LOWER_TRANSPOSED : L^T x = b from the CSR of L (diagonal last), e.g. the
 *                      second half of an incomplete-Cholesky preconditioner   */
enum { SPTRSV_TRI_LOWER = 0, SPTRSV_TRI_UPPER = 1, SPTRSV_TRI_LOWER_TRANSPOSED = 2 };

/* Fill `o` with the defaults above (LEVELS, k = 0, 20, 1.5, 500, 0.97, both value
 * copies, device 0, LOWER, one schedule block, sched_threads 0, no coarsening, host
 * analysis). */
void sptrsv_analyze_opts_default(sptrsv_analyze_opts *o);

typedef struct {
    int32_t n;
    int64_t nnz;
    int32_t levels;          /* number of wavefronts = longest path in vertices (Sec. 6.2) */
    int32_t supersteps;      /* S of the chosen schedule                                   */
    int32_t k;               /* cores of the schedule (1 for LEVELS)                       */
    int32_t max_level_rows;  /* widest wavefront                                           */
    double avg_wavefront;    /* n / levels (Sec. 6.2)                                      */
    int64_t device_bytes;    /* bytes resident on the device for this plan                 */
    double analyze_ms;       /* host wall time of sptrsv_analyze                           */
    int32_t phases;          /* dependency-free row groups walked by the executors          */
    int32_t ring_rows;       /* shared-memory x ring proven safe for one-block walks (0: none) */
    double schedule_ms;      /* host wall time of the superstep schedule alone (part of
                                analyze_ms): wavefronts for LEVELS, GrowLocal otherwise   */
    int32_t sched_blocks;    /* diagonal blocks the schedule was built on (1: whole DAG)    */
    int32_t coarse_vertices; /* vertices of the DAG GrowLocal scheduled: Funnel parts, else n */
} sptrsv_stats;

/* Analyse a factor (Sec. 2.2 DAG, Sec. 1 wavefronts, Sec. 3 schedule, Sec. 5
 * reordering) and, unless opts->device == -1, upload a superstep-contiguous
 * copy to the device.
 *   csr   : host CSR, validated (errors NOT_LOWER, UNSORTED_OR_DUP, ZERO_DIAG, ARG).
 *   opts  : may be NULL for the defaults.
 *   out   : receives the plan; NULL on error.
 * The call is synchronous; it owns no caller memory afterwards. */
int sptrsv_analyze(const sptrsv_csr *csr, const sptrsv_analyze_opts *opts, sptrsv_plan **out);

/* Statistics of an analysed plan. */
int sptrsv_plan_stats(const sptrsv_plan *plan, sptrsv_stats *out);

/* Copy the schedule to caller host buffers of n int32 each (any may be NULL):
 *   level[v] : wavefront of row v (0-based)
 *   sigma[v] : superstep of row v (0-based; Def. 2.1 sigma minus one)
 *   pi[v]    : core of row v (0-based; Def. 2.1 pi minus one)
 *   perm[r]  : original row at position r of the Sec. 5 reordering
 *              (sorted by superstep, then core, then original id). */
int sptrsv_plan_export(const sptrsv_plan *plan, int32_t *level, int32_t *sigma, int32_t *pi,
                       int32_t *perm);

/* Funnel plans (coarsen = FUNNEL): the part of every row, n int32 in the caller's
 * numbering; parts are numbered 0..coarse_vertices-1.  For inspection and tests
 * (Sec. 4: every part is an in-funnel of the triangle-reduced DAG).  Errors: ARG
 * (NULL, or a plan not coarsened in this process, e.g. loaded from a file). */
int sptrsv_plan_export_parts(const sptrsv_plan *plan, int32_t *part);

/* ------------------------------------------------------- saved plans */
/* Write an analysed plan to `path` so that another process can rebuild it with
 * sptrsv_plan_load without running the scheduler again: the file holds the
 * factor `csr`, the superstep schedule (sigma, pi; Sec. 3) and, once a
 * block-local solve has run, that executor's row partition.  The schedule and
 * the partition depend only on the pattern, so the analysis cost (the paper's
 * amortisation threshold, Table 7.6) is paid once per pattern.
 *   csr  : the factor in the plan's triangle format, host memory; its pattern
 *          must be the analysed one (checked: same wavefronts and the schedule
 *          valid on it, Def. 2.1); its values are saved as given.
 *   path : written through "<path>.tmp" and renamed.
 * Format: little-endian binary, magic "SPTRSVPL", version 1, a checksum over
 * the payload.  Errors: ARG (NULL, other size or pattern), IO (cannot write). */
int sptrsv_plan_save(const sptrsv_plan *plan, const sptrsv_csr *csr, const char *path);

/* Rebuild a saved plan.  opts->device and opts->values apply (NULL = defaults);
 * the schedule, its mode, k and the triangle come from the file.  Nothing read
 * is trusted: the factor is validated as in sptrsv_analyze, the schedule must
 * satisfy Def. 2.1 on it (a wavefront schedule must equal the wavefronts), and
 * a saved partition must list every block's rows in (wavefront, id) order, so a
 * damaged file gives an error and never a plan that could stall a solve.
 * Errors: IO (missing, truncated, wrong size), ARG (not a plan file, other
 * version or byte order, checksum mismatch, invalid schedule or partition),
 * the validation errors of sptrsv_analyze, OOM, CUDA. */
int sptrsv_plan_load(const char *path, const sptrsv_analyze_opts *opts, sptrsv_plan **out);

/* Host-only: the row -> thread block partition the block-local executor
 * (SPTRSV_SYNC_LOCAL) builds for `blocks` thread blocks, for inspection and
 * tests.  Sec. 3's locality goal at SM granularity: in (wavefront, id) order a
 * row joins the block holding most of its parents of the two previous
 * wavefronts (weight 4 for the previous one, 1 for the one before) unless that
 * block took ceil(1.25 * width / blocks) rows of the row's wavefront or holds
 * row_cap rows; else the block with the fewest rows of the wavefront.
 *   A            : the factor (validated as in sptrsv_analyze)
 *   row_cap      : rows one block may hold (0 = unlimited)
 *   block_of_row : out, n entries, the block of each row
 *   position     : out, n entries, the row's position in its block's list;
 *                  every block's list is in (wavefront, id) order
 * Errors: ARG (sizes, NULL outputs, rows exceeding blocks * row_cap), and the
 * validation errors of sptrsv_analyze. */
int sptrsv_local_partition(const sptrsv_csr *A, int32_t blocks, int32_t row_cap, int32_t *block_of_row,
                           int32_t *position);
/* Host-only: the same for any partition kind (SPTRSV_PART_PARENTS, RANGES or GRID;
 * GRID falls back to PARENTS on a factor without nested-stride structure), as the
 * block-local executors build it.  Arguments and errors as sptrsv_local_partition,
 * plus ARG for another kind. */
int sptrsv_block_partition(const sptrsv_csr *A, int32_t kind, int32_t blocks, int32_t row_cap,
                           int32_t *block_of_row, int32_t *position);

/* Release a plan and its device memory (NULL is a no-op).  The caller must
 * ensure no enqueued solve still uses it. */
void sptrsv_destroy(sptrsv_plan *plan);

/* ---------------------------------------------------------------- solve */
enum { SPTRSV_F64 = 0, SPTRSV_F32 = 1 };             /* dtype of b and x */
enum {
    SPTRSV_SYNC_AUTO = 0,   /* autotuned per plan                                          */
    SPTRSV_SYNC_GRID = 1,   /* persistent grid, one grid-wide barrier per superstep         */
    SPTRSV_SYNC_FLAGS = 2,  /* persistent grid, per-row ready flags on cross-CTA parents    */
    SPTRSV_SYNC_CTA = 3,    /* one thread block walks all supersteps (small factors); each
                               phase is staged into shared memory by TMA bulk copies ahead of
                               use when the plan's largest phase fits                       */
    SPTRSV_SYNC_CTA_REGS = 4, /* one thread block, register prefetch only (no staging)      */
    SPTRSV_SYNC_LOCAL = 5,  /* persistent grid, one block per SM (threads up to 1024); rows
                               partitioned over the blocks so that most dependencies, above
                               all each row's last-finishing parent, stay inside one block
                               (Sec. 3's locality principle applied to SMs); a block keeps its
                               rows' values in shared memory and polls them there, other
                               parents in global memory.  One right-hand side per solve
                               (nrhs == 1).  The partition is built on the first solve in this
                               mode (synchronous: device-to-host copy, host pass, upload) and
                               kept in the plan.  ARG if nrhs > 1 or if the rows do not fit the
                               shared memory of the grid's blocks                            */
    SPTRSV_SYNC_CHUNKS = 6, /* the block-local partition of SYNC_LOCAL executed one row per
                               lane: each block's (wavefront, id) list is cut into chunks of
                               up to 32 rows of one wavefront, a warp waits until every
                               parent of its chunk has landed and then runs Eq. 2.1 for all
                               of its rows at once (full-warp FP64 instructions; entries
                               stored sliced, 32 lanes per entry slot).  A row's sum runs in a
                               fixed order (parents of other blocks first, then its own block's,
                               each in column order): the same bits every run.  Each block first
                               writes b_i / A_ii of its rows, in chunk order, into the plan's
                               workspace, so no step waits on a gather of b.  One right-hand
                               side; at most 768 threads per block when no row has more than
                               three off-diagonal entries, else 512 (ARG above); ARG as for
                               SYNC_LOCAL                                                     */
    SPTRSV_SYNC_RESIDENT = 7 /* one thread block with the whole factor in shared memory (small
                               factors): it copies the plan's row pointers, row ids, columns,
                               scaled values and b_i / A_ii once, keeps x there, and walks the
                               phases one row per thread with a block barrier between phases,
                               so no dependency step touches global memory.  One right-hand
                               side, up to 1024 threads; ARG if nrhs > 1 or if the factor needs
                               more than one SM's shared memory (8 (2 n + m) + 4 (m + 2 n +
                               phases + 2) bytes in FP64, m = off-diagonal entries)          */
};
enum {
    SPTRSV_PART_AUTO = 0,    /* the partition the plan holds (saved, built or tuned), else PARENTS */
    SPTRSV_PART_PARENTS = 1, /* rows follow their parents (see sptrsv_local_partition)          */
    SPTRSV_PART_RANGES = 2,  /* contiguous ranges of row ids, n / blocks rows each: the natural
                                order keeps a structured grid's neighbours together, and every
                                dependency goes to the same or a later block                    */
    SPTRSV_PART_GRID = 3     /* a factor whose off-diagonal offsets are dominated by nested
                                strides 1 | s1 | s2 (a 3D grid in natural order, detected from
                                the pattern) is cut into pencils along the fastest stride, tiled
                                over the other two: the blocks' dependency graph is acyclic and a
                                dependency path crosses few blocks.  Other factors: PARENTS     */
};
enum {
    SPTRSV_PREC_F64 = 0,         /* FP64 values and arithmetic (needs SPTRSV_VALUES_F64)    */
    SPTRSV_PREC_F32_REFINE = 1   /* FP32 sweeps + FP64 residual r = b - Lx and FP64 update
                                    x += d, repeated until converged (needs VALUES_F32)     */
};

typedef struct {
    int32_t sync;        /* SPTRSV_SYNC_*                                                    */
    int32_t lanes;       /* lanes per row: 0 = auto, or 1, 2, 4, 8, 16, 32                   */
    int32_t precision;   /* SPTRSV_PREC_* for dtype F64 (dtype F32 always solves in FP32)    */
    int32_t max_iters;   /* refinement: maximum correction sweeps after the first (6, <= 14) */
    double refine_tol;   /* refinement stops when ||d||inf <= refine_tol * ||x||inf or when the
                            FP64 backward error of the iterate is <= refine_tol (1e-13)       */
    int32_t blocks_per_sm; /* persistent grid size per SM; 0 = auto                          */
    int32_t threads;     /* threads per block; 0 = auto                                      */
    double timeout_s;    /* limit of every bounded device wait, seconds (default 2.0)         */
    int32_t rhs_tile;    /* multi-RHS mapping: 0 = auto (lanes follow right-hand sides when
                            nrhs >= 3), 1 = lanes split each row's entries, 4/8/16/32 = a tile of
                            that many right-hand sides per row, each row's columns and values
                            loaded once for the whole tile                                     */
    int32_t eager_sum;   /* SYNC_FLAGS / SYNC_LOCAL with 2..8 lanes splitting a row's entries: SPTRSV_EAGER_*.
                            ON: while a row waits for its last parents its lanes keep the
                            partial sum reduced, so the lane that receives the last parent
                            publishes after one FMA (best when a row's parents finish at
                            different times); OFF: reduce once all parents are in (best when
                            they arrive together, e.g. stencils).  AUTO = tuned value, else ON.
                            Polled sums follow the parents' arrival order: with ON, or with
                            several entries per lane, the last bits of x may differ between
                            runs (always within the solve's accuracy)                          */
    int32_t partition;   /* SYNC_LOCAL / SYNC_CHUNKS: SPTRSV_PART_*, the row -> thread block
                            partition.  A plan keeps one partition; asking for another kind
                            rebuilds it (synchronous host pass)                                 */
} sptrsv_solve_opts;
enum { SPTRSV_EAGER_AUTO = 0, SPTRSV_EAGER_ON = 1, SPTRSV_EAGER_OFF = 2 };

void sptrsv_solve_opts_default(sptrsv_solve_opts *o);

typedef struct {
    int32_t status;        /* SPTRSV_OK, ERR_TIMEOUT or ERR_NOT_CONVERGED                     */
    int32_t sweeps;        /* dependent sweeps run (1 for a plain solve)                      */
    int64_t barriers;      /* grid-wide barriers executed (device counter)                    */
    int64_t flag_waits;    /* cross-CTA ready-flag waits that had to spin (device counter)    */
    double dnorm;          /* refinement: last ||d||inf / ||x||inf (0 for a plain solve)      */
    int32_t sync;          /* sync mode actually used                                         */
    int32_t lanes;         /* lanes per row actually used                                     */
    int32_t grid;          /* thread blocks launched                                          */
    int32_t threads;       /* threads per block                                               */
    double berr;           /* refinement: last normwise backward error max|r| /
                              (||L||inf max|x| + max|b|) computed in FP64 (0 for a plain solve) */
    int64_t cross_edges;   /* SYNC_LOCAL / SYNC_CHUNKS: dependency edges whose parent belongs to
                              another thread block (each one global-memory hop; fixed by the
                              partition); the other modes: -1                                  */
    int64_t edges;         /* dependency edges of the factor (off-diagonal entries)            */
    double latency_s;      /* serving: completion - submission of the request, seconds (for
                              host-buffer requests the copies included); 0 otherwise            */
} sptrsv_report;

/* Solve L X = B for nrhs right-hand sides (Eq. 2.1 in the plan's schedule).
 *   b, x   : device pointers, column-major n x nrhs, leading dimension ld >= n; b is
 *            read only, x receives the solution in ORIGINAL row order.  b and x
 *            must not overlap.  dtype SPTRSV_F64 (double) or SPTRSV_F32 (float).
 *   opts   : may be NULL for defaults.
 *   stream : enqueue on this stream.
 *   report : NULL -> fully asynchronous (device errors surface on the next call
 *            with a report); non-NULL -> the call synchronises `stream` and fills it.
 * A plan's control words and device workspace (refinement vectors, staged right-hand
 * sides) are shared by all of its solves: solves of one plan must not run concurrently
 * (enqueue them on one stream); different plans may run at the same time.
 * Errors: ARG (sizes, dtype/precision without the needed value copy), NO_DEVICE,
 * LAUNCH (grid not co-resident), CUDA, TIMEOUT, NOT_CONVERGED (x still written). */
int sptrsv_solve(sptrsv_plan *plan, const void *b, void *x, int32_t nrhs, int64_t ld,
                 int32_t dtype, const sptrsv_solve_opts *opts, sptrsv_stream stream,
                 sptrsv_report *report);

/* sptrsv_solve with b and x in HOST memory (Eq. 2.1 as above): b_host (column-major,
 * leading dimension ld >= n) is copied into the plan's device staging buffer, the solve
 * runs there, and x is copied back into x_host, all enqueued on `stream` in that order.
 * Pinned host memory keeps the copies asynchronous; pageable memory works but the copies
 * synchronise.  x_host holds the result once the stream has passed this call (report
 * non-NULL: the call synchronises and fills it).  The staging buffer (2 n nrhs elements)
 * is allocated on first use and kept with the plan.  Errors as sptrsv_solve, plus ARG
 * for NULL host pointers. */
int sptrsv_solve_host(sptrsv_plan *plan, const void *b_host, void *x_host, int32_t nrhs, int64_t ld,
                      int32_t dtype, const sptrsv_solve_opts *opts, sptrsv_stream stream,
                      sptrsv_report *report);

/* Autotuner: time every candidate launch shape (sync mode x lanes per row x threads x
 * blocks per SM) of sptrsv_solve on the caller's b/x with CUDA events (x is overwritten),
 * remember the fastest in the plan for this (dtype, precision, nrhs class), and return it.
 * Later sptrsv_solve calls with opts->sync == SPTRSV_SYNC_AUTO use the remembered shape.
 *   base    : fixed fields (precision, tolerances, timeout); may be NULL.
 *   best    : receives the winning options (may be NULL); best_ms its time (may be NULL).
 * Synchronises `stream`.  Errors as sptrsv_solve; LAUNCH if no candidate could run. */
int sptrsv_autotune(sptrsv_plan *plan, const void *b, void *x, int32_t nrhs, int64_t ld,
                    int32_t dtype, const sptrsv_solve_opts *base, sptrsv_stream stream,
                    sptrsv_solve_opts *best, double *best_ms);

/* -------------------------------------------------------------- batching */
/* Many independent factors, each with its own block of right-hand sides, solved
 * by one persistent launch replayed from a CUDA graph.  Factors are independent,
 * so thread blocks pull (factor, RHS block of <= 32 columns) items from a queue,
 * longest critical path first, and walk each item's supersteps alone.  In
 * SPTRSV_PREC_F32_REFINE a block runs the item's whole refinement loop (FP32
 * sweeps, FP64 residuals, convergence test).  With opts->sync ==
 * SPTRSV_SYNC_AUTO the first run times the row mappings once per factor class
 * (lanes per row or right-hand-side tile) and keeps the fastest. */
typedef struct sptrsv_batch sptrsv_batch;

/* Build a batch over `count` plans (all on one device, analysed with the value
 * copy the precision needs); nrhs[f] right-hand sides for factor f.  dtype must
 * be SPTRSV_F64.  opts: precision, max_iters, refine_tol, threads (per block),
 * blocks_per_sm, sync (AUTO = autotune on first run, anything else = default
 * mapping).  The plans must outlive the batch. */
int sptrsv_batch_create(sptrsv_plan *const *plans, int32_t count, const int32_t *nrhs, int32_t dtype,
                        const sptrsv_solve_opts *opts, sptrsv_batch **out);

/* Run the batch: b[f], x[f] are device pointers (column-major, leading dimension
 * ld[f] >= n_f) for factor f.  Enqueued on `stream` (the first run also captures
 * the graph and may autotune, synchronising `stream`).  reports: NULL, or an
 * array of `count` reports (the call then synchronises and returns the first
 * failing factor's status, e.g. SPTRSV_ERR_NOT_CONVERGED). */
int sptrsv_batch_run(sptrsv_batch *batch, const void *const *b, void *const *x, const int64_t *ld,
                     sptrsv_stream stream, sptrsv_report *reports);

/* Release a batch (NULL is a no-op); enqueued runs must have finished. */
void sptrsv_batch_destroy(sptrsv_batch *batch);

/* One-shot convenience: create, run once, synchronise, destroy. */
int sptrsv_batch_solve(sptrsv_plan *const *plans, int32_t count, const void *const *b, void *const *x,
                       const int32_t *nrhs, const int64_t *ld, int32_t dtype, const sptrsv_solve_opts *opts,
                       sptrsv_stream stream, sptrsv_report *reports);

/* --------------------------------------------------------------- serving */
/* Continuous batching over resident factors.  A dispatcher thread admits
 * submitted requests in arrival order as soon as their device workspace fits
 * the HBM budget left by the registered factors, packs admitted requests into
 * one launch of the batched executor on a free stream slot and keeps admitting
 * while earlier launches run, so requests that arrive while others are on the
 * GPU overlap with them.  A launch lasts as long as its longest request, so one
 * launch takes requests of one duration class (their factor's wavefront count
 * in decades: < 1e3, < 1e4, longer), oldest class first.  Slots are CUDA
 * streams: give the process at least as many hardware queues
 * (CUDA_DEVICE_MAX_CONNECTIONS, default 8, up to 32, read when the CUDA context
 * is created) or launches queue behind each other.  Each request's result does not depend on
 * what it was batched with (it is computed by one thread block alone).
 * SPTRSV_SERVE_SERIAL_F64 serves the same stream the plain way - one request
 * per FP64 sptrsv_solve launch, one stream, arrival order - as a baseline with
 * identical bookkeeping. */
typedef struct sptrsv_server sptrsv_server;
enum { SPTRSV_SERVE_CONTINUOUS = 0, SPTRSV_SERVE_SERIAL_F64 = 1 };

typedef struct {
    int32_t mode;        /* SPTRSV_SERVE_*                                                  */
    int32_t streams;     /* concurrent launches in flight (8)                               */
    int32_t max_batch;   /* requests packed into one launch at most (256)                   */
    int32_t precision;   /* continuous mode: SPTRSV_PREC_F32_REFINE (default) or _F64       */
    int32_t max_iters;   /* refinement limits, as in sptrsv_solve_opts (6, 1e-13)           */
    double refine_tol;
    int32_t threads;     /* threads per block of the batched executor (256)                 */
    int32_t device;      /* CUDA device (0)                                                 */
} sptrsv_serve_opts;

typedef struct {
    int64_t submitted, completed, rejected, launches;
    double mean_batch;              /* requests per launch                                  */
    double p50_ms, p99_ms, max_ms, mean_ms;   /* latency = completion - submission          */
    double solves_per_s;            /* completed / (last completion - first submission)     */
    int64_t peak_workspace_bytes, arena_bytes, factor_bytes;
} sptrsv_serve_statistics;

void sptrsv_serve_opts_default(sptrsv_serve_opts *o);
/* Create a server with an HBM budget (bytes) for resident factors + request workspace.
 * Starts the dispatcher thread.  The workspace arena (budget minus factor bytes) is
 * allocated by the first submit. */
int sptrsv_serve_create(size_t hbm_budget, const sptrsv_serve_opts *opts, sptrsv_server **out);
/* Make an analysed plan resident (it must outlive the server); BUDGET if it does not fit.
 * All factors must be registered before the first submit. */
int sptrsv_serve_register(sptrsv_server *server, sptrsv_plan *plan, int32_t *factor_id);
/* Submit L_f x = b for nrhs right-hand sides: b, x are caller-owned device pointers
 * (column-major, leading dimension ld) that must stay valid until the request completes.
 * Returns at once with req_id; BUDGET if the request could never fit the budget. */
int sptrsv_serve_submit(sptrsv_server *server, int32_t factor_id, const double *b, double *x,
                        int32_t nrhs, int64_t ld, uint64_t *req_id);
/* Submit with HOST buffers (the serving boundary of a client that holds b and wants x in
 * host memory): b_host is n x nrhs column-major with leading dimension ldb, x_host receives
 * the solution (leading dimension ldx).  When the request is admitted its b is copied into
 * device staging carved from the HBM budget next to its workspace; after the solve x is
 * copied back into x_host on the same stream, and the request completes only then: poll and
 * wait report it done once x_host holds the result, and its latency (serve statistics)
 * includes both copies.  x_host is passed here, not at poll time, so that the device-to-host
 * copy is part of the request.  Both buffers must stay valid and x_host unread until the
 * request completed.  Page-locked buffers (cudaMallocHost, cudaHostRegister) keep the copies
 * asynchronous; pageable ones work but the dispatcher thread waits for each copy.  Errors as
 * sptrsv_serve_submit (BUDGET counts the staging too). */
int sptrsv_serve_submit_host(sptrsv_server *server, int32_t factor_id, const double *b_host, int64_t ldb,
                             double *x_host, int64_t ldx, int32_t nrhs, uint64_t *req_id);
/* PENDING until the request finished; then fills `out`, forgets the request and returns its
 * status (0, or e.g. SPTRSV_ERR_NOT_CONVERGED). */
int sptrsv_serve_poll(sptrsv_server *server, uint64_t req_id, sptrsv_report *out);
/* As poll, blocking up to timeout_s seconds (PENDING on timeout). */
int sptrsv_serve_wait(sptrsv_server *server, uint64_t req_id, double timeout_s, sptrsv_report *out);
/* Block until every submitted request has completed (PENDING on timeout). */
int sptrsv_serve_drain(sptrsv_server *server, double timeout_s);
int sptrsv_serve_stats(sptrsv_server *server, sptrsv_serve_statistics *out);
/* Stop the dispatcher, wait for in-flight launches, free the server (NULL: no-op). */
void sptrsv_serve_destroy(sptrsv_server *server);

/* --------------------------------------------------------- no allocation */
/* Largest factor sptrsv_solve_csr_noalloc accepts (rows). */
#define SPTRSV_NOALLOC_MAX_ROWS (1 << 20)

/* Allocation-free solve for callers that cannot let a library call cudaMalloc
 * (device memory drawn only from the caller's own pool or budget, or a
 * latency-critical loop where an allocation may synchronise the device).  The
 * paper has no counterpart: this is a deployment convenience.
 *
 * Solves L x = b for one right-hand side directly on a caller-owned DEVICE CSR
 * factor (0-based, int32, columns strictly increasing, diagonal last and
 * non-zero), rows taken in natural order with per-row ready flags - no
 * analysis, no plan.  b and x are device vectors of n doubles; x must not
 * overlap b or the factor.  Allocates nothing: its scratch (one ready flag per
 * row plus 256 bytes of control words, 4 MiB + 256 B in all) is a fixed array
 * that every GPU loading this library holds until the process exits.
 *   - n > SPTRSV_NOALLOC_MAX_ROWS is rejected with SPTRSV_ERR_ARG.
 *   - The first call on a device (with that device current) resolves the
 *     array's device address once.
 *   - Every call shares the array; the flags keep the last call's epoch and
 *     the control words are cleared at the start of each call.  Calls that
 *     overlap on the GPU (e.g. on two streams) race: serialise them.
 *   - The call synchronises `stream`.  Malformed factors are detected on the
 *     device where they would break memory safety (SPTRSV_ERR_ARG,
 *     SPTRSV_ERR_NOT_LOWER); waits are bounded (SPTRSV_ERR_TIMEOUT). */
int sptrsv_solve_csr_noalloc(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                             const double *val, const double *b, double *x, sptrsv_stream stream);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif
#ifdef __cplusplus
}
#endif
#endif /* SPTRSV_H */
