/*
 * race.h — C ABI of the GB300 SymmSpMV library (RACE-scheduled symmetric
 * sparse matrix-vector multiplication from upper-triangle CRS storage).
 *
 * Paper: C. Alappat et al., "A Recursive Algebraic Coloring Technique for
 * Hardware-Efficient Symmetric Sparse Matrix-Vector Multiplication",
 * arXiv 1907.06487.  Section, algorithm and equation names below refer to it.
 *
 * General conventions
 *   - Every entry point returns an int status (RACE_OK = 0 or a RACE_ERR_*
 *     code); none throws, none traps on the device.  race_strerror() maps a
 *     code to text.  race_last_error_detail() gives a one-line reason for
 *     the most recent failure on the calling thread.
 *   - "host" pointers are CPU memory; "device" pointers are CUDA global
 *     memory of the current device.  Streams are cudaStream_t passed as
 *     void* (NULL = legacy default stream).  All device work is enqueued on
 *     the caller's stream; nothing synchronises the device unless stated.
 *   - Vectors seen by symm_spmv / symm_spmm / spmv_full are in the
 *     schedule's PERMUTED order (the paper runs all kernels on the permuted
 *     matrix, Sec. 4.1 and 6.1).  race_permute / race_unpermute convert.
 *   - Outputs are overwritten (b = A x), not accumulated.
 *   - x and b (X and B) must not alias.
 */
#ifndef RACE_GB300_H
#define RACE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define RACE_OK               0
#define RACE_ERR_INVALID      1  /* malformed input: n <= 0, entry below the
                                    diagonal, duplicate or out-of-range column,
                                    non-monotone row_ptr, non-finite value,
                                    bad parameter, NULL pointer             */
#define RACE_ERR_OVERFLOW     2  /* a count does not fit the int32 layout   */
#define RACE_ERR_NOMEM        3  /* host or device allocation failed        */
#define RACE_ERR_CUDA         4  /* a CUDA runtime call failed              */
#define RACE_ERR_TIMEOUT      5  /* a bounded device wait gave up           */
#define RACE_ERR_UNSUPPORTED  6  /* valid request this build does not serve */

/* ---- value types --------------------------------------------------------- */
#define RACE_F64 0   /* matrix values stored as double                       */
#define RACE_F32 1   /* matrix values stored as float; products and sums in
                        double (x, b and accumulation stay FP64)             */

/* ---- balancing unit (Sec. 4.3: rows or nonzeros) ------------------------- */
#define RACE_BAL_ROWS 0   /* paper default                                   */
#define RACE_BAL_NNZ  1   /* vertex weight = nonzeros of its full row        */

/* ---- flags for race_params.flags ----------------------------------------- */
#define RACE_FLAG_HOST_ONLY 1u  /* build the schedule on the host only: no
                                   device upload (race_export / race_get_info
                                   work, compute entry points return
                                   RACE_ERR_UNSUPPORTED).  Needs no GPU.     */
#define RACE_FLAG_NO_WINDOWS 2u /* skip building the shared-memory window
                                   tiles (faster builds; the window
                                   executors then fall back to
                                   RACE_EXEC_ROWS_RED)                      */
#define RACE_FLAG_NATURAL_ORDER 4u /* no RACE schedule: identity permutation
                                   and one phase whose single leaf holds every
                                   row.  For comparisons on the input order
                                   (the row-parallel executors run as usual;
                                   the leaf executors then run serially).   */
#define RACE_FLAG_PSEUDO_PERIPHERAL 8u /* stage-0 roots: instead of the last
                                   unvisited vertex itself, a pseudo-
                                   peripheral vertex of its connected
                                   component (George and Liu's iteration,
                                   ACM TOMS 5, 1979: BFS, take a vertex of
                                   minimum degree in the deepest level, lowest
                                   index on ties, repeat while the
                                   eccentricity grows).  The paper's inputs
                                   are RCM-ordered, whose last row is such a
                                   vertex (Sec. 6.1); this flag gives other
                                   orders the same start.  Recursion roots
                                   are unchanged.                           */
#define RACE_FLAG_ONE_LEVEL_STAGE0 32u /* stage-0 level groups of one level
                                   or more instead of two (k = 1 in the
                                   pairing and balancing of Sec. 4.4.3 at
                                   stage 0 only).  With upper storage in level
                                   order a row of level j updates b only in
                                   levels j and j + 1, so groups of the same
                                   colour one level apart never share an
                                   entry of b (they are not distance-2
                                   independent: an update of every neighbour
                                   would conflict); up to twice the stage-0
                                   groups.  Deeper stages keep k = 2: a
                                   group's halo neighbours are not confined
                                   to the next sub-level.                   */
#define RACE_FLAG_RCM 16u /* relabel the matrix by reverse Cuthill-McKee
                                   before the construction, as the paper does
                                   with all of its inputs (Sec. 6.1): each
                                   component (in the order of its lowest
                                   vertex) from its pseudo-peripheral vertex,
                                   breadth first, the neighbours newly reached
                                   from a vertex by increasing degree (lowest
                                   index on ties), the sequence reversed.  The
                                   RACE levels then keep the RCM order inside
                                   each level; the schedule's permutation is
                                   composed with it.  With
                                   RACE_FLAG_NATURAL_ORDER: the RCM order
                                   alone, one leaf.                         */

/* Upper-triangle CRS matrix in HOST memory (Sec. 3.2, Alg. "SymmSpMV"):
 * row i holds the entries (i, j) with j >= i.  Columns may come in any
 * order within a row; a missing diagonal is treated as an explicit 0.0.
 * The library copies what it needs; the caller keeps ownership.           */
typedef struct {
    int32_t n;              /* number of rows = columns, > 0                 */
    int64_t nnz;            /* stored entries, = row_ptr[n]                  */
    const int32_t *row_ptr; /* n+1 offsets, row_ptr[0] = 0, non-decreasing   */
    const int32_t *col;     /* nnz column indices, row <= col < n            */
    const void *val;        /* nnz values: double (RACE_F64) or float (F32)  */
    int32_t val_type;       /* RACE_F64 | RACE_F32                           */
} race_csr_upper;

/* Parameters of the schedule (Sec. 4.4.3 and 5.1).                          */
typedef struct {
    int32_t dist_k;      /* distance of the colouring; must be 2 (SymmSpMV) */
    int32_t n_workers;   /* N_t: number of schedule workers, >= 1           */
    double eps[8];       /* epsilon_s for stage s = 0..7 (later stages use
                            eps[7]); each in [0.5, 1).  Paper's choice:
                            0.8, 0.8, then 0.5                              */
    int32_t max_depth;   /* number of stages allowed: 0 = no colouring (one
                            serial leaf), 1 = stage 0 only, ...; -1 = as
                            deep as the epsilon rule goes (paper)           */
    int32_t balance;     /* RACE_BAL_ROWS | RACE_BAL_NNZ                    */
    int32_t group_lanes; /* lanes that execute one leaf row together on the
                            GPU: 0 = automatic, else 4, 8, 16 or 32         */
    uint32_t flags;      /* RACE_FLAG_*                                     */
} race_params;

/* Summary of a built schedule.                                             */
typedef struct {
    int32_t n;           /* rows                                           */
    int64_t nnz_upper;   /* stored upper entries incl. diagonal            */
    int32_t n_levels;    /* BFS levels of the whole graph (N_l)            */
    int32_t n_phases;    /* globally synchronised phases after flattening  */
    int32_t n_leaves;    /* non-empty leaves over all phases               */
    int32_t n_nodes;     /* nodes of the RACE tree incl. the root          */
    int32_t depth;       /* deepest stage + 1                              */
    int32_t n_workers;   /* N_t                                            */
    int32_t val_type;    /* RACE_F64 | RACE_F32                            */
    int32_t group_lanes; /* lanes per leaf row on the GPU                  */
    double eta;          /* parallel efficiency (Sec. 5: N_r / (N_eff * N_t)) */
    int64_t neff_root;   /* effective row count of the root (Sec. 5)       */
} race_info;

typedef struct race_schedule race_schedule;  /* opaque */

/* Set params to the paper's defaults: dist_k 2, eps = {0.8, 0.8, 0.5...},
 * max_depth -1, balance rows, group_lanes automatic, n_workers given.      */
void race_default_params(race_params *p, int32_t n_workers);

/* race_build — the RACE preprocessing (Sec. 4): level construction (Alg.
 * "Construction of levels"), distance-2 level groups with epsilon-driven
 * thread assignment (Sec. 4.4.3), load balancing (Alg. "Load Balancing"),
 * recursion with the distance-1 halo (Sec. 4.4.2), the tree and its
 * efficiency eta (Sec. 5), flattened into phases.  The matrix is permuted
 * symmetrically and uploaded to the device on `stream` (unless
 * RACE_FLAG_HOST_ONLY); the call returns after the upload has completed.
 * On success *out owns host and device copies until race_free.
 * Errors: RACE_ERR_INVALID (malformed matrix or parameters, unknown flag
 * bits, RACE_FLAG_PSEUDO_PERIPHERAL together with RACE_FLAG_NATURAL_ORDER),
 * _UNSUPPORTED (dist_k other than 2), _OVERFLOW, _NOMEM, _CUDA.            */
int race_build(const race_csr_upper *a, const race_params *p, void *stream, race_schedule **out);

/* race_build_coloring — the multicolouring schedules the paper compares
 * RACE with (Sec. 3.3, Sec. 6.3), built in-house from its description:
 *   RACE_COLOR_MC:   every row is a unit;
 *   RACE_COLOR_ABMC: units are blocks of block_rows consecutive rows of the
 *                    (RCM-relabelled, with RACE_FLAG_RCM) input order -- the
 *                    partitioning step, for which the paper uses METIS and a
 *                    block size from a scan over 4..128 -- 1 <= block_rows <=
 *                    4096.
 * Units are coloured first fit in index order: a unit takes the smallest
 * colour no earlier unit within distance 2 of it (in the symmetric graph)
 * holds, so the rows of one colour never share an entry of b (the
 * distance-2 condition of Sec. 4.2).  The permutation lists the units colour
 * by colour; each colour is a phase and each unit a leaf, so every executor
 * and entry point serves the result like a RACE schedule (race_get_info
 * reports one tree node; eta = N / (N_eff N_t) with N_eff the sum over
 * phases of their longest leaf, at most 1).  n_workers: N_t for eta.
 * flags: RACE_FLAG_HOST_ONLY, RACE_FLAG_NO_WINDOWS, RACE_FLAG_RCM.
 * Errors as race_build; RACE_ERR_INVALID also for an unknown method or a
 * block size out of range.                                                */
#define RACE_COLOR_MC 0
#define RACE_COLOR_ABMC 1
int race_build_coloring(const race_csr_upper *a, int32_t method, int32_t block_rows, int32_t n_workers, uint32_t flags,
                        void *stream, race_schedule **out);

/* race_upload — turns a schedule built with RACE_FLAG_HOST_ONLY into a
 * device schedule (uploads it on `stream`, returns after the copies have
 * completed); no-op for a device schedule.  Lets callers build schedules on
 * many host threads or processes and use the GPU only for the upload.
 * Errors: RACE_ERR_NOMEM, RACE_ERR_CUDA (the schedule stays host-only).    */
int race_upload(race_schedule *s, void *stream);

/* symm_spmv — b = A x for the symmetric A whose upper triangle was given,
 * i.e. b = A_u x + A_u^T x - diag(A) x (Alg. "SymmSpMV"), with the
 * schedule's current executor (race_set_launch; RACE_EXEC_LEAF_GROUP after
 * race_build).  The leaf executors (RACE_EXEC_LEAF_GROUP, _LEAF_CTA,
 * _WINDOW_RACE, _PERSIST_GROUP, _PERSIST_CTA, _PHASE_DF64) run the schedule
 * phase by phase, so that no two concurrent leaves write the same entry of
 * b; the row-parallel executors (_ATOMIC, _ROWS_RED, _STREAM_RED,
 * _PIPE_RED, _WINDOW_RED, _DF64_RED, _SELL_DF64, _STAGED) run all rows at
 * once on the schedule's permuted matrix and resolve the concurrent writes
 * to b by reductions at L2.  x, b: device arrays of n doubles in permuted
 * order.                                                                   */
int symm_spmv(const race_schedule *s, const double *x_d, double *b_d, void *stream);

/* Executors of SymmSpMV (symm_spmv_exec).                                  */
#define RACE_EXEC_LEAF_GROUP 0  /* one leaf per group of lanes, rows in order,
                                   plain loads/stores of b (the paper's model:
                                   a leaf runs on one thread)               */
#define RACE_EXEC_LEAF_CTA   1  /* one leaf per thread block, the leaf's rows
                                   in parallel; updates within a leaf are
                                   reductions at L2; leaves of a phase never
                                   share an entry of b                      */
#define RACE_EXEC_ATOMIC     2  /* comparison point: no phases, every update
                                   a reduction at L2 (ignores the schedule)  */

#define RACE_EXEC_ROWS_RED   3  /* all rows at once in row blocks (streamed,
                                   coalesced); the transposed part and the row
                                   sums are reductions at L2 on the permuted
                                   matrix                                   */

#define RACE_EXEC_STREAM_RED 4  /* as ROWS_RED, with row blocks staged into
                                   shared memory by bulk asynchronous copies
                                   (multi-stage pipeline, persistent grid)  */

#define RACE_EXEC_PIPE_RED   5  /* one row per thread, software-pipelined over
                                   the thread's rows (x gathers of row i,
                                   val/col of row i+1 and row pointers of row
                                   i+2 in flight together); updates of b as
                                   reductions at L2                         */

#define RACE_EXEC_WINDOW_RED 6  /* tiles of consecutive rows whose write set
                                   (rows + upper targets, at most 2048) is
                                   a shared-memory window: x staged, updates
                                   accumulated by shared-memory atomics, then
                                   flushed coalesced as L2 reductions       */
#define RACE_EXEC_WINDOW_RACE 7 /* the same windows over the RACE leaves, one
                                   launch per phase; a leaf's tiles run in
                                   order on one block and the windows are
                                   flushed with plain loads and stores: the
                                   leaves of a phase are distance-2
                                   independent, so no two blocks write one
                                   entry of b (conflict-free, no atomics in
                                   global memory)                           */
#define RACE_EXEC_DF64_RED  8   /* as ROWS_RED (group_lanes lanes per row):
                                   FP64 row sums, and the transposed updates
                                   a_ij x_i of (4 - fp64_quarters) of every
                                   four row groups formed off the FP64 pipe
                                   by an integer product of the two
                                   significands (the exact product
                                   truncated, relative error below 2^-51
                                   each; the result stays within 1e-12
                                   sum_j |a_ij x_j| of the exact one).  The
                                   name is kept from the double-float
                                   product this executor used first.  First use
                                   checks the off-diagonal values once and
                                   returns RACE_ERR_UNSUPPORTED if one is
                                   nonzero and outside [2^-50, 2^51) in
                                   magnitude; rows whose x_i lies outside
                                   that range scatter in FP64.              */
#define RACE_EXEC_SELL_DF64 9   /* the arithmetic of DF64_RED on a SELL-32-
                                   sigma copy of the permuted upper matrix
                                   (chunks of 32 rows stored column by
                                   column, rows sorted by length within
                                   windows of 1024): one warp per chunk, one
                                   lane per row, coalesced value and column
                                   loads.  First use builds and uploads the
                                   copy (about the matrix's size again);
                                   regs_per_row = entries per lane and step
                                   (4, 8 or 16).                            */
#define RACE_EXEC_STAGED 10     /* as ROWS_RED with one row per lane: warp
                                   tiles of 32 consecutive rows whose stored
                                   values and columns are copied into shared
                                   memory by the bulk-copy (TMA) engine, two
                                   stages per warp so the next tile's copy
                                   overlaps the current tile's work; x
                                   gathered, the transposed update and the
                                   row sums reductions at L2.  Per quarter of
                                   the warps the row sums run in FP64 or in
                                   double-float arithmetic
                                   (rowsum_fp64_quarters) and the transposed
                                   products in FP64 or by DF64_RED's integer
                                   product (fp64_quarters); the
                                   result stays within 1e-12 sum_j
                                   |a_ij x_j| of the exact one.  Entries
                                   whose value or x lies outside
                                   [2^-50, 2^51) in magnitude (zero excepted)
                                   and rows of more than 64 entries are taken
                                   in FP64.  regs_per_row: entries per lane
                                   and step (4, or 8 when >= 8).  Needs no
                                   preparation and no memory beyond the
                                   schedule's.                              */
#define RACE_EXEC_PERSIST_GROUP 11 /* LEAF_GROUP's work (one leaf per group of
                                   group_lanes lanes, rows in order, plain
                                   loads and stores of b) with every phase
                                   in one cooperative launch: the phases
                                   are separated by a grid barrier inside
                                   the kernel instead of kernel boundaries
                                   (Sec. 4.4.3).  Every barrier wait is
                                   bounded; one that gives up records
                                   RACE_ERR_TIMEOUT (race_poll_status) and
                                   the launch ends with b incomplete.
                                   Calls on one schedule must not overlap
                                   (they share the barrier words).          */
#define RACE_EXEC_PERSIST_CTA 12 /* the same for LEAF_CTA's work (one leaf
                                   per block, the leaf's rows in parallel,
                                   updates inside a leaf as L2 reductions)  */
#define RACE_EXEC_PHASE_DF64 13 /* DF64_RED's arithmetic (one row per lane,
                                   FP64 row sums, fp64_quarters of the row
                                   groups' transposed products in FP64, the
                                   rest by the integer product) phase by
                                   phase: one
                                   launch per phase over the rows of the
                                   phase's leaves (a list of them built with
                                   the schedule, 4 bytes per row), 256 rows
                                   a block at a time.  No two concurrently
                                   running leaves share an entry of b; the
                                   rows of one leaf may run in different
                                   blocks, so updates inside a leaf are L2
                                   reductions.
                                   blocks_per_sm, regs_per_row (4 or 8) as
                                   for DF64_RED; SymmSpMM runs DF64_RED's
                                   row-parallel kernel.  Same range check
                                   and error bound as DF64_RED.             */

/* Launch shape of a kernel family; set by an autotuner or by hand.          */
typedef struct {
    int32_t executor;        /* symm_spmv: RACE_EXEC_*; spmv_full: 0 = row
                                blocks in registers, 1 = staged stream,
                                2 = one row per thread, pipelined           */
    int32_t group_lanes;     /* lanes per row group: 1, 2, 4, 8, 16 or 32   */
    int32_t rows_per_group;  /* consecutive rows a group streams: 1,2,4,8
                                (RACE_EXEC_ROWS_RED and spmv_full)          */
    int32_t blocks_per_sm;   /* resident 256-thread blocks per SM, 0 = max  */
    int32_t regs_per_row;    /* row entries held in registers by the
                                pipelined executors: 4, 8 or 16; entries
                                per lane and step of RACE_EXEC_DF64_RED
                                (4, or 8 when >= 8)                         */
    int32_t fp64_quarters;   /* RACE_EXEC_DF64_RED (and its SymmSpMM): in
                                this many of every four row iterations of a
                                warp (0..4) the transposed updates use FP64
                                multiplies, in the rest the integer product
                                of the significands; shares the work between the
                                FP64 and integer pipes, spread evenly over
                                each SM's four FP64 units                */
    int32_t rowsum_fp64_quarters; /* RACE_EXEC_STAGED: in this many quarters
                                of the warps (0..4) the row sums are FP64
                                multiply-adds, in the rest double-float
                                arithmetic (other executors: always FP64) */
} race_launch;

/* race_set_launch / race_get_launch — which = 0: symm_spmv, which = 1:
 * spmv_full.  Out-of-range shapes return RACE_ERR_INVALID.                 */
int race_set_launch(race_schedule *s, int32_t which, const race_launch *l);
int race_get_launch(const race_schedule *s, int32_t which, race_launch *l);

/* race_probe_scatter — diagnostic, computes nothing of SymmSpMV.  Replays,
 * over the schedule's permuted upper matrix and with the row-parallel
 * executors' access pattern (one row per thread, four entries per step),
 * either the transposed update's reductions alone (mode 0: b[j] += 1.0 for
 * every stored a_ij with j != i; b is not zeroed) or the column stream
 * alone (mode 1: b[i] = sum of row i's column indices).  Timing both
 * separates the cost of the reductions at L2, the floor of every executor
 * that scatters by reductions, from the loads.  b_d: device array of n
 * doubles.  RACE_ERR_INVALID for another mode.                            */
int race_probe_scatter(const race_schedule *s, int32_t mode, double *b_d, void *stream);

/* race_probe_peaks — diagnostic ceilings for the roofline, computes nothing
 * of SymmSpMV.  The paper's roofline takes its memory term as a range from
 * the load-only to the copy bandwidth (Sec. 3, Table "test bed"); GB300's
 * FP64 rate is the second roof of the FP64-heavy SymmSpMM.
 *   what = 0: reads in_d[0, n) once (16-byte loads, streaming), the bits
 *             of each block's words folded by XOR into out_d[block]: time it
 *             for the load-only bandwidth (8 n bytes);
 *   what = 1: eight independent chains of `iters` FP64 fused multiply-adds
 *             per thread: 8 * iters * threads FMAs, threads = 1024 per SM.
 * Grid: 4 blocks of 256 threads per SM; out_d: device array of at least
 * 4096 doubles.  in_d (what 0): device, 16-byte aligned.
 * Errors: RACE_ERR_INVALID (bad what, n < 0, misaligned input, iters < 1),
 * _UNSUPPORTED (more than 4096 blocks), _CUDA.                            */
int race_probe_peaks(int32_t what, const double *in_d, int64_t n, double *out_d, int32_t iters, void *stream);

/* race_probe_reductions — diagnostic, computes nothing of SymmSpMV: the ways
 * the contributions of the transposed update (Alg. "SymmSpMV": b[j] +=
 * a_ij x_i) can be combined on this GPU, each timed over the same m target
 * indices idx_d[0, m) (device int32, clamped to [0, max_index]):
 *   mode 0: reduction at L2 (red.global.add.f64), target[idx[i]] += 1;
 *   mode 1: plain load, add and store of target[idx[i]], as a
 *           conflict-free schedule would allow (repeated indices race);
 *   mode 2: FP64 atomic add into the block's shared memory, slot
 *           idx[i] mod 4096;
 *   mode 3: the same into the shared memory of the other block of a
 *           two-block cluster (distributed shared memory);
 *   mode 4: bulk reduction of a 16-double row from shared memory into
 *           target[16 idx[i] .. 16 idx[i] + 15] (cp.reduce.async.bulk).
 * target_d: device doubles, 16-byte aligned, n_target at least max_index + 1
 * (16 (max_index + 1) for mode 4; and at least 8 per SM for modes 2 and 3,
 * whose blocks store one value each at the end).  Grid: 8 blocks of 256
 * threads per SM.  Errors: RACE_ERR_INVALID, _CUDA.                       */
int race_probe_reductions(int32_t mode, const int32_t *idx_d, int64_t m, int32_t max_index, double *target_d,
                          int64_t n_target, void *stream);

/* race_poll_status — synchronises `stream`, then returns RACE_ERR_TIMEOUT
 * (and clears it) if a bounded device wait of this schedule's kernels gave
 * up since the last poll, else RACE_OK.                                    */
int race_poll_status(race_schedule *s, void *stream);

/* race_probe_wait_timeout — diagnostic of the bounded device waits,
 * computes nothing usable: runs the RACE_EXEC_STAGED kernel on x_d / b_d
 * (device arrays of n doubles, not aliasing; b_d is left undefined) with
 * every stage's mbarrier expecting 16 bytes more than its copies deliver
 * and a spin limit of 4096 polls, so every wait gives up while none of the
 * copies is left in flight.  The kernel records RACE_ERR_TIMEOUT in the
 * schedule's status word: race_poll_status then returns it once and clears
 * it.  No device fault, trap or endless wait is involved.  The paper has no
 * counterpart (failure detection of this library's own kernels).
 * Errors: RACE_ERR_INVALID (NULL, aliasing), _UNSUPPORTED (host-only
 * schedule), _CUDA.                                                        */
int race_probe_wait_timeout(const race_schedule *s, const double *x_d, double *b_d, void *stream);

/* race_probe_barrier_timeout — diagnostic of the one-launch executors'
 * grid barriers, computes nothing usable: runs RACE_EXEC_PERSIST_CTA on
 * x_d / b_d (device arrays of n doubles, not aliasing; b_d is left
 * undefined) with every barrier expecting one block more than the launch
 * has (a wrong worker count made on the host) and a limit of 4096 polls
 * (about 16 ms), so the first barrier gives up in every block and the
 * kernel ends.  The
 * kernel records RACE_ERR_TIMEOUT in the schedule's status word:
 * race_poll_status then returns it once and clears it.  The paper has no
 * counterpart (failure detection of this library's own kernels).
 * Errors: RACE_ERR_INVALID (NULL, aliasing), _UNSUPPORTED (host-only
 * schedule, or a schedule of a single phase: no barrier), _CUDA.          */
int race_probe_barrier_timeout(const race_schedule *s, const double *x_d, double *b_d, void *stream);

/* symm_spmv_exec — symm_spmv with an explicit executor (RACE_EXEC_*).
 * Same arguments, layout and errors as symm_spmv.                          */
int symm_spmv_exec(const race_schedule *s, int32_t executor, const double *x_d, double *b_d, void *stream);

/* symm_spmm — B = A X for k right-hand sides, X and B row-major n x k
 * device arrays (element (i, c) at i*k + c) in permuted row order.
 * 1 <= k <= 16.                                                            */
int symm_spmm(const race_schedule *s, int32_t k, const double *X_d, double *B_d, void *stream);

/* spmv_full — the traffic baseline: Alg. "SpMV using the CRS format" on the
 * full (both triangles) CRS of the same permuted matrix, row-parallel, no
 * schedule.  The full matrix is built and uploaded on the first call (or
 * by race_prepare_full) and kept with the schedule.  k = 1.               */
int spmv_full(const race_schedule *s, const double *x_d, double *b_d, void *stream);

/* symm_gs — `sweeps` symmetric Gauss-Seidel sweeps for A x = b under the
 * schedule (the paper names Gauss-Seidel among the kernels with distance-k
 * dependencies that RACE serves): a forward pass over the phases in order,
 * the rows of each leaf ascending, then a backward pass over the phases in
 * reverse, rows descending; each row x_i <- (b_i - sum_{j != i} a_ij x_j) /
 * a_ii from the current x.  Leaves of a phase share no edge, so the result
 * is the serial sweep in that execution order.  b_d (input) and x_d (start
 * value in, result out) are caller-owned device arrays of n doubles in
 * permuted order and must not alias; the full CRS is built on first use as
 * for spmv_full.  One launch per phase and pass on `stream`; each leaf runs
 * on a group of the schedule's group_lanes lanes (race_set_launch; 1, 2,
 * 4, 8, 16 or 32), four entries a lane per step.  Colourings with leaves of
 * one or a few rows (race_build_coloring) keep every lane busy; RACE's
 * leaves of many rows are chains of dependent row updates.  A zero
 * diagonal gives inf or nan entries.
 * Errors: RACE_ERR_INVALID (NULL, aliasing, sweeps < 0), _UNSUPPORTED
 * (host-only schedule), _OVERFLOW, _NOMEM, _CUDA.                          */
int symm_gs(const race_schedule *s, const double *b_d, double *x_d, int32_t sweeps, void *stream);

/* symm_kacz — `sweeps` symmetric Kaczmarz sweeps for A x = b under the
 * schedule (the paper names the Kaczmarz solver among the kernels RACE
 * serves): the passes of symm_gs, each row projecting x onto its hyperplane,
 * f = (b_i - sum_j a_ij x_j) / sum_j a_ij^2, x_j += f a_ij for every stored
 * column j of the row.  A row update writes x at all its columns, so
 * concurrent leaves must share no column: the schedule's distance-2
 * independence, checked once per schedule on the host (schedules built with
 * RACE_FLAG_ONE_LEVEL_STAGE0 are write-disjoint for half storage only and
 * are refused with RACE_ERR_UNSUPPORTED).  Otherwise arguments, layout and
 * errors as for symm_gs; a zero row gives inf or nan entries.              */
int symm_kacz(const race_schedule *s, const double *b_d, double *x_d, int32_t sweeps, void *stream);

/* race_matrix_powers — the powers A x, A^2 x, ..., A^p x of the symmetric
 * matrix (the paper's conclusion names in-place matrix powers among the
 * kernels a level-based formulation serves): column q of Y (entries
 * q*n .. q*n+n-1) = A^(q+1) x, each column computed from the previous one,
 * no vector storage besides Y.  x_d: n doubles, Y_d: n*p doubles, device,
 * permuted order, not overlapping; Y is overwritten.  1 <= p <= 64.
 *   RACE_MPK_SWEEPS: p calls of symm_spmv with the schedule's executor.
 *   RACE_MPK_WAVEFRONT: one cooperative launch over (power, row block)
 *     items: block t of power q starts once power q-1 is complete up to the
 *     last block that block t's columns reach (in level order the rows of a
 *     level couple only to the neighbouring levels, Sec. 4.1), so several
 *     powers advance together over the matrix.  Arithmetic as
 *     RACE_EXEC_DF64_RED with the schedule's fp64_quarters (all FP64 when a
 *     stored value lies outside [2^-50, 2^51)).  FP64-stored values
 *     only.  The first call builds the block table on the host and uploads
 *     it (allocates and waits for `stream`), and a call with a larger p than
 *     before allocates its done flags: make those calls outside stream
 *     capture.  Every wait is bounded; race_poll_status reports a timeout.
 * Errors: RACE_ERR_INVALID (NULL, overlap, p, mode), _UNSUPPORTED (host-only
 * schedule; FP32 values in the wavefront mode), _NOMEM, _CUDA.            */
#define RACE_MPK_SWEEPS 0
#define RACE_MPK_WAVEFRONT 1
int race_matrix_powers(race_schedule *s, int32_t p, const double *x_d, double *Y_d, int32_t mode, void *stream);

/* Build and upload the full CRS used by spmv_full now (optional).          */
int race_prepare_full(race_schedule *s, void *stream);

/* race_permute: out[new] = in[perm[new]] (original -> permuted order);
 * race_unpermute: out[perm[new]] = in[new].  in/out: device arrays of n*k
 * doubles, row-major with k columns; must not alias.                       */
int race_permute(const race_schedule *s, const double *in_d, double *out_d, int32_t k, void *stream);
int race_unpermute(const race_schedule *s, const double *in_d, double *out_d, int32_t k, void *stream);

/* Copy the permutation perm[new] = old (n int32) to host memory.          */
int race_get_perm(const race_schedule *s, int32_t *perm_host);

/* Copy the permuted upper CRS to host memory: row_ptr (n+1), col (nnz),
 * val (nnz of the stored type).  Any pointer may be NULL to skip it.       */
int race_get_matrix(const race_schedule *s, int32_t *row_ptr, int32_t *col, void *val);

/* Copy the flattened phases: stage_ptr (n_phases+1) offsets into the leaf
 * arrays; leaf_lo/leaf_hi (n_leaves) row ranges [lo, hi) in permuted order.*/
int race_get_phases(const race_schedule *s, int32_t *stage_ptr, int32_t *leaf_lo, int32_t *leaf_hi);

int race_get_info(const race_schedule *s, race_info *info);

/* race_export — canonical byte image of the schedule (for bit-exact
 * comparison and caching).  With buf == NULL, *size receives the needed
 * size.  Layout (little-endian): int32 magic 0x45434152, version 1, n,
 * n_workers, dist_k, balance, max_depth, n_nodes, n_phases, n_leaves, 0, 0;
 * double eps[8], eta; int32 perm[n]; int32 stage_ptr[n_phases+1];
 * n_leaves x (int32 lo, hi); then the tree in preorder, per node: int32
 * stage, color, lo, hi, n_threads, thread_lo, n_levels_in_parent,
 * n_sublevels, n_children, phase_count, phase_offset; int64 size, neff.    */
int race_export(const race_schedule *s, void *buf, size_t *size);

/* race_import — a schedule rebuilt from a race_export image and the matrix
 * it was built from, without running the construction of Sec. 4 again (a
 * schedule cache: the construction takes seconds on large matrices, the
 * import one pass over the matrix).  The matrix is canonicalised and
 * permuted by the image's permutation; the image is checked entirely:
 * header, sizes, permutation, phase offsets, leaves covering every row
 * exactly once, the tree's shape, and that no two leaves of one phase update
 * the same entry of b on this matrix (the distance-2 condition of Sec. 4.2).
 * image/size: caller-owned bytes, only read.  flags: RACE_FLAG_HOST_ONLY and
 * RACE_FLAG_NO_WINDOWS, as for race_build.  The launch shape starts at the
 * defaults of race_build and group_lanes is automatic.  race_export of the
 * result reproduces the image byte for byte.
 * An image built from another matrix of the same size is refused when its
 * phases conflict on this one; if they happen not to, it is accepted (the
 * executors need only that) and keeps the other matrix's tree statistics
 * (eta, N_eff, levels).
 * Errors: RACE_ERR_INVALID (malformed image, or phases that conflict on this
 * matrix; reason in race_last_error_detail), _OVERFLOW, _NOMEM, _CUDA.     */
int race_import(const race_csr_upper *a, const void *image, size_t size, uint32_t flags, void *stream,
                race_schedule **out);

/* ---- batches and tuning (beyond the paper: many matrices of uneven size in one
 * captured graph; launch shapes picked by an autotuner) ------------------- */
typedef struct race_batch race_batch;  /* opaque */

/* race_batch_create — captures from `stream` (not the legacy default
 * stream) one symm_spmv (k == 1) or symm_spmm (1 < k <= 16) per schedule,
 * with the schedule's current launch shape, on the caller-owned device
 * arrays X_d[i] / B_d[i] (n_i x k row-major, permuted order), into one CUDA
 * graph whose matrices run as up to 8 parallel branches (matrices are
 * independent; each goes to the branch with the least stored work so far,
 * largest first), forked from and joined into `stream`.  The arrays must
 * stay valid while the batch is used; two entries must not share an output
 * array.  The call enqueues nothing; race_batch_launch replays the batch.
 * Errors: RACE_ERR_INVALID, RACE_ERR_CUDA.                                  */
int race_batch_create(race_schedule *const *s, int32_t count, int32_t k, const double *const *X_d,
                      double *const *B_d, void *stream, race_batch **out);
int race_batch_launch(race_batch *b, void *stream);
void race_batch_free(race_batch *b);

/* race_autotune — times the candidate launch shapes (executors
 * RACE_EXEC_ROWS_RED, RACE_EXEC_PIPE_RED and, when the matrix's values are
 * in its range, RACE_EXEC_DF64_RED, with their lane, row and register
 * shapes, default and 4 blocks per SM, RACE_EXEC_DF64_RED also 6 blocks per
 * SM, with 0, 1 or 2 FP64 quarters) of symm_spmv (k == 1) or
 * symm_spmm (k > 1) on the given buffers: one warm-up and `reps` timed
 * calls each, CUDA events on `stream`.  Keeps the fastest as the
 * schedule's launch shape and returns it in *best (and its time per call
 * in microseconds in *best_us; either may be NULL).  B_d is overwritten.   */
int race_autotune(race_schedule *s, int32_t k, const double *X_d, double *B_d, int32_t reps, void *stream,
                  race_launch *best, float *best_us);

/* ---- learned RACE-parameter predictor (beyond the paper, which picks the
 * epsilon_s by a parameter study, Sec. 5.1) ------------------------------- */

/* race_features — 16 FP32 features of an upper-triangle CRS (host memory,
 * any column order within a row) describing its rows and its BFS levels
 * from the schedule's root: see csrc/features.cpp for the list.            */
int race_features(const race_csr_upper *a, float *feat16);

/* The predictor is a 16 -> 64 -> 64 -> 3 perceptron (ReLU, linear output)
 * mapping features to (eps_0, eps_1, depth) in scaled units.  Its
 * parameters are one packed FP32 device array of race_mlp_param_count()
 * floats: W1[64][16] b1[64] W2[64][64] b2[64] W3[3][64] b3[3].            */
int32_t race_mlp_param_count(void);
/* floats of activation scratch for a batch (z1, h1, z2, h2, y)             */
int64_t race_mlp_act_size(int32_t batch);
/* floats of backward scratch for a batch                                   */
int64_t race_mlp_work_size(int32_t batch);

/* race_mlp_forward — x_d: batch x 16 features (row-major); act_d: scratch
 * of race_mlp_act_size(batch); y_d (may be NULL): batch x 3 outputs.       */
int race_mlp_forward(const float *params_d, int32_t batch, const float *x_d, float *act_d, float *y_d, void *stream);

/* race_mlp_backward — gradient of L = 1/(2 batch) sum_b sum_k w_k (y_bk -
 * t_bk)^2 after race_mlp_forward on the same act_d.  target_d: batch x 3;
 * out_weight_d: 3 weights w_k; grad_d: packed like the parameters;
 * work_d: race_mlp_work_size(batch) floats; loss_terms_d: batch x 3 terms
 * whose sum is L.                                                          */
int race_mlp_backward(const float *params_d, int32_t batch, const float *x_d, float *act_d, const float *target_d,
                      const float *out_weight_d, float *grad_d, float *work_d, float *loss_terms_d, void *stream);

/* race_mlp_adam — one Adam step (bias-corrected, step >= 1) in place.      */
int race_mlp_adam(float *params_d, const float *grad_d, float *m_d, float *v_d, float lr, float beta1, float beta2,
                  float eps, int32_t step, void *stream);

/* symm_spmv_noalloc — b = A x like symm_spmv, for callers that must not
 * allocate device memory themselves or through this library: for example a
 * plug-in whose host application owns every device allocation, code that
 * runs under a fixed device-memory budget, or a latency-critical loop where
 * cudaMalloc's implicit device synchronisation is not acceptable.  The paper
 * has no counterpart; it is a variant of the streaming SymmSpMV kernel
 * (RACE_EXEC_STREAM_RED) that needs no schedule handle.
 *
 * Arguments (all device pointers owned by the caller): an upper-triangle
 * CRS with n rows and nnz stored entries -- row_ptr_d (n+1, row_ptr[0] = 0,
 * non-decreasing, row_ptr[n] = nnz; checked on the device before anything
 * is computed), col_d and val_d (nnz, FP64), each row's columns in [row, n)
 * (not checked: that would cost a pass over col); any row order the caller
 * chooses (e.g. a schedule's permuted matrix); x_d (n) and b_d (n), not
 * aliasing.  row_ptr_d, col_d and val_d must start at 16-byte boundaries
 * (the kernel stages them with bulk copies; cudaMalloc and torch give 256).
 * b is overwritten; when the call is refused (any error code below but
 * _CUDA and _TIMEOUT) b is left untouched.
 *
 * Scratch: the kernel's row-block table and status word live in a fixed
 * device array of about 3.4 MB that every GPU loading the library holds
 * until the process exits; nothing is allocated per call.  Limits: n at most
 * 16,777,216 and nnz at most 268,435,456 (RACE_ERR_OVERFLOW beyond), no row
 * with more than 512 stored entries (RACE_ERR_UNSUPPORTED).
 *
 * The first call on a device looks up the device address of that array (a
 * one-time set-up per device, with that device current); make that first
 * call before any stream capture.  Every call shares the one array and it
 * keeps the last call's contents, so calls that overlap on the GPU (other
 * streams or threads) race with each other: serialise them.  The call
 * enqueues its work on `stream` and waits for that stream twice (to size the
 * launch and to read the status), so it returns only when b is complete.
 * Errors: RACE_ERR_INVALID (n < 1, nnz < n, NULL, aliasing, misaligned
 * arrays, malformed row_ptr), _OVERFLOW, _UNSUPPORTED, _CUDA, _TIMEOUT; after
 * _CUDA or _TIMEOUT b is undefined.                                        */
int symm_spmv_noalloc(int32_t n, int64_t nnz, const int32_t *row_ptr_d, const int32_t *col_d, const double *val_d,
                      const double *x_d, double *b_d, void *stream);

void race_free(race_schedule *s);
const char *race_strerror(int code);
const char *race_last_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* RACE_GB300_H */
