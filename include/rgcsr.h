/*
 * rgcsr.h -- C ABI of librgcsr: Row-grouped CSR (RgCSR) sparse
 * matrix-vector multiplication on NVIDIA GB300 (sm_103a), after Oberhuber,
 * Suzuki and Vacata, "New Row-grouped CSR format for storing the sparse
 * matrices on GPU with implementation in CUDA".
 *
 * General rules for every entry point
 * -----------------------------------
 *  - Pointers are DEVICE pointers unless the name ends in `_host`.
 *  - The library never allocates device memory.  The caller allocates every
 *    array (sizes come from the *_plan calls or are stated below) and owns
 *    it; scratch space is passed in as `workspace` / `workspace_bytes`.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Calls return after enqueueing unless stated otherwise; the
 *    *_plan calls synchronise `stream` once to return sizes to the host.
 *  - Return value: RGCSR_OK (0) or a negative RGCSR_ERR_* code.  Nothing
 *    traps or asserts on the device.  rgcsr_status_string() names a code.
 *  - Index types: columns and row lengths int32, group offsets int64; CSR
 *    row pointers may be int32 or int64.  Rows and columns < 2^31.
 *  - Value types: RGCSR_F64 and RGCSR_F32 (x and y have the same type), and
 *    the reduced-storage RGCSR_BF16 / RGCSR_F16 (x and y are float).
 *  - Every SpMV overwrites y (y = A x, not y += A x), as the paper's
 *    kernels do.  Empty rows give +0.  n_rows == 0 is a no-op.
 */
#ifndef RGCSR_H
#define RGCSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rgcsr_stream_t;   /* identical to cudaStream_t */

/* status codes */
#define RGCSR_OK                     0
#define RGCSR_ERR_INVALID_ARG       -1   /* NULL pointer, bad size or option   */
#define RGCSR_ERR_BAD_ROWPTR        -2   /* row_ptr[0] != 0, decreasing, or row_ptr[n] != nnz */
#define RGCSR_ERR_COL_OOB           -3   /* a column index outside [0, n_cols) */
#define RGCSR_ERR_INDEX_OVERFLOW    -4   /* a size exceeds its index type      */
#define RGCSR_ERR_UNSUPPORTED_DTYPE -5   /* value type not valid for this call */
#define RGCSR_ERR_CUDA              -6   /* a CUDA runtime call failed         */
#define RGCSR_ERR_WORKSPACE         -7   /* workspace missing or too small     */
#define RGCSR_ERR_BAD_PERM          -8   /* row_perm not a permutation of [0, n_rows) */
#define RGCSR_ERR_CORRUPT           -9   /* an RgCSR matrix fails rgcsr_check_matrix */
#define RGCSR_ERR_TIMEOUT          -10   /* a bounded device wait gave up (results invalid) */

/* element types */
#define RGCSR_F64  0
#define RGCSR_F32  1
#define RGCSR_BF16 2
#define RGCSR_F16  3
#define RGCSR_I32  4
#define RGCSR_I64  5

/* A CSR matrix (Sec. 3.1): row r holds entries row_ptr[r] .. row_ptr[r+1]-1
 * of col_idx/values.  Column order inside a row is kept as given (the paper
 * assumes ascending columns); duplicates and explicit zeros are entries. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    const void *row_ptr;        /* n_rows+1 entries of row_ptr_type          */
    int32_t row_ptr_type;       /* RGCSR_I32 or RGCSR_I64                    */
    int32_t value_type;         /* RGCSR_F64 or RGCSR_F32                    */
    const int32_t *col_idx;     /* nnz                                       */
    const void *values;         /* nnz of value_type                         */
} rgcsr_csr;

/* An RgCSR matrix (Sec. 3.4).  Rows are cut into groups of G consecutive
 * rows; group g has R_g = min(G, n_rows - g*G) rows and K_g = the longest
 * row length in it.  Slot j of row r = g*G + t is stored at
 *     group_ptr[g] + j*R_g + t        (0 <= j < K_g),
 * so the j-th entries of a group's rows are contiguous.  Slots past a row's
 * length are padding ("artificial zeros"): value bits 0, column 0; kernels
 * never multiply them because row_lengths bounds every row's loop. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    int32_t group_size;         /* G >= 1 (set by the caller before plan)    */
    int32_t value_type;         /* storage type of `values`                  */
    int64_t n_groups;           /* ceil(n_rows / G)                  (plan) */
    int64_t n_stored;           /* group_ptr[n_groups] = nnz + padding (plan) */
    int64_t max_row_len;        /*                                   (plan) */
    void *values;               /* n_stored elements of value_type           */
    int32_t *columns;           /* n_stored                                  */
    int64_t *group_ptr;         /* n_groups + 1 ("groupPointers")            */
    int32_t *row_lengths;       /* n_rows       ("rowLengths")               */
    float *row_scale;           /* n_rows; BF16/F16 storage only, else NULL  */
    int64_t *slot_to_csr;       /* optional n_stored: CSR position per slot, -1 = padding */
    int32_t *row_perm;          /* optional n_rows row order (Sec. 4.4.2, Table 7): stored row k
                                   is CSR row row_perm[k], so groups are formed over the
                                   reordered rows; NULL = identity.  Set before rgcsr_plan,
                                   which checks that it is a permutation.  x, y, X and Y
                                   stay in the CSR's own row order: kernels write row k's
                                   result to y[row_perm[k]].  row_lengths, row_scale and
                                   the slabs are in stored order; slot_to_csr holds
                                   positions in the CSR as given.                    */
} rgcsr_matrix;

/* Kernel selection for rgcsr_spmv_ex (autotuning and ablations). */
#define RGCSR_KERNEL_AUTO   0    /* default: when the groups are dense (padding <=
                                    25% of the stored slots, no row longer than 64
                                    and 8x the mean) and rows are short (<= 8 per
                                    row on average) at G = 32, the LEAN vector-load
                                    variant 1 (FP64: 4); dense FP32 with longer
                                    rows, the TMA kernel, variant 2; other dense
                                    matrices, the LEAN kernel; otherwise the
                                    warp-split kernel                               */
#define RGCSR_KERNEL_PAPER  1    /* one block per group, one thread per row (Sec. 3.4 listing) */
#define RGCSR_KERNEL_SPLIT  2    /* one thread per row; long rows of a warp finished
                                    by the whole warp with a shuffle reduction      */
#define RGCSR_KERNEL_TMA    3    /* G == 32 only: group slabs staged in shared memory by
                                    bulk copies (cp.async.bulk) into a ring per warp,
                                    persistent grid; needs 16-byte aligned values,
                                    columns and row_lengths and n_rows >= 32.
                                    Variants 0-3 (F64/F32): one group (or a piece
                                    of one) per copy; 4-6 (every value type):
                                    several whole groups per copy while they fit  */
#define RGCSR_KERNEL_LEAN   4    /* one thread per row, no long-row split, sized for
                                    full occupancy (rows of similar lengths)        */
#define RGCSR_KERNEL_SELL   5    /* comparator, not the method: sliced ELLPACK on the
                                    same slabs (Sec. 3.4) -- every row runs all K_g
                                    slots of its group, padding multiplied          */
#define RGCSR_XLOAD_NC      0    /* x through the read-only (non-coherent) path    */
#define RGCSR_XLOAD_PLAIN   1    /* x with ordinary global loads                   */
#define RGCSR_XLOAD_TEX     2    /* x by texture fetches from a texture object over
                                    x (the paper's texture binding, Sec. 3.4, 4.3);
                                    the library creates one per x buffer on first
                                    use and keeps it (at most 64 per device: the
                                    65th clears the cache after a device
                                    synchronisation).  PLAIN and TEX need an
                                    explicit PAPER, SPLIT or LEAN (variant 0)
                                    kernel; x up to the device's 1D linear texture
                                    width (RGCSR_ERR_INVALID_ARG beyond)           */
typedef struct {
    int32_t kernel;             /* RGCSR_KERNEL_*                                  */
    int32_t block_threads;      /* 0 = default (256); multiple of 32, <= 256       */
    int32_t x_load;             /* RGCSR_XLOAD_*                                   */
    int32_t split_weight;       /* 0 = default; cost of one warp-cooperative step
                                   relative to one thread-per-row step, x 4        */
    int32_t variant;            /* configuration of the chosen kernel, 0 = default:
                                   TMA: 0..3 = (slot-rows per chunk, ring stages)
                                   (8,2), (8,4), (16,2), (4,4); 4..6 = chunks of
                                   whole consecutive groups (up to 16) while they
                                   fit: (32,2), (32,3), (16,4), four warps per
                                   CTA; LEAN: 1, 2, 4 =
                                   G = 32 with vector loads: a lane owns 4 rows
                                   (F64: 2) of a group, 2 slot-rows in flight
                                   (1), or 2 rows, 4 slot-rows in flight (2), or
                                   4 rows (F64: 2), 4 slot-rows in flight (4);
                                   5, 6, 7 = the same software-pipelined (the
                                   next slot-rows' loads issued before the
                                   current x gathers) with 16-byte value loads
                                   (a lane owns 16 / value size rows: F64 2,
                                   F32 4, BF16/F16 8), 2, 1 or 4 slot-rows per
                                   stage; 8 = as 1 with 8 slot-rows in flight
                                   (a short row's whole slab at once); 9 =
                                   BF16/FP16 storage only: as 1 with six
                                   blocks per SM;
                                   16-byte aligned values and columns; other
                                   kernels: 0                                     */
    int32_t wait_limit;         /* TMA kernel: non-blocking probes of a stage's
                                   mbarrier before a wait gives up, 0 = default
                                   (2^26, about a second).  A wait that runs out
                                   records RGCSR_STATUS_TIMEOUT, lets the warp's
                                   copies in flight finish (default bound), leaves
                                   the rows of its remaining groups unwritten and
                                   ends the warp.  Small values exist to test that
                                   path; other kernels ignore the field.          */
} rgcsr_launch;

/* ----------------------------------------------------------------------- */
/* Conversion CSR -> RgCSR (Sec. 3.4: groups, padding, groupPointers,       */
/* rowLengths).  Two phases so that the caller can allocate:                */
/*   1. rgcsr_plan   -- validates the CSR, writes row_lengths and group_ptr */
/*                      (both caller-allocated: n_rows and ceil(n/G)+1),    */
/*                      sets n_groups, n_stored, max_row_len, nnz, sizes.   */
/*                      Synchronises `stream`.                              */
/*   2. rgcsr_convert -- scatters values/columns (and slot_to_csr if non-   */
/*                      NULL) into caller-allocated n_stored arrays.        */
/*                      M->value_type must equal A->value_type; M is the   */
/*                      descriptor rgcsr_plan filled for A.  Async.          */
/* With M->row_perm set, both phases work on the rows in that order (plan   */
/* returns RGCSR_ERR_BAD_PERM if it is not a permutation of [0, n_rows)).   */
/* ----------------------------------------------------------------------- */
size_t rgcsr_plan_workspace_bytes(int64_t n_rows, int32_t group_size);
int rgcsr_plan(const rgcsr_csr *A, rgcsr_matrix *M, void *workspace,
               size_t workspace_bytes, rgcsr_stream_t stream);
int rgcsr_convert(const rgcsr_csr *A, const rgcsr_matrix *M, rgcsr_stream_t stream);

/* Row ordering (Sec. 4.4.2, Table 7).  The paper's "descending" order sorts
 * rows by their number of non-zeros, largest first, so that each group holds
 * rows of similar length and little padding is needed.
 * rgcsr_descending_order writes row_perm[k] = the CSR row placed at stored
 * position k: row lengths non-increasing in k, rows of equal length in
 * increasing row index (a stable sort, so the order is unique).  row_perm is
 * a caller-allocated device int32[n_rows]; the workspace (device, caller-
 * owned) needs rgcsr_row_order_workspace_bytes(n_rows) bytes.  Asynchronous
 * on `stream`.  Lengths are read from A->row_ptr as given; an invalid row_ptr
 * still yields a permutation, which rgcsr_plan then rejects with the CSR.
 * Put the result in M->row_perm before rgcsr_plan. */
size_t rgcsr_row_order_workspace_bytes(int64_t n_rows);
int rgcsr_descending_order(const rgcsr_csr *A, int32_t *row_perm, void *workspace,
                           size_t workspace_bytes, rgcsr_stream_t stream);

/* rgcsr_plan without a workspace argument, for callers that cannot
 * allocate device memory: code that only receives device pointers from
 * another component and has no allocator of its own, or that runs where a
 * cudaMalloc/cudaFree (each of which may synchronise the whole device) is
 * not acceptable, e.g. inside a framework whose caching allocator owns all
 * device memory.  The paper has no counterpart; it is an interface variant.
 *
 * Same inputs, outputs, validation and stream synchronisation as
 * rgcsr_plan.  The scratch is one fixed array of RGCSR_PLAN_NOALLOC_SCRATCH_BYTES
 * inside the library, present on every GPU that loads the library until the
 * process exits; the call allocates nothing.  It serves matrices whose
 * rgcsr_plan_workspace_bytes(n_rows, group_size) fits in that array (up to
 * 16,709,631 groups, i.e. about 534 million rows at G = 32); larger ones
 * return RGCSR_ERR_WORKSPACE without touching the device.
 * Every call looks up the array's device address on the current device
 * (nothing is cached, so a device reset does not leave a stale address).
 * All calls share the one array: calls whose GPU work overlaps (several
 * host threads or streams at once) race on it and must be serialised. */
#define RGCSR_PLAN_NOALLOC_SCRATCH_BYTES 65536
int rgcsr_plan_noalloc(const rgcsr_csr *A, rgcsr_matrix *M, rgcsr_stream_t stream);

/* ----------------------------------------------------------------------- */
/* SpMV y = A x on an RgCSR matrix (Sec. 3.4 kernel; peak model of the     */
/* same section).  x: n_cols elements, y: n_rows elements; F64 storage     */
/* takes double x/y, every other storage float x/y.  x and y must not      */
/* overlap.  Async.                                                        */
/* ----------------------------------------------------------------------- */
int rgcsr_spmv(const rgcsr_matrix *M, const void *x, void *y, rgcsr_stream_t stream);
int rgcsr_spmv_ex(const rgcsr_matrix *M, const void *x, void *y,
                  const rgcsr_launch *launch, rgcsr_stream_t stream);
/* The kernel and variant that RGCSR_KERNEL_AUTO (and so rgcsr_spmv) runs
 * for M, by the rule given at RGCSR_KERNEL_AUTO.  Host only: reads M's
 * fields, not its arrays (whose addresses decide the 16-byte alignment
 * condition).  RGCSR_ERR_INVALID_ARG for a malformed descriptor. */
int rgcsr_auto_kernel(const rgcsr_matrix *M, int32_t *kernel, int32_t *variant);

/* x staged in shared memory (the x read-path study of Sec. 4.3, not the
 * paper's kernel).  For every block of RGCSR_XWINDOW_ROWS consecutive stored
 * rows, rgcsr_xwindow_plan finds the columns the block's stored entries use
 * (padding excluded), sorts them and cuts them into ranges wherever two
 * consecutive used columns lie more than RGCSR_XWINDOW_GAP apart; a block
 * with at most RGCSR_XWINDOW_MAX_RANGES ranges of at most
 * RGCSR_XWINDOW_CAP_BYTES of x in all (x elements are 8 bytes for F64
 * storage, else 4) is "staged", any other block (or one with more than 8,192
 * stored entries) gets n_ranges = 0.  rgcsr_spmv_xwindow computes y = A x with
 * one thread per stored row; a staged block first copies its ranges of x into
 * shared memory and gathers from there, the others read x through the
 * read-only path.  A 3D 7-point stencil's block of 256 rows touches three
 * bands of x (1,024 elements), a banded matrix one.
 *   windows: caller-allocated device array of rgcsr_xwindow_count(n_rows)
 *   records, filled by rgcsr_xwindow_plan (async) and valid for M's pattern.
 *   Every value type.  Async. */
#define RGCSR_XWINDOW_ROWS        256
#define RGCSR_XWINDOW_MAX_RANGES  4
#define RGCSR_XWINDOW_GAP         64
#define RGCSR_XWINDOW_CAP_BYTES   32768
typedef struct {
    int32_t n_ranges;           /* 0 = not staged                             */
    int32_t total;              /* staged elements, sum of len                */
    int32_t lo[RGCSR_XWINDOW_MAX_RANGES];    /* first column of each range    */
    int32_t len[RGCSR_XWINDOW_MAX_RANGES];   /* columns in each range         */
} rgcsr_xwindow;
int64_t rgcsr_xwindow_count(int64_t n_rows);
int rgcsr_xwindow_plan(const rgcsr_matrix *M, rgcsr_xwindow *windows, rgcsr_stream_t stream);
int rgcsr_spmv_xwindow(const rgcsr_matrix *M, const rgcsr_xwindow *windows, const void *x, void *y,
                       rgcsr_stream_t stream);

/* Long-row segments, for matrices whose row lengths vary wildly (the
 * paper's weak point, Sec. 4.4.2: one very long row makes its whole group
 * wait).  The slots j >= threshold of every longer row are cut into
 * segments of `segment` slots; one warp sums each segment, and the last
 * segment of a row to finish (a counter in `arrivals`, no waiting) adds the
 * row's partials in a fixed order (lane l of its warp takes partials l,
 * l + 32, ..., then a fixed shuffle tree), so the result does not depend on
 * scheduling; the remaining slots of every row go through the warp-split
 * kernel, one launch earlier.  The
 * RgCSR format itself is unchanged; the segment lists are a launch schedule.
 *   1. set threshold and segment, call rgcsr_long_rows_plan (sets
 *      n_segments, n_long_rows; synchronises `stream`);
 *   2. allocate seg_row, seg_start (n_segments int32), long_row,
 *      long_first, long_count (n_long_rows int32), arrivals (n_segments
 *      int32) and partials (n_segments doubles for F64 storage, floats
 *      otherwise; scratch of the SpMV);
 *   3. rgcsr_long_rows_build fills the lists and zeroes arrivals (async);
 *   4. rgcsr_spmv_long_rows computes y = A x (two launches, async).  One
 *      SpMV per schedule may be in flight at a time: arrivals and partials
 *      are its scratch, and every counter is back at 0 when it ends.      */
typedef struct {
    int32_t threshold;          /* T >= 0                                     */
    int32_t segment;            /* S >= 1 slots per segment                   */
    int64_t n_segments;         /* (plan)                                     */
    int64_t n_long_rows;        /* (plan) rows longer than T                  */
    int32_t *seg_row, *seg_start;
    int32_t *long_row, *long_first, *long_count;
    void *partials;
    int32_t *arrivals;          /* n_segments; a row's counter sits at its
                                   first segment                              */
} rgcsr_long_rows;
size_t rgcsr_long_rows_workspace_bytes(int64_t n_rows);
int rgcsr_long_rows_plan(const rgcsr_matrix *M, rgcsr_long_rows *S, void *workspace,
                         size_t workspace_bytes, rgcsr_stream_t stream);
int rgcsr_long_rows_build(const rgcsr_matrix *M, const rgcsr_long_rows *S, void *workspace,
                          size_t workspace_bytes, rgcsr_stream_t stream);
int rgcsr_spmv_long_rows(const rgcsr_matrix *M, const rgcsr_long_rows *S, const void *x, void *y,
                         rgcsr_stream_t stream);

/* Group tiles, a launch schedule for G <= 32 (one warp per task, lane t
 * on row t of the group, so every load of a value or column slab is
 * coalesced).  A group whose longest row K_g exceeds `tile` slot-rows is cut
 * into ceil(K_g / tile) tasks of at most `tile` slot-rows each; tasks of
 * one group write per-row partial sums, and the last of them to finish
 * (an arrival counter per group, no waiting) adds the partials in a fixed
 * order (task q into sum q mod NS, NS = 8 for F32 storage and 4 for the
 * others, then a fixed tree) and writes y, so the result does not depend
 * on scheduling.  With rows in descending length order (row_perm, Sec.
 * 4.4.2) the groups are dense and every warp's work is bounded by `tile`
 * slot-rows, which removes the long-row imbalance that the paper names as
 * the format's weak point.
 *   1. set tile, call rgcsr_tiles_plan (sets n_extra, n_split, n_partials;
 *      synchronises `stream`);
 *   2. allocate first_extra, part_base (n_groups+1 int64), extra_group
 *      (n_extra int32), arrivals (n_groups int32) and partials
 *      (n_partials * 32 elements: double for F64 storage, float otherwise);
 *   3. rgcsr_tiles_build fills them and zeroes `arrivals` (async);
 *   4. rgcsr_spmv_tiles computes y = A x in one launch (async).  Tasks
 *      0 .. n_groups-1 are the first tile of every group; task n_groups + e
 *      is extra tile e, of group extra_group[e].  One SpMV per schedule may
 *      be in flight at a time (partials and arrivals are its scratch; each
 *      group's counter is back at 0 when the launch ends).
 * RGCSR_ERR_INVALID_ARG if G > 32 or tile < 1. */
typedef struct {
    int32_t tile;               /* slot-rows per task, >= 1                   */
    int32_t variant;            /* 0 = default; 1, 2: fewer / more slot-rows
                                   in flight per lane; 3, 4, 5: software-
                                   pipelined across a warp's tiles, 5 with
                                   twice the slot-rows per step; 6, 7: each
                                   step's columns loaded one step ahead
                                   (tuning)                                   */
    int64_t n_groups;           /* (plan) the matrix's group count            */
    int64_t n_extra;            /* (plan) tasks beyond one per group          */
    int64_t n_split;            /* (plan) groups cut into more than one task  */
    int64_t n_partials;         /* (plan) tasks of split groups               */
    int64_t *first_extra;       /* n_groups+1: extra tasks of g are
                                   first_extra[g] .. first_extra[g+1]-1      */
    int64_t *part_base;         /* n_groups+1: partial slot of g's first task */
    int32_t *extra_group;       /* n_extra                                    */
    int32_t *arrivals;          /* n_groups                                   */
    void *partials;             /* n_partials * 32                            */
} rgcsr_tiles;
size_t rgcsr_tiles_workspace_bytes(int64_t n_groups);
int rgcsr_tiles_plan(const rgcsr_matrix *M, rgcsr_tiles *T, void *workspace,
                     size_t workspace_bytes, rgcsr_stream_t stream);
int rgcsr_tiles_build(const rgcsr_matrix *M, const rgcsr_tiles *T, rgcsr_stream_t stream);
int rgcsr_spmv_tiles(const rgcsr_matrix *M, const rgcsr_tiles *T, const void *x, void *y,
                     rgcsr_stream_t stream);

/* The same SpMV from and to HOST memory: copies x_host (n_cols elements) to
 * the caller's device buffer x_dev, computes y_dev = A x_dev -- with the
 * group-tile schedule if tiles is not NULL, else the long-row schedule if
 * long_rows is not NULL, else rgcsr_spmv_ex with `launch` (NULL = default)
 * -- and copies y_dev to y_host (n_rows elements), all on `stream`.  Pinned
 * host buffers make the copies asynchronous; the caller synchronises before
 * reading y_host. */
int rgcsr_spmv_host(const rgcsr_matrix *M, const void *x_host, void *y_host,
                    void *x_dev, void *y_dev, const rgcsr_launch *launch,
                    const rgcsr_long_rows *long_rows, const rgcsr_tiles *tiles,
                    rgcsr_stream_t stream);

/* Y = A X for k right-hand sides (the SpMV of Sec. 3.4 applied to several
 * vectors at once; not in the paper).  X: row-major [n_cols x k] with row
 * stride ldx >= k elements; Y: row-major [n_rows x k], stride ldy >= k,
 * overwritten.  Element types as for rgcsr_spmv.  The matrix is streamed
 * once per chunk of up to 32 columns (16 for F64).  Async. */
int rgcsr_spmm(const rgcsr_matrix *M, int32_t k, const void *X, int64_t ldx, void *Y,
               int64_t ldy, rgcsr_stream_t stream);

/* Y = A X with a few lanes per row, for matrices whose rows vary in length.
 * A sub-warp of S lanes owns a row; lane q holds 4 consecutive columns of
 * its result (chunks of 32, 16, 8, 4 columns use S = 8, 4, 2, 1, then single
 * columns), so one non-zero costs one contiguous 16*S-byte read of X.  With
 * long_rows (a schedule built by rgcsr_long_rows_plan/build for M; NULL =
 * none) the slots >= threshold of longer rows go to per-segment partial sums
 * that a last pass adds in order (deterministic).  partials: device scratch
 * of partials_count >= n_segments * min(k, 32) elements (double for F64
 * storage, float otherwise); unused without segments.  X, Y, ldx, ldy and
 * element types as for rgcsr_spmm; 16-byte aligned X and Y with ldx, ldy
 * multiples of 16 bytes enable vector loads.  k = 1 with ldx = ldy = 1 runs
 * the SpMV (rgcsr_spmv_long_rows, or rgcsr_spmv without a schedule).  Async.
 * RGCSR_ERR_WORKSPACE if partials is too small. */
int rgcsr_spmm_long_rows(const rgcsr_matrix *M, const rgcsr_long_rows *long_rows, int32_t k,
                         const void *X, int64_t ldx, void *Y, int64_t ldy, void *partials,
                         int64_t partials_count, rgcsr_stream_t stream);

/* Y = A X on the group-tile schedule T of M (rgcsr_tiles_plan/build; G <=
 * 32): lane t of a warp owns row t of a tile and KC consecutive columns of
 * its result (chunks of 8, 4, then 1 columns), so value/column loads are
 * coalesced slot-rows and each non-zero reads one KC-wide piece of X.  Tiles
 * of a split group add their KC partial sums per row in tile order (the last
 * to arrive writes Y).  partials: device scratch of partials_count >=
 * T->n_partials * 32 * min(k, 8) elements (double for F64 storage, float
 * otherwise); unused without split groups.  X, Y, ldx, ldy and element types
 * as for rgcsr_spmm; k = 1 with ldx = ldy = 1 runs rgcsr_spmv_tiles.  One
 * product per schedule in flight at a time.  Async.  RGCSR_ERR_WORKSPACE if
 * partials is too small. */
int rgcsr_spmm_tiles(const rgcsr_matrix *M, const rgcsr_tiles *tiles, int32_t k, const void *X,
                     int64_t ldx, void *Y, int64_t ldy, void *partials, int64_t partials_count,
                     rgcsr_stream_t stream);

/* ----------------------------------------------------------------------- */
/* Batched SpMV: many RgCSR matrices of uneven sizes in one launch (not in  */
/* the paper).  The members' arrays are concatenated; member m uses         */
/*   values/columns from val_off, row_lengths/row_scale/y from row_off,     */
/*   its own group pointers (n_groups+1 entries starting at 0) from         */
/*   group_off, x from x_off,                                               */
/* and its own group size.  All members share one value type.              */
/* ----------------------------------------------------------------------- */
typedef struct {
    int64_t n_rows, n_cols;
    int64_t val_off, row_off, group_off, x_off;
    int32_t group_size;
    int32_t reserved;
} rgcsr_batch_desc;

typedef struct {
    int32_t n_matrices;
    int32_t value_type;             /* as in rgcsr_matrix                     */
    int64_t n_tasks;                /* from rgcsr_batch_tasks                  */
    const rgcsr_batch_desc *desc;   /* device [n_matrices]                     */
    const int32_t *tasks;           /* device [2 * n_tasks]: (member, first row) */
    const void *values;             /* concatenated slabs                      */
    const int32_t *columns;
    const int64_t *group_ptr;
    const int32_t *row_lengths;
    const float *row_scale;         /* BF16/F16 storage only                   */
} rgcsr_batch;

/* HOST function: cuts every member into blocks of 32 rows and writes one
 * (member, first row) pair per block into the host array `tasks` (capacity
 * pairs; NULL to count only).  *n_tasks receives the number of pairs. */
int rgcsr_batch_tasks(const rgcsr_batch_desc *desc, int32_t n_matrices, int32_t *tasks,
                      int64_t capacity, int64_t *n_tasks);
/* y_m = A_m x_m for every member, one persistent launch; no host sync and
 * no allocation, so it may be captured in a CUDA graph.  Async. */
int rgcsr_spmv_batched(const rgcsr_batch *B, const void *x, void *y, rgcsr_stream_t stream);

/* ----------------------------------------------------------------------- */
/* Reduced-precision value storage (not in the paper, which stores single  */
/* or double precision).  Per row i the scale is                            */
/*   s_i = 2^ceil(log2 max_j |a_ij|)  (1 for an empty or all-zero row,     */
/*         exponent clamped to the binary32 normal range [-126, 127]),      */
/* and each stored value becomes q_ij = round-to-nearest-even(a_ij / s_i)  */
/* in bfloat16 (RGCSR_BF16) or IEEE binary16 (RGCSR_F16), computed from the */
/* exact double quotient, subnormals kept; padding becomes +0.  The SpMV of */
/* such a matrix computes y_i = s_i * sum_j q_ij x_j in float.              */
/*                                                                          */
/* src: an F64 or F32 matrix.  dst: dst->value_type (BF16/F16), dst->values */
/* (n_stored 2-byte elements) and dst->row_scale (n_rows floats) allocated  */
/* by the caller; dst->columns, group_ptr and row_lengths normally point to */
/* src's arrays.  The size fields and row_perm of dst are copied from src */
/* (row_scale is in stored row order).  Async.                              */
/* ----------------------------------------------------------------------- */
int rgcsr_quantize(const rgcsr_matrix *src, rgcsr_matrix *dst, rgcsr_stream_t stream);

/* ----------------------------------------------------------------------- */
/* Backward pass of Y = A X (not in the paper).  With an upstream gradient  */
/* dY:  dX = A^T dY  (an SpMM with an RgCSR matrix of A^T, built once from  */
/* the CSR transpose below) and  dA_p = sum_b dY[row_p, b] X[col_p, b]      */
/* for every stored entry p (rgcsr_sampled_dot).                            */
/* ----------------------------------------------------------------------- */
/* Workspace of rgcsr_csr_transpose (about 20 bytes per stored entry). */
size_t rgcsr_transpose_workspace_bytes(int64_t nnz, int64_t n_rows, int64_t n_cols);
/* CSR of A^T by a stable radix sort of the entries by column: t_row_ptr
 * (n_cols+1), t_col_idx (nnz; the original row of each entry, increasing
 * within every transposed row), perm (nnz, optional: the original CSR
 * position of each transposed entry) and t_values (nnz of A's value type,
 * optional: values[perm]).  Needs nnz < 2^32.  Async. */
int rgcsr_csr_transpose(const rgcsr_csr *A, int64_t *t_row_ptr, int32_t *t_col_idx, int64_t *perm,
                        void *t_values, void *workspace, size_t workspace_bytes,
                        rgcsr_stream_t stream);
/* row_index[p] = the row of stored entry p (nnz int32).  Async. */
int rgcsr_csr_row_index(const rgcsr_csr *A, int32_t *row_index, rgcsr_stream_t stream);
/* M->values[s] = src[src_index[s]], or 0 where src_index[s] < 0 (padding);
 * src has M's value type (F64/F32).  Refreshes an RgCSR matrix from values
 * kept in CSR order, e.g. with src_index = M->slot_to_csr.  Async. */
int rgcsr_gather_values(const rgcsr_matrix *M, const void *src, const int64_t *src_index,
                        rgcsr_stream_t stream);
/* rgcsr_gather_values, skipped when M already holds these values: `state`
 * is a caller-allocated device record of RGCSR_VALUES_STATE_BYTES bytes
 * (8-byte aligned), zero-filled before its first use ("holds nothing"),
 * one per matrix.  The call hashes src[0, n_src) -- a 64-bit sum, over the
 * 8-byte words of src's bytes, of a bijective mix (the SplitMix64
 * finalizer) of each word combined with its position, so any single changed
 * element changes the hash -- compares the hash with the one the record
 * holds, stores the new one, and gathers only if they differ or the record
 * held nothing; the decision is taken on the device (two launches, no host
 * synchronisation).  Several elements changed at once leave the hash
 * unchanged only by chance (about 2^-64); zero the record to force a
 * refresh.  One call per record in flight.  F64 or F32.  Async. */
#define RGCSR_VALUES_STATE_BYTES 16384
int rgcsr_gather_values_if_changed(const rgcsr_matrix *M, const void *src, int64_t n_src,
                                   const int64_t *src_index, void *state, rgcsr_stream_t stream);
/* out[s] = inner[outer[s]], or -1 where outer[s] < 0 (n entries).  Async. */
int rgcsr_compose_index(const int64_t *outer, const int64_t *inner, int64_t n, int64_t *out,
                        rgcsr_stream_t stream);
/* out[p] = sum_{b<k} G[row_index[p]*ldg + b] * X[col_idx[p]*ldx + b] for
 * p < nnz, summed in increasing b; value_type F64 or F32.  Async. */
int rgcsr_sampled_dot(int64_t nnz, int32_t k, const int32_t *row_index, const int32_t *col_idx,
                      const void *G, int64_t ldg, const void *X, int64_t ldx, void *out,
                      int32_t value_type, rgcsr_stream_t stream);
/* The same value gradient read straight from an RgCSR matrix of A:
 * dval[slot_to_csr[s]] = sum_{b<k} G[r_s*ldg + b] * X[columns[s]*ldx + b]
 * for every stored slot s that holds an entry (padding, slot_to_csr < 0, is
 * skipped), r_s being the slot's CSR row (through row_perm if set); dval is
 * in the CSR's entry order (nnz elements of M's value type, F64 or F32).
 * Needs M->slot_to_csr.  Async. */
int rgcsr_spmv_bwd_values(const rgcsr_matrix *M, int32_t k, const void *G, int64_t ldg, const void *X,
                          int64_t ldx, void *dval, rgcsr_stream_t stream);

/* ----------------------------------------------------------------------- */
/* Vector kernels and solvers around the SpMV (Sec. 1: a Krylov iteration   */
/* is SpMV + SAXPY + SDOT).  value_type RGCSR_F64 (double vectors) or       */
/* RGCSR_F32 (float vectors).  All async unless stated.                     */
/* ----------------------------------------------------------------------- */
/* Scratch of rgcsr_dot, in bytes. */
size_t rgcsr_dot_workspace_bytes(void);
/* *result (a DEVICE double) = sum_i x_i y_i in a fixed order
 * (deterministic): double vectors accumulate in double; float vectors use
 * the compensated dot product Dot2 of Ogita, Rump and Oishi (2005) in float
 * per thread, as accurate as twice float precision, then sum in double. */
int rgcsr_dot(int64_t n, const void *x, const void *y, double *result, void *workspace,
              size_t workspace_bytes, int32_t value_type, rgcsr_stream_t stream);
/* y = alpha x + beta y. */
int rgcsr_axpby(int64_t n, double alpha, const void *x, double beta, void *y, int32_t value_type,
                rgcsr_stream_t stream);
/* Damped Jacobi update x_out = x + omega * dinv .* (b - Ax). */
int rgcsr_jacobi_step(int64_t n, double omega, const void *dinv, const void *b, const void *Ax,
                      const void *x, void *x_out, int32_t value_type, rgcsr_stream_t stream);
/* out = alpha * d .* x. */
int rgcsr_diag_scale(int64_t n, double alpha, const void *d, const void *x, void *out,
                     int32_t value_type, rgcsr_stream_t stream);
/* dst = src converted between RGCSR_F64 and RGCSR_F32 (round to nearest). */
int rgcsr_convert_vector(int64_t n, const void *src, int32_t src_type, void *dst, int32_t dst_type,
                         rgcsr_stream_t stream);
/* Reads `bytes` bytes at data (device, 16-byte aligned, bytes a multiple of
 * 16) with 16-byte streaming loads on 8 CTAs of 256 threads per SM, and
 * writes nothing (sink, one device float, is written only if the float sum
 * of the data is exactly -1234567).  Not part of the method: it measures
 * what a plain read of a given size reaches on this GPU, the reference for
 * a memory-bound kernel that moves the same bytes.  RGCSR_ERR_INVALID_ARG
 * for an unaligned pointer or size. */
int rgcsr_stream_read(const void *data, int64_t bytes, void *sink, rgcsr_stream_t stream);
/* Random-gather ceiling: *loads (host int64, written before the launch) =
 * SMs x 1024 threads x 4 x iters random 8-byte loads of x[0, n) (device
 * doubles, n a power of two, 32 <= n <= 2^32), indices from a per-thread
 * xorshift generator, four loads in flight per thread; writes nothing (sink,
 * one device double, is written only if the loads sum to exactly -1234567).
 * Not part of the method: with x resident in L2 it measures how many
 * scattered x gathers per second the SMs can issue, the ceiling of an SpMV
 * whose columns have no locality.  RGCSR_ERR_INVALID_ARG for a bad n or
 * iters < 1. */
int rgcsr_gather_probe(const void *x, int64_t n, int32_t iters, void *sink, int64_t *loads,
                       rgcsr_stream_t stream);
/* Runs *fmas (host int64, written before the launch) = SMs x 2048 threads x
 * 8 independent chains x iters double-precision FMAs, and writes nothing
 * (sink, one device double, is written only if the chains end at exactly
 * -1234567).  Not part of the method: it measures the FP64 FMA rate, the
 * arithmetic ceiling of an FP64 SpMV (one FMA per non-zero).
 * RGCSR_ERR_INVALID_ARG if iters < 1 or a pointer is NULL. */
int rgcsr_fp64_fma_probe(int32_t iters, void *sink, int64_t *fmas, rgcsr_stream_t stream);

/* Conjugate gradients for a symmetric positive definite square A, from
 * x = 0, stopping when ||r|| <= rel_tol ||b|| (the recurrence residual,
 * checked on the host every check_every iterations) or after max_iter
 * iterations.  Vectors are double for F64 storage, float otherwise.
 * An iteration is the SpMV q = A d and one cooperative kernel (every block
 * resident) for dq, alpha, x, r, rr', beta and d, with two grid barriers;
 * where a cooperative launch is not possible, three kernels instead.  A
 * barrier wait is bounded (rgcsr_set_wait_limit); one that gives up makes
 * the call return RGCSR_ERR_TIMEOUT at its next check, with x invalid.
 * Writes *iterations and *rel_residual (host); synchronises `stream`. */
size_t rgcsr_cg_workspace_bytes(int64_t n, int32_t value_type);
int rgcsr_cg(const rgcsr_matrix *A, const void *b, void *x, double rel_tol, int32_t max_iter,
             int32_t check_every, void *workspace, size_t workspace_bytes, int32_t *iterations,
             double *rel_residual, rgcsr_stream_t stream);
/* Polls before a grid barrier of rgcsr_cg / rgcsr_ir_cg gives up; 0 restores
 * the default (about a second).  For tests of the timeout path: a barrier
 * whose blocks are all resident ends in microseconds.  RGCSR_ERR_INVALID_ARG
 * if polls < 0. */
int rgcsr_set_wait_limit(int32_t polls);
/* Mixed-precision iterative refinement: outer loop in FP64 (r = b - A_hi x
 * with the F64 matrix A_hi, stop when ||r|| <= outer_tol ||b|| or after
 * max_outer corrections), inner CG in float on A_lo (F32, BF16 or F16
 * storage of the same matrix) to a relative residual of max(inner_tol,
 * outer_tol / (2 ||r|| / ||b||)) -- no further than the outer goal needs --,
 * x += d in FP64.  b, x: double.
 * Writes the number of corrections, the total inner iterations and the
 * final true relative residual (host); synchronises `stream`. */
size_t rgcsr_ir_cg_workspace_bytes(int64_t n);
int rgcsr_ir_cg(const rgcsr_matrix *A_hi, const rgcsr_matrix *A_lo, const double *b, double *x,
                double outer_tol, int32_t max_outer, double inner_tol, int32_t max_inner,
                void *workspace, size_t workspace_bytes, int32_t *outer_iters, int32_t *inner_iters,
                double *rel_residual, rgcsr_stream_t stream);

/* ----------------------------------------------------------------------- */
/* Hybrid ELLPACK + COO (Sec. 3.3), the paper's comparison format.  The ELL */
/* part is column-major, n_rows x ell_width (slot j of row r at j*n_rows+r, */
/* padding: value 0, column -1); entries past a row's first ell_width go to */
/* COO (row, column, value), ordered by row and then by stored order.       */
/* ell_width < 0 in hyb_plan selects it by the byte-cost rule              */
/*   minimise n*K*(sv+si) + 2*nnz_coo(K)*(sv+2*si),  ties -> smaller K.     */
/* ----------------------------------------------------------------------- */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    int32_t value_type;         /* RGCSR_F64 or RGCSR_F32                    */
    int32_t ell_width;          /* K1                                (plan) */
    int64_t nnz_coo;            /*                                   (plan) */
    int64_t max_row_len;        /*                                   (plan) */
    void *ell_val;              /* ell_width * n_rows                        */
    int32_t *ell_col;           /* ell_width * n_rows                        */
    int32_t *coo_row;           /* nnz_coo                                   */
    int32_t *coo_col;           /* nnz_coo                                   */
    void *coo_val;              /* nnz_coo                                   */
} hyb_matrix;

/* Workspace for hyb_plan and hyb_convert (one buffer serves both). */
size_t hyb_workspace_bytes(int64_t n_rows, int64_t n_cols);
/* Validates the CSR, picks ell_width (if < 0) and counts nnz_coo.  Sets the
 * size fields of H; synchronises `stream`.  Rows longer than n_cols + 1
 * (only possible with duplicate columns) give RGCSR_ERR_INVALID_ARG. */
int hyb_plan(const rgcsr_csr *A, int32_t ell_width, hyb_matrix *H, void *workspace,
             size_t workspace_bytes, rgcsr_stream_t stream);
/* Fills the caller-allocated ELL and COO arrays.  Async. */
int hyb_convert(const rgcsr_csr *A, const hyb_matrix *H, void *workspace,
                size_t workspace_bytes, rgcsr_stream_t stream);
/* y = A x: the ELL step writes y, the COO step adds the overflow.  Rows whose
 * COO entries span several warps' tiles are combined with atomic adds, so
 * their last bits may differ between runs.  Async. */
int hyb_spmv(const hyb_matrix *H, const void *x, void *y, rgcsr_stream_t stream);
/* Y = A X for k right-hand sides: X row-major [n_cols x k] with row stride
 * ldx >= k, Y row-major [n_rows x k] with stride ldy >= k, overwritten.  The
 * ELL step writes Y (one thread per row, up to 8 columns per pass; 16-byte
 * X loads when X and ldx are 16-byte aligned), the COO step adds the
 * overflow with one lane per column (up to 32 per pass) and one atomic add
 * per row run and column, so the last bits of rows with COO entries in
 * several runs may differ between calls.  Element types as for hyb_spmv.
 * Async. */
int hyb_spmm(const hyb_matrix *H, int32_t k, const void *X, int64_t ldx, void *Y, int64_t ldy,
             rgcsr_stream_t stream);

/* ----------------------------------------------------------------------- */
/* Structural checks (a stand-in for a device memory checker)               */
/* ----------------------------------------------------------------------- */
/* rgcsr_check_matrix verifies on the device that M's arrays form the layout
 * of Sec. 3.4 (see rgcsr_matrix), so that no kernel can index outside them.
 * Each failed check sets its bit in report->flags:                          */
#define RGCSR_CHECK_GROUP_PTR   1   /* group_ptr[0] != 0, group_ptr[n_groups] != n_stored, or a
                                       group whose slab is not R_g * K_g slots (K_g: its longest row) */
#define RGCSR_CHECK_ROW_LENGTHS 2   /* a row length < 0 or > max_row_len, or lengths not summing to nnz */
#define RGCSR_CHECK_COLUMN      4   /* a slot inside its row's length with a column outside [0, n_cols) */
#define RGCSR_CHECK_PADDING     8   /* a padding slot (past its row's length) whose value bits or
                                       column are not 0 */
#define RGCSR_CHECK_PERM       16   /* a row_perm entry outside [0, n_rows), or entries that are not a
                                       permutation (a sum of hashed entries: a non-permutation passes
                                       only by a 2^-64 chance) */
#define RGCSR_CHECK_SCALE      32   /* BF16/F16 storage: row_scale NULL, or an entry not finite and > 0 */
#define RGCSR_CHECK_SLOT_MAP   64   /* slot_to_csr (when not NULL): not -1 on a padding slot, or outside
                                       [0, nnz) on a valid one */
typedef struct {
    int32_t flags;              /* RGCSR_CHECK_* bits of the failed checks, 0 = none */
    int32_t reserved;
    int64_t group;              /* lowest group failing RGCSR_CHECK_GROUP_PTR, else -1 */
    int64_t row;                /* lowest stored row failing a length, scale or permutation check, else -1 */
    int64_t slot;               /* lowest slot failing a column, padding or slot-map check, else -1 */
} rgcsr_check_report;
/* Every load of the check stays inside the sizes M declares (n_groups + 1,
 * n_rows, n_stored), whatever the arrays hold.  Returns RGCSR_OK
 * (report->flags == 0), RGCSR_ERR_CORRUPT, or RGCSR_ERR_INVALID_ARG /
 * RGCSR_ERR_UNSUPPORTED_DTYPE for a malformed descriptor.  Synchronises
 * `stream`; calls from several host threads are serialised (the library keeps
 * one device record). */
int rgcsr_check_matrix(const rgcsr_matrix *M, rgcsr_check_report *report, rgcsr_stream_t stream);
/* Checks mode, on with rgcsr_set_checks(1) or RGCSR_CHECKS=1 in the
 * environment when the library loads: every product on an rgcsr_matrix
 * (rgcsr_spmv, rgcsr_spmv_ex, rgcsr_spmv_host, rgcsr_spmv_long_rows,
 * rgcsr_spmv_tiles, rgcsr_spmv_xwindow, rgcsr_spmm, rgcsr_spmm_long_rows,
 * rgcsr_spmm_tiles, rgcsr_spmv_bwd_values, rgcsr_cg, rgcsr_ir_cg) first runs
 * rgcsr_check_matrix on it; if that fails, the product returns
 * RGCSR_ERR_CORRUPT without launching anything and RGCSR_STATUS_CORRUPT joins
 * the status bits.  The check synchronises the stream, so the mode is for
 * debugging; on a stream being captured into a CUDA graph it is skipped.
 * Returns the previous setting. */
int rgcsr_set_checks(int on);

/* ----------------------------------------------------------------------- */
/* Misc                                                                     */
/* ----------------------------------------------------------------------- */
/* Device-side error bits, sticky until read: RGCSR_STATUS_TIMEOUT means a
 * kernel gave up waiting for a bulk copy (after ~1 s) and left some rows of
 * its output unwritten.  rgcsr_get_status copies the bits of the current
 * device to *status_out and clears them; synchronises `stream`. */
#define RGCSR_STATUS_TIMEOUT 1
/* RGCSR_STATUS_CORRUPT: in checks mode (below) a product refused a matrix
 * that failed rgcsr_check_matrix. */
#define RGCSR_STATUS_CORRUPT 2
int rgcsr_get_status(int *status_out, rgcsr_stream_t stream);
const char *rgcsr_status_string(int status);
/* Library version as major*10000 + minor*100 + patch. */
int rgcsr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RGCSR_H */
