/*
 * argcsr.h -- C ABI of the GB300 (sm_103a) Adaptive Row-grouped CSR library.
 *
 * The library implements the method of Heller & Oberhuber, "Adaptive
 * Row-grouped CSR format for storing of sparse matrices on GPU": conversion
 * of a CSR matrix (Section 2) into the ARG-CSR format (Section 3) and the
 * sparse matrix-vector product y = A x on it (Section 4).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers named d_* are device pointers on the current CUDA device,
 *    owned by the caller and borrowed for the duration of the call (or, for
 *    asynchronous calls, until the given stream has passed the call).
 *    Pointers named h_* are host pointers.
 *  - argcsr_stream_t is a CUDA stream handle (it has the same type as
 *    cudaStream_t); NULL means the legacy default stream.  Kernels are
 *    launched on that stream, in stream order.
 *  - Index arrays are int32; the slot offsets of the format are int32 as in
 *    the paper's group descriptor (Listing 1), so a matrix may hold at most
 *    2^31 - 1 slots (ARGCSR_EOVERFLOW otherwise).
 *  - Every call returns a status; nothing aborts the process.  After
 *    ARGCSR_ECUDA, argcsr_last_error_message() describes the CUDA error.
 *  - There is no CPU fallback: every computation runs in this library's
 *    CUDA kernels.
 */
#ifndef ARGCSR_H
#define ARGCSR_H

#include <stdint.h>

#if defined(__GNUC__)
#define ARGCSR_API __attribute__((visibility("default")))
#else
#define ARGCSR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ARGCSR_OK        = 0,
    ARGCSR_EINVAL    = -1,  /* an argument or the CSR input is malformed  */
    ARGCSR_ENOMEM    = -2,  /* device allocation failed                   */
    ARGCSR_ECUDA     = -3,  /* a CUDA runtime call or launch failed       */
    ARGCSR_EOVERFLOW = -4,  /* more than 2^31 - 1 slots would be needed   */
    ARGCSR_ENOTSUP   = -5   /* valid request the library does not support */
} argcsr_status;

/* Element type of the stored values and of x and y. */
typedef enum {
    ARGCSR_F64  = 0,  /* values f64; x, y f64; f64 arithmetic                 */
    ARGCSR_F32  = 1,  /* values f32; x, y f32; f32 arithmetic                 */
    ARGCSR_BF16 = 2   /* values bf16; x, y f32; f32 arithmetic (bf16 storage) */
} argcsr_dtype;

typedef struct CUstream_st *argcsr_stream_t;
typedef struct argcsr_matrix *argcsr_t;
typedef struct argcsr_batch *argcsr_batch_t;
typedef struct argcsr_graph *argcsr_graph_t;

/* Conversion parameters (Section 3).
 *   group_size          G, the number of chunks per group; the paper's
 *                       blockDim.x.  32, 64 or 128.
 *   desired_chunk_size  D >= 1, the paper's desiredChunkSize: a group is
 *                       closed once its nonzeros exceed D * G.
 *   vec_width           V in {1, 2, 4}.  1 is the paper's layout (element j
 *                       of chunk c at offset + j*G + c).  V > 1 rounds the
 *                       chunk size up to a multiple of V and stores element j
 *                       of chunk c at offset + (j/V)*G*V + c*V + j%V, so a
 *                       thread reads V consecutive elements at once.
 *   one_thread_per_row  0: the paper's adaptive step (spare threads of a
 *                       group go to its longest rows, Section 3 step 2).
 *                       1: leave it out -- every row keeps one thread and C
 *                       is the group's longest row, the state the greedy
 *                       starts from.  With D * G above the nonzeros of any
 *                       G consecutive rows every group holds G rows and the
 *                       layout is Sliced ELLPACK / Row-grouped CSR (Section
 *                       2).  For measuring what the adaptive step gains. */
typedef struct {
    int32_t group_size;
    int32_t desired_chunk_size;
    int32_t vec_width;
    int32_t one_thread_per_row;
} argcsr_params;

/* Sizes of a converted matrix. */
typedef struct {
    int32_t n_rows;
    int32_t n_cols;
    int64_t nnz;
    int64_t n_groups;          /* number of argcsrGroupInfo records          */
    int64_t n_slots;           /* S = sum over groups of chunkSize * G       */
    int32_t group_size;
    int32_t desired_chunk_size;
    int32_t vec_width;
    int32_t dtype;             /* argcsr_dtype                               */
    int64_t spmv_bytes;        /* algorithmic bytes of one SpMV: nnz*(value
                                  + 4) + n_cols*x + n_rows*y + 4*n_rows
                                  + 16*n_groups (padding not counted)        */
    int64_t device_bytes;      /* device memory the handle holds             */
    int32_t one_thread_per_row;
    int32_t reserved;
} argcsr_info_t;

/* ---------------------------------------------------------------------------
 * argcsr_create_from_csr -- CSR -> ARG-CSR conversion (Section 3).
 *
 * Input: a CSR matrix (Section 2) of n_rows x n_cols with nnz entries:
 *   d_rowPointers int32[n_rows + 1], d_columns int32[nnz],
 *   d_values      nnz elements of `dtype` (f64, f32 or bf16).
 * The CSR arrays are validated on the device (rowPointers[0] == 0,
 * non-decreasing, rowPointers[n_rows] == nnz, 0 <= columns < n_cols): a
 * malformed input returns ARGCSR_EINVAL and no handle.  Explicit zeros and
 * repeated columns are kept as entries.
 *
 * Steps, all in device kernels on `stream`: grouping of rows (a group is
 * closed after the row that takes its nonzero count above D*G, or before a
 * row would become its (G+1)-th row); per group the chunk size of the greedy
 * thread assignment (the smallest C with sum over rows of max(1, ceil(len/C))
 * <= G, rounded up to a multiple of V); per row the group-local inclusive
 * prefix of its thread count (threadsMapping); group offsets; the chunk-wise
 * copy into the interleaved values/columns arrays, padded with column -1 and
 * value +0.0.
 *
 * The group records are kept on the device in execution order (by chunk
 * size, largest first; see argcsr_device_arrays); argcsr_export returns them
 * in row order.
 *
 * The call synchronises `stream` twice (to size the output and to return the
 * validation status) and returns only when the handle is complete.  The
 * handle owns its device arrays (allocated from a stream-ordered pool owned
 * by this library, or from the caller's allocator, see argcsr_set_allocator)
 * until argcsr_destroy.  *out is set to NULL on error.
 * ------------------------------------------------------------------------ */
ARGCSR_API argcsr_status argcsr_create_from_csr(
    int32_t n_rows, int32_t n_cols, int64_t nnz,
    const int32_t *d_rowPointers, const int32_t *d_columns, const void *d_values,
    argcsr_dtype dtype, const argcsr_params *params,
    argcsr_stream_t stream, argcsr_t *out);

/* argcsr_create_from_csr_as -- the same conversion with the values stored
 * in another type than the input's: in_dtype is the type of d_values,
 * storage_dtype the handle's.  Supported: the same type (a bit copy, as in
 * argcsr_create_from_csr), f64 -> f32, f64 -> bf16 and f32 -> bf16, each
 * rounded to nearest even while the values are copied into their slots;
 * other pairs return ARGCSR_ENOTSUP.  Sections 2 and 3 leave the value type
 * open (the paper's kernels are templated on it). */
ARGCSR_API argcsr_status argcsr_create_from_csr_as(
    int32_t n_rows, int32_t n_cols, int64_t nnz,
    const int32_t *d_rowPointers, const int32_t *d_columns, const void *d_values,
    argcsr_dtype in_dtype, argcsr_dtype storage_dtype, const argcsr_params *params,
    argcsr_stream_t stream, argcsr_t *out);

/* ---------------------------------------------------------------------------
 * argcsr_spmv -- y = A x on ARG-CSR (Section 4).
 *
 * d_x: n_cols elements, d_y: n_rows elements, both f64 for ARGCSR_F64 and
 * f32 otherwise.  x and y must not overlap (ARGCSR_EINVAL).  Every row of y
 * is written, empty rows with 0.  Asynchronous on `stream`; one kernel.
 * For f64 the result equals the CSR sum up to summation order: each chunk
 * is summed in element order with fused multiply-adds, then the partial sums
 * of a row's chunks are added.
 * ------------------------------------------------------------------------ */
ARGCSR_API argcsr_status argcsr_spmv(argcsr_t A, const void *d_x, void *d_y,
                                     argcsr_stream_t stream);

/* argcsr_spmv_axpby -- y = alpha A x + beta y (the SpMV of Section 4 with a
 * scaled update, as iterative solvers use it).  Computed per row in the
 * accumulation type (f64 for ARGCSR_F64, f32 otherwise; alpha and beta are
 * rounded to it) as fma(alpha, s, beta * y) with s the row's product; when
 * beta == 0, y is only written (it may hold anything, NaN included).  Same
 * arguments and errors as argcsr_spmv. */
ARGCSR_API argcsr_status argcsr_spmv_axpby(argcsr_t A, double alpha, const void *d_x, double beta,
                                           void *d_y, argcsr_stream_t stream);

/* ---------------------------------------------------------------------------
 * argcsr_probe_gather -- a roofline probe for measurements; not an operation
 * of the paper.  It makes the memory accesses of argcsr_spmv on A (Section 4:
 * the group records, the padded column and value streams of Listing 1's
 * layout, and one gather of x per stored column) without its arithmetic, so
 * that its duration is the ceiling those accesses alone set.
 *   mode & 3:        0 columns + x gathers; 1 columns + values + x gathers;
 *                    2 columns only (no gathers)
 *   (mode >> 2) & 3: the gather's load instruction: 0 read-only path,
 *                    1 read-only without L1 allocation, 2 L2 only,
 *                    3 default caching load
 * The work is split as the product splits it (G = 32: a warp per group,
 * and for V = 1 groups of chunk size above 64 get a whole block each;
 * G = 64 or 128: G threads per group).  ARGCSR_F64 handles only, and the
 * load instruction choice (mode >> 2) only for G = 32 (ARGCSR_ENOTSUP
 * otherwise);
 * other modes return ARGCSR_EINVAL.  d_x as in argcsr_spmv.  Writes no
 * caller memory.  Asynchronous on `stream`; one kernel.
 * ------------------------------------------------------------------------ */
ARGCSR_API argcsr_status argcsr_probe_gather(argcsr_t A, const void *d_x, int32_t mode,
                                             argcsr_stream_t stream);

/* ---------------------------------------------------------------------------
 * argcsr_set_allocator -- device memory from the caller (for example a
 * framework's caching allocator) instead of the library's stream-ordered
 * pool, for every array the library allocates from then on: handles,
 * conversion scratch, batches, solver and serving workspaces.
 *   alloc(bytes, stream, ctx) returns device memory usable in stream order
 *     on `stream`, 256-byte aligned (ARGCSR_EINVAL otherwise), or NULL
 *     (ARGCSR_ENOMEM);
 *   free(ptr, stream, ctx) gives it back; the library's last use of it is
 *     enqueued on `stream`, and the memory must not be reused before that
 *     stream reaches this point.
 * Both NULL restores the pool.  Only one of them NULL: ARGCSR_EINVAL.  The
 * allocator cannot change while memory it handed out (or the pool's) is
 * still held: ARGCSR_EINVAL.  The callbacks may run on the serving engine's
 * worker thread.  (Not from the paper: an integration point.)
 * ------------------------------------------------------------------------ */
typedef void *(*argcsr_alloc_fn)(size_t bytes, argcsr_stream_t stream, void *ctx);
typedef void (*argcsr_free_fn)(void *ptr, argcsr_stream_t stream, void *ctx);
ARGCSR_API argcsr_status argcsr_set_allocator(argcsr_alloc_fn alloc, argcsr_free_fn free_fn, void *ctx);

/* Sizes and byte counts of a handle (host only, no device work). */
ARGCSR_API argcsr_status argcsr_info(argcsr_t A, argcsr_info_t *out);

/* ---------------------------------------------------------------------------
 * argcsr_export -- copy the format's arrays to host memory (synchronous on
 * the legacy default stream after a device synchronisation).
 *   h_groupInfo       int32[4 * n_groups]: {firstRow, size, offset, chunkSize}
 *                     per group (Listing 1), groups in row order;
 *   h_threadsMapping  int32[n_rows];
 *   h_columns         int32[n_slots];
 *   h_values          n_slots elements of the handle's dtype.
 * Any pointer may be NULL to skip that array.
 * ------------------------------------------------------------------------ */
ARGCSR_API argcsr_status argcsr_export(argcsr_t A, int32_t *h_groupInfo,
                                       int32_t *h_threadsMapping, int32_t *h_columns,
                                       void *h_values);

/* Borrow the handle's device arrays (valid until argcsr_destroy).  Any
 * output pointer may be NULL.  The device copy of groupInfo holds the same
 * records as argcsr_export in execution order -- by chunk size, largest
 * first, so that the product's blocks get groups of equal work -- not in row
 * order; every record names its first row, and sorting by it gives the
 * format's order. */
ARGCSR_API argcsr_status argcsr_device_arrays(argcsr_t A, const int32_t **d_groupInfo,
                                              const int32_t **d_threadsMapping,
                                              const int32_t **d_columns,
                                              const void **d_values);

/* Free the handle's arrays in stream order on `stream` and the handle
 * itself.  NULL-safe.  Work already queued on other streams that reads the
 * handle must be ordered before `stream` by the caller. */
ARGCSR_API argcsr_status argcsr_destroy(argcsr_t A, argcsr_stream_t stream);

/* ---------------------------------------------------------------------------
 * argcsr_spmm -- Y = A X for k right-hand sides (k in {1, 2, 4, 8, 16}).
 * The Section 4 kernel with k multiply-adds per slot: X is n_cols x k and Y
 * is n_rows x k, row-major with leading dimensions ldx, ldy >= k (elements);
 * element type as for argcsr_spmv.  X and Y must not overlap.  16-byte
 * aligned arrays with ld * element size a multiple of 16 use vector loads.
 * Asynchronous on `stream`; one kernel.
 * ------------------------------------------------------------------------ */
ARGCSR_API argcsr_status argcsr_spmm(argcsr_t A, int32_t k, const void *d_X, int64_t ldx,
                                     void *d_Y, int64_t ldy, argcsr_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batches: products of many independent matrices in one persistent launch.
 *
 * argcsr_batch_create borrows `count` handles (they must outlive the batch;
 * all with group_size 32 -- ARGCSR_ENOTSUP otherwise -- and the same dtype
 * and vec_width).  Right-hand sides and results are packed in matrix order:
 * matrix i's X block starts at row col_offsets[i] of an (sum n_cols) x k
 * row-major array, its Y block at row row_offsets[i] of (sum n_rows) x k
 * (argcsr_batch_offsets returns both prefix sums, count + 1 entries each).
 * argcsr_batch_spmm runs every group of every matrix in one launch with a
 * fixed grid (two waves of the blocks that fit on the SMs); warps take
 * contiguous runs of the concatenated group list for k < 4 and stride
 * through it for k >= 4 (rows of X stay in cache while all warps sweep the
 * same few matrices).  X and Y must be 16-byte aligned.
 * argcsr_batch_graph_create captures that launch
 * (for fixed X, Y and k) in a CUDA graph replayed by argcsr_graph_launch.
 * ------------------------------------------------------------------------ */
ARGCSR_API argcsr_status argcsr_batch_create(int32_t count, const argcsr_t *mats,
                                             argcsr_stream_t stream, argcsr_batch_t *out);
ARGCSR_API argcsr_status argcsr_batch_info(argcsr_batch_t batch, int64_t *total_rows,
                                           int64_t *total_cols, int64_t *total_groups,
                                           int64_t *total_nnz, int64_t *total_slots);
ARGCSR_API argcsr_status argcsr_batch_offsets(argcsr_batch_t batch, int64_t *h_row_offsets,
                                              int64_t *h_col_offsets);
ARGCSR_API argcsr_status argcsr_batch_spmm(argcsr_batch_t batch, int32_t k, const void *d_X,
                                           void *d_Y, argcsr_stream_t stream);
ARGCSR_API argcsr_status argcsr_batch_graph_create(argcsr_batch_t batch, int32_t k,
                                                   const void *d_X, void *d_Y,
                                                   argcsr_graph_t *out);
ARGCSR_API argcsr_status argcsr_graph_launch(argcsr_graph_t graph, argcsr_stream_t stream);
ARGCSR_API argcsr_status argcsr_graph_destroy(argcsr_graph_t graph);
ARGCSR_API argcsr_status argcsr_batch_destroy(argcsr_batch_t batch, argcsr_stream_t stream);

/* ---------------------------------------------------------------------------
 * argcsr_autotune -- choose group_size and desired_chunk_size for a matrix
 * by measurement.  The paper reports that the best desiredChunkSize depends
 * on the matrix (Section 5: regular matrices want large values, irregular
 * ones small) and uses 128 threads per block; this call converts the CSR
 * input with every candidate (G in the bits of group_size_mask: 1 = 32,
 * 2 = 64, 4 = 128; bit 8 adds the one-thread-per-row layouts of each G;
 * D in {1, 2, 3, 4, 6, 8, 12, 16, 32}; V = 1, and V = 2 as well when bit
 * 16 is set), times
 * `reps` products with k right-hand sides, and returns the fastest in *best
 * (its time per product in *best_us).  Candidates whose layout has the same
 * size as one already timed are skipped.  Synchronous on `stream`.
 * ------------------------------------------------------------------------ */
ARGCSR_API argcsr_status argcsr_autotune(int32_t n_rows, int32_t n_cols, int64_t nnz,
                                         const int32_t *d_rowPointers, const int32_t *d_columns,
                                         const void *d_values, argcsr_dtype dtype, int32_t k,
                                         int32_t group_size_mask, int32_t reps,
                                         argcsr_stream_t stream, argcsr_params *best,
                                         float *best_us);

/* argcsr_autotune_batch -- the same search for a batch: for every
 * candidate desiredChunkSize in {1, 2, 4, 8, 16, 32} (G = 32, V = 1) convert
 * all `count` matrices, time `reps` argcsr_batch_spmm launches with k
 * right-hand sides, keep the fastest.  Matrix i is given by host arrays of
 * sizes and of device pointers to its CSR arrays.  Synchronous. */
ARGCSR_API argcsr_status argcsr_autotune_batch(int32_t count, const int32_t *h_n_rows,
                                               const int32_t *h_n_cols, const int64_t *h_nnz,
                                               const int32_t *const *h_rowPointers,
                                               const int32_t *const *h_columns,
                                               const void *const *h_values, argcsr_dtype dtype,
                                               int32_t k, int32_t reps, argcsr_stream_t stream,
                                               argcsr_params *best, float *best_us);

/* ---------------------------------------------------------------------------
 * Iterative solution of A x = b (SPD A) with conjugate gradients on ARG-CSR.
 * The paper names iterative solvers as the consumer of SpMV (Section 1);
 * the solver is textbook CG with iterative refinement, not part of the
 * paper's method.
 *
 * argcsr_residual: r = b - A x, with FP64 vectors and FP64 accumulation for
 * every storage type (f32 / bf16 values are widened exactly).  d_b, d_x,
 * d_r: f64 device arrays of n_rows / n_cols / n_rows elements.
 *
 * argcsr_cg_solve: iterative refinement in FP64 around an inner CG in the
 * storage's working precision.
 *   repeat:  r = b - A_residual x            (FP64)
 *            stop if ||r||_2 <= tol ||b||_2
 *            CG on A d = r / ||r||, until its residual falls by inner_tol
 *            x += ||r|| d                     (FP64)
 * The inner CG works in FP32 for ARGCSR_F32 / ARGCSR_BF16 storage (FP32
 * accumulation) and in FP64 for ARGCSR_F64.  A_residual (NULL: A) supplies
 * the FP64 residual; pass an FP64 copy when low-precision storage rounds the
 * matrix.  d_x holds the initial guess on entry and the solution on return.
 * All scalars stay on the device; the host reads them every check_every
 * inner iterations.  Work arrays (4 vectors of the working type, 1 FP64
 * vector) come from the library's pool.  Synchronous on `stream`.
 * ------------------------------------------------------------------------ */
typedef struct {
    double tol;           /* target ||b - A x|| / ||b|| (> 0)                    */
    double inner_tol;     /* inner residual reduction; 0: 1e-5 (FP32), tol (FP64) */
    int32_t max_iters;    /* cap on inner CG iterations over the whole solve     */
    int32_t max_outer;    /* cap on refinement steps                              */
    int32_t check_every;  /* inner iterations between host checks; 0: 16          */
    int32_t reserved;
} argcsr_cg_params;

typedef struct {
    int32_t outer_iters;  /* refinement steps taken                               */
    int32_t inner_iters;  /* CG iterations over all steps                         */
    int32_t converged;    /* 1 if ||b - A x|| <= tol ||b|| at exit                */
    int32_t reserved;
    double rel_residual;  /* ||b - A x|| / ||b|| at exit (FP64, A = A_residual)   */
} argcsr_cg_result;

ARGCSR_API argcsr_status argcsr_residual(argcsr_t A, const double *d_b, const double *d_x,
                                         double *d_r, argcsr_stream_t stream);
ARGCSR_API argcsr_status argcsr_cg_solve(argcsr_t A, argcsr_t A_residual, const double *d_b,
                                         double *d_x, const argcsr_cg_params *params,
                                         argcsr_stream_t stream, argcsr_cg_result *result);

/* Baseline for the solver: the same CG in FP64 with the plain CSR vector
 * kernel (Section 2 format) as the operator; n x n matrix, f64 values. */
ARGCSR_API argcsr_status argcsr_baseline_csr_cg(int32_t n, int64_t nnz, const int32_t *d_rowPointers,
                                                const int32_t *d_columns, const double *d_values,
                                                const double *d_b, double *d_x,
                                                const argcsr_cg_params *params,
                                                argcsr_stream_t stream, argcsr_cg_result *result);

/* ---------------------------------------------------------------------------
 * Serving: SpMV and CG-solve requests on a pool of device-resident matrices
 * with continuous batching (a library runtime; the paper has no serving
 * layer).  A worker thread owns the GPU side.  Oldest first, it admits
 * requests while a stream slot (num_streams, max_inflight) and HBM budget
 * are free; CG jobs leave spmv_streams slots to SpMV, and SpMV requests
 * pass CG requests that wait for a slot or for memory:
 *   - SpMV requests on the same matrix are fused, up to max_batch of them,
 *     into one SpMM launch; their x vectors become the columns of X.
 *   - A CG request becomes a resumable job on its own stream.
 * Work admitted while other requests run overlaps with them on the device.
 *
 * Budget: matrices count toward hbm_budget_bytes when added.  Each request
 * also counts while it runs: its work arrays are packed X/Y for fused SpMV,
 * and 4 vectors of the working type + 1 FP64 vector for CG.  A request that
 * cannot fit even on an idle server fails with ARGCSR_ENOMEM.
 *
 * Request buffers are device pointers owned by the caller, kept alive until
 * the request is done:
 *   - SpMV: d_x (n_cols) in, d_y (n_rows) out; f64 for ARGCSR_F64 matrices,
 *     f32 otherwise.
 *   - CG: d_b in, d_x in (initial guess) / out; both f64.  Tolerance as in
 *     argcsr_cg_solve.
 *
 * Register every matrix before the first request (later: ARGCSR_EINVAL).
 * Matrices are borrowed
 * and must outlive the server.  argcsr_server_destroy serves what is queued,
 * then stops.  Times are host microseconds (a monotonic clock).
 * ------------------------------------------------------------------------ */
typedef struct argcsr_server *argcsr_server_t;
typedef struct {
    int64_t hbm_budget_bytes;  /* 0: no limit                                   */
    int32_t max_inflight;      /* requests on the GPU at once; 0: 64            */
    int32_t num_streams;       /* stream slots; 0: 8                            */
    int32_t max_batch;         /* SpMV requests per fused launch (<= 16); 0: 16 */
    int32_t cg_check_every;    /* inner CG iterations per job step; 0: 16       */
    int32_t spmv_streams;      /* slots CG jobs leave to SpMV, below num_streams;
                                  0: num_streams / 4 (1 for 2 or 3 streams,
                                  none for 1)                                   */
} argcsr_server_params;

typedef struct {
    int32_t state;             /* 0 queued, 1 running, 2 done, 3 failed         */
    int32_t status;            /* argcsr_status of the request                  */
    int32_t iters;             /* CG: inner iterations                          */
    int32_t batch;             /* requests fused with this one (SpMV)           */
    int32_t converged;         /* CG: reached the tolerance                     */
    int32_t reserved;
    double t_submit_us, t_start_us, t_done_us;
    double rel_residual;       /* CG: ||b - A x|| / ||b|| at the end            */
} argcsr_request_info;

ARGCSR_API argcsr_status argcsr_server_create(const argcsr_server_params *params, argcsr_server_t *out);
ARGCSR_API argcsr_status argcsr_server_add_matrix(argcsr_server_t server, argcsr_t A,
                                                  argcsr_t A_residual, int32_t *id);
ARGCSR_API argcsr_status argcsr_server_submit_spmv(argcsr_server_t server, int32_t matrix,
                                                   const void *d_x, void *d_y, int64_t *request);
ARGCSR_API argcsr_status argcsr_server_submit_cg(argcsr_server_t server, int32_t matrix,
                                                 const double *d_b, double *d_x, double tol,
                                                 int32_t max_iters, int64_t *request);
ARGCSR_API argcsr_status argcsr_server_query(argcsr_server_t server, int64_t request,
                                             argcsr_request_info *info);
/* Wait for one request (timeout_s <= 0: no limit); ARGCSR_ENOTSUP on timeout. */
ARGCSR_API argcsr_status argcsr_server_wait(argcsr_server_t server, int64_t request,
                                            double timeout_s, argcsr_request_info *info);
/* Forget a finished request (its record is kept until then, so that it can
 * be queried); ARGCSR_EINVAL if it is unknown or not finished. */
ARGCSR_API argcsr_status argcsr_server_release(argcsr_server_t server, int64_t request);
/* Wait until every submitted request is done; ARGCSR_ENOTSUP on timeout. */
ARGCSR_API argcsr_status argcsr_server_drain(argcsr_server_t server, double timeout_s);
ARGCSR_API argcsr_status argcsr_server_stats(argcsr_server_t server, int64_t *matrix_bytes,
                                             int64_t *work_bytes, int64_t *pending,
                                             int64_t *unfinished);
ARGCSR_API argcsr_status argcsr_server_destroy(argcsr_server_t server);

/* ---------------------------------------------------------------------------
 * argcsr_convert_noalloc -- the CSR -> ARG-CSR conversion of
 * argcsr_create_from_csr for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a library facility.
 *
 * Who needs it: code whose device memory is all handed out up front and
 * owned by someone else -- a framework arena or caching allocator that must
 * stay the only allocator in the process, a service under a hard per-process
 * memory cap, or a latency-critical loop where cudaMalloc/cudaFree would
 * stall the device.  Such callers can still size and own their outputs.
 *
 * What it does not do: call cudaMalloc, cudaFree, cudaHostAlloc, a memory
 * pool, or any allocating library routine, on the device or the host (the
 * sizes come back through a copy into a local variable).  All intermediate
 * arrays live in one
 * file-scope __device__ array of ARGCSR_NOALLOC_SCRATCH_BYTES bytes, which
 * every GPU that loads this library holds until the process exits.  That
 * caps the matrix at ARGCSR_NOALLOC_MAX_ROWS rows; more rows return
 * ARGCSR_EINVAL (see argcsr_last_error_message()) with no device work.
 *
 * Set-up: the first call on a device looks up the device address of the
 * scratch array (cudaGetSymbolAddress) with that device current.  Make that
 * first call before any stream capture on the device.
 *
 * Sharing: every call on a device uses the same scratch array, which keeps
 * the previous call's contents (the parts that must start at zero are
 * cleared by each call).  Calls whose work overlaps on the GPU -- on two
 * streams, or from two host threads -- race on it: order them.
 *
 * Inputs are those of argcsr_create_from_csr.  Outputs, caller-owned device
 * memory in the layout of argcsr_export:
 *   d_groupInfo      int32[4 * group_capacity] ({firstRow, size, offset,
 *                    chunkSize} per group, 16-byte aligned),
 *   d_threadsMapping int32[n_rows] (always written),
 *   d_out_columns    int32[slot_capacity],
 *   d_out_values     slot_capacity elements of `dtype`;
 *   with vec_width above 1 both are written V elements at a time and must
 *   be 16-byte aligned (ARGCSR_EINVAL otherwise).
 * *h_n_groups and *h_n_slots receive the required sizes.  If a capacity is
 * too small the call returns ARGCSR_EINVAL after setting them, writes no
 * group records or slots, and can be repeated with larger buffers (pass 0
 * capacities to query the sizes).  Synchronises `stream` like
 * argcsr_create_from_csr.
 * ------------------------------------------------------------------------ */
#define ARGCSR_NOALLOC_MAX_ROWS 1048576
#define ARGCSR_NOALLOC_SCRATCH_BYTES 18166016
ARGCSR_API argcsr_status argcsr_convert_noalloc(
    int32_t n_rows, int32_t n_cols, int64_t nnz,
    const int32_t *d_rowPointers, const int32_t *d_columns, const void *d_values,
    argcsr_dtype dtype, const argcsr_params *params,
    int32_t *d_groupInfo, int64_t group_capacity, int32_t *d_threadsMapping,
    int32_t *d_out_columns, void *d_out_values, int64_t slot_capacity,
    int64_t *h_n_groups, int64_t *h_n_slots, argcsr_stream_t stream);

/* ---------------------------------------------------------------------------
 * Baseline: SpMV straight on CSR (Section 2), for comparison only.
 *   variant 0: one thread per row (scalar CSR);
 *   variant 1: a group of 2..32 lanes per row, sized from the mean row
 *              length (vector CSR).
 * Arrays as in argcsr_create_from_csr; x, y as in argcsr_spmv.  No
 * validation of the CSR content beyond the argument checks.
 * ------------------------------------------------------------------------ */
ARGCSR_API argcsr_status argcsr_baseline_csr_spmv(
    int32_t n_rows, int32_t n_cols, int64_t nnz,
    const int32_t *d_rowPointers, const int32_t *d_columns, const void *d_values,
    argcsr_dtype dtype, int32_t variant, const void *d_x, void *d_y,
    argcsr_stream_t stream);

/* Miscellaneous ------------------------------------------------------------ */

/* Human-readable name of a status code (static storage). */
ARGCSR_API const char *argcsr_status_string(argcsr_status status);

/* Text of the last CUDA error this library saw in the calling thread
 * (static thread-local storage; empty if none). */
ARGCSR_API const char *argcsr_last_error_message(void);

/* Number of kernels this library has launched in this process. */
ARGCSR_API uint64_t argcsr_launch_count(void);

/* Return the cached, currently unused memory of the library's pool on the
 * current device to the driver. */
ARGCSR_API argcsr_status argcsr_trim_pool(void);

/* ---------------------------------------------------------------------------
 * Kernel tracing, a profiling aid (off by default).  Between
 * argcsr_trace_begin and argcsr_trace_end the library records a CUDA event
 * pair around every kernel it launches, on the stream it launches on.
 * argcsr_trace_begin creates the events of the first 2048 launches up front
 * (on the current device), so that they are not created inside the traced
 * region.
 * argcsr_trace_end waits for the recorded events and sums the durations per
 * kernel; argcsr_trace_kernel then reads, for kernel index 0 .. count-1, its
 * name (static storage), number of launches and total milliseconds.
 * ------------------------------------------------------------------------ */
ARGCSR_API argcsr_status argcsr_trace_begin(void);
/* As argcsr_trace_begin, but events are recorded only around launches of
 * the kernel named `name` (for instance "k_spmv_g32"; NULL: every kernel).
 * An event pair delays the launch that follows it by a few microseconds on
 * the device, so a timed region that needs the duration of one kernel traces
 * only that one.  ARGCSR_EINVAL if the name has 64 characters or more. */
ARGCSR_API argcsr_status argcsr_trace_begin_kernel(const char *name);
ARGCSR_API argcsr_status argcsr_trace_end(void);
ARGCSR_API int32_t argcsr_trace_kernel_count(void);
ARGCSR_API argcsr_status argcsr_trace_kernel(int32_t index, const char **name, int64_t *launches,
                                             double *total_ms);

/* Library version string, e.g. "argcsr 0.1 sm_103a". */
ARGCSR_API const char *argcsr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ARGCSR_H */
