/*
 * spx.h -- C ABI of libspx, a sparse matrix-vector product (SpMV) and Krylov
 * solver library for NVIDIA GB300 (sm_103a).
 *
 * Operations and where they are defined (arXiv 2103.10116, "Porting a sparse
 * linear algebra math library to Intel GPUs"):
 *   - SpMV y = A x and the CSR / COO storage formats: Section 5.
 *   - CG, BiCGSTAB, GMRES: the Krylov methods of Section 5 (textbook forms of
 *     the references cited there).
 *   - ELL and hybrid (ELL + COO) storage, merge-path CSR, FP32 inner / FP64
 *     outer iterative refinement, batched solves and the request server are
 *     library extensions; the paper has no counterpart for them.
 *
 * Conventions for every entry point:
 *   - Return value: an spx_status; SPX_OK (0) on success.  No C++ exception
 *     crosses this boundary.  On failure spx_last_error() returns a message
 *     for the calling thread.
 *   - Pointers are DEVICE pointers (cudaMalloc / PyTorch CUDA memory of the
 *     context's device) unless a parameter says "host".
 *   - Indices are int32; values are IEEE double (SPX_F64) or float (SPX_F32).
 *   - Work is enqueued asynchronously on the context's stream unless stated
 *     otherwise; argument errors are reported synchronously.
 *   - Vectors passed as input and output of one call must not alias.
 */
#ifndef SPX_H
#define SPX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spx_ctx spx_ctx;
typedef struct spx_matrix spx_matrix;
typedef struct spx_batch spx_batch;
typedef struct spx_server spx_server;

typedef enum {
    SPX_OK = 0,
    SPX_ERR_INVALID = 1,     /* malformed argument or matrix (e.g. bad row_ptr / column index) */
    SPX_ERR_TOO_LARGE = 2,   /* a format's padded footprint does not fit (e.g. ELL of a power-law matrix) */
    SPX_ERR_OOM = 3,         /* device allocation failed */
    SPX_ERR_CUDA = 4,        /* a CUDA runtime call failed; message in spx_last_error() */
    SPX_ERR_UNSUPPORTED = 5, /* combination not implemented (e.g. kernel not valid for the format) */
    SPX_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    SPX_ERR_NOT_FOUND = 7    /* unknown request id or export part */
} spx_status;

typedef enum { SPX_CSR = 0, SPX_ELL = 1, SPX_COO = 2, SPX_HYB = 3 } spx_format;
typedef enum { SPX_F64 = 0, SPX_F32 = 1 } spx_dtype;
typedef enum { SPX_CG = 0, SPX_BICGSTAB = 1, SPX_GMRES = 2, SPX_CGS = 3 } spx_solver;
/* OR into the solver argument of spx_solve / spx_solve_fixed / spx_server_submit:
 * Jacobi preconditioning with M = diag(A) (a zero diagonal entry counts as 1).
 * CG becomes preconditioned CG; BiCGSTAB, CGS and GMRES are preconditioned from
 * the right, so the residual they test is always b - A x. */
#define SPX_PRECOND_JACOBI 0x100
/* OR SPX_PRECOND_BLOCK(bs) instead for block-Jacobi preconditioning (Section 2
 * lists block-Jacobi among the library's preconditioners): M = the block
 * diagonal of A with blocks of bs consecutive rows and columns, bs in
 * {1, 2, 4, 8, 16, 32}; the last block holds the remaining rows.  Each block is
 * inverted once per matrix and solve precision by Gauss-Jordan elimination
 * with partial pivoting in FP64 (a block with an exactly zero pivot counts as
 * the identity) and applied as a dense bs x bs product; the inverses take
 * n * bs values of device memory.  Applied as Jacobi is: preconditioned CG, right
 * preconditioning for the others.  Any other flag bits give SPX_ERR_INVALID. */
#define SPX_PRECOND_BLOCK_JACOBI 0x200
#define SPX_PRECOND_BLOCK_SHIFT 16
#define SPX_PRECOND_BLOCK(bs) (SPX_PRECOND_BLOCK_JACOBI | ((bs) << SPX_PRECOND_BLOCK_SHIFT))
/* OR into SPX_PRECOND_BLOCK(bs) for adaptive storage of the block inverses in
 * FP64 solves (the adaptive-precision block-Jacobi Section 2 cites): a block
 * whose 1-norm condition number times 2^-24 is at most 1e-2 is applied from an
 * FP32 copy of its inverse (half the bytes), the others from FP64; the
 * arithmetic stays FP64.  Ignored by FP32 solves, which store FP32 inverses. */
#define SPX_PRECOND_BLOCK_ADAPTIVE 0x400
/* OR into the solver argument of spx_solve (or a request of spx_server_submit /
 * spx_server_submit_matrix): run the whole solve in ONE kernel launch on one
 * thread-block cluster (16 SMs, or 8 where the device runs no cluster of 16 or
 * the system has fewer than 65 536 rows).  Block k of the cluster owns a slice
 * of rows; the Krylov vectors live in a device workspace of 64 bytes per row
 * cached in the matrix handle; the dot products are summed over the cluster in
 * a fixed order, so the result does not depend on timing.  The iterations are
 * the textbook recurrences of Section 5 (CG, BiCGSTAB, CGS; the true residual
 * at exit with at most 3 restarts, as spx_solve); SPX_PREC_MIXED as
 * spx_precision describes it.  For callers that run many mid-size solves (tens of thousands
 * to about a million rows) at once on separate streams, such as the request
 * server: each solve then occupies its own SMs and pays no launch per
 * iteration.  A lone solve of a large system is faster without the flag (the
 * general path spreads each iteration over the whole GPU).  CSR matrices of at
 * most 2^30 rows, no preconditioner, not spx_solve_fixed, not GMRES; otherwise
 * SPX_ERR_UNSUPPORTED (also when no such cluster fits the device). */
#define SPX_SOLVE_ONE_CLUSTER 0x800

/* Arithmetic of a solve: all FP64; all FP32 (values, vectors, dots and
 * scalars in float); or MIXED, Krylov iterations in float on an FP32 copy of
 * the values with FP64 corrections on the FP64 values:
 *   - CG: reliable updates (residual replacement, Sleijpen and van der Vorst):
 *     the FP32 iterate is accumulated in a correction that is added to the
 *     FP64 x whenever the FP32 recurrence residual has fallen below 0.1 of its
 *     largest value since the last update (or to tol ||b||, or the budget is
 *     spent); then b - A x is formed in FP64 and its rounding replaces the
 *     FP32 residual, the search direction kept.  info->restarts counts the
 *     updates.
 *   - BiCGSTAB, CGS, GMRES: FP64 iterative refinement (outer residual
 *     r = b - A x and update x += d in double); an inner cycle solves
 *     A d = r / ||r|| to 1e-4 relative in at most 500 iterations, at most 20
 *     cycles; an inner CGS cycle also ends once its recurrence residual has
 *     gone 20 iterations without halving.  info->restarts counts the cycles. */
typedef enum { SPX_PREC_F64 = 0, SPX_PREC_F32 = 1, SPX_PREC_MIXED = 2 } spx_precision;

typedef enum {
    SPX_CONVERGED = 0,  /* true relative residual <= tol */
    SPX_MAX_ITER = 1,   /* iteration limit reached first */
    SPX_BREAKDOWN = 2,  /* a Krylov denominator became exactly zero */
    SPX_STAGNATED = 3,  /* recurrence converged but the true residual stayed above tol after the restarts */
    SPX_SOLVE_TIMEOUT = 4
} spx_solve_status;

/* SpMV kernel choice for a matrix (spx_matrix_set_kernel). */
typedef enum {
    SPX_KERNEL_AUTO = 0,        /* format default, chosen from row-length statistics */
    SPX_KERNEL_CSR_VECTOR = 1,  /* CSR: one sub-warp of `param` lanes (1..32, power of 2) per row */
    SPX_KERNEL_CSR_MERGE = 2,   /* CSR: merge-path split of rows + nonzeros, TMA-staged tiles */
    SPX_KERNEL_ELL = 3,         /* ELL / HYB ELL part: one thread per `param` rows (1, 2, or 4 in FP32; default 2) */
    SPX_KERNEL_COO = 4,         /* COO / HYB COO part: 1 = row-block (COO format; the default for short rows
                                   of similar length), 8/16 = warp-independent split,
                                   216/232 = the split on tile-transposed copies of the COO arrays with 16/32
                                   entries per lane (built on first use; default otherwise: 216),
                                   104/108/116 = tiled segmented reduction with 4/8/16 items per thread */
    SPX_KERNEL_CSR_SPLIT = 5,   /* CSR: each lane takes `param` (8 or 16) consecutive nonzeros, warps independent */
    SPX_KERNEL_CSR_TILED = 7,   /* CSR: as SPX_KERNEL_CSR_SPLIT with `param` (16 or 32) nonzeros per lane, on
                                   a tile-transposed copy of the nonzeros with per-granule row descriptors
                                   (built on first use; one more copy of the column indices and values).
                                   The automatic choice for heavy-tailed rows, with 32 */
    SPX_KERNEL_CSR_ROWS = 6     /* CSR: tiles of 128 rows bulk-copied to shared memory, 1, 2 or 4 threads
                                   per row (rows of similar length; SPX_ERR_TOO_LARGE if a tile's nonzeros
                                   do not fit in shared memory); param = stages + 10 x threads per row,
                                   stages = shared-memory stages per block (2: the next tile copied while
                                   this one is reduced): 1 or 2 = that many stages, one thread per row;
                                   12, 22, 42 = two stages, 1, 2 or 4 threads per row; 0 = two stages,
                                   and when the mean row length is 16 or more 2 (FP64) or 4 (FP32)
                                   threads per row, else one */
} spx_kernel;

/* spx_matrix_create flags */
#define SPX_HOST_INPUT 1u     /* row_ptr / col_idx / values are host pointers */
#define SPX_MIXED_SHADOW 2u   /* also keep an FP32 copy of FP64 values (for SPX_PREC_MIXED) */

/* Device allocator supplied by the caller (for example PyTorch's caching
 * allocator).  alloc returns NULL on failure.  stream is a cudaStream_t. */
typedef void *(*spx_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*spx_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* ------------------------------------------------------------------ context */

/* Create a context bound to CUDA device `device` and stream `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  With alloc == NULL the
 * library allocates with cudaMallocAsync / cudaFreeAsync on that stream.
 * The context owns no user memory.  Errors: SPX_ERR_INVALID (bad device),
 * SPX_ERR_CUDA. */
int spx_ctx_create(spx_ctx **out, int device, void *stream, spx_alloc_fn alloc, spx_free_fn free,
                   void *user);
/* Destroy a context.  Matrices, batches and servers created from it must be
 * destroyed first.  NULL is accepted. */
int spx_ctx_destroy(spx_ctx *ctx);
/* Rebind the context to another stream of the same device. */
int spx_ctx_set_stream(spx_ctx *ctx, void *stream);

/* Size the launch grids of the context's kernels for `sms` SMs instead of the
 * whole device (sms <= 0: the whole device; larger values are clamped to it).
 * For several contexts whose solves run at once on separate streams, such as
 * the request server's slots: a mid-size solve's kernels have a few
 * microseconds of work each, and grids that fill the device keep another
 * stream's kernels from starting beside them.  Scratch buffers stay sized for
 * the whole device, so matrices may be shared between contexts of any setting.
 * Takes effect for later launches (captured solver graphs are keyed by it).
 * *effective (may be NULL) receives the value in force. */
int spx_ctx_set_grid_sms(spx_ctx *ctx, int sms, int *effective);

/* Synchronise ctx's stream and report whether any bounded device-side wait
 * (look-back flags of the load-balanced SpMV kernels, bulk-copy mbarriers)
 * gave up since the last check: SPX_ERR_TIMEOUT, after which the error word
 * is cleared and the context stays usable; else SPX_OK.  Solves check this
 * themselves; asynchronous calls (spx_spmv) are checked by calling it. */
int spx_ctx_check(spx_ctx *ctx);


/* ------------------------------------------------------------------ matrices */

/* Create a matrix in `format` (spx_format) with value type `dtype`
 * (spx_dtype) from CSR arrays (Section 5): row_ptr[nrows+1], col_idx[nnz],
 * values[nnz] of type `values_dtype`.  The input arrays are borrowed for the
 * duration of the call only (device pointers, or host pointers with
 * SPX_HOST_INPUT); the handle owns every array it builds.  The call
 * validates the CSR structure on the device (row_ptr[0] = 0, non-decreasing,
 * row_ptr[nrows] = nnz, 0 <= col < ncols); duplicates, unsorted columns and
 * explicit zeros are accepted and kept in order.  hyb_width: ELL width of the
 * HYB format, -1 = footprint-optimal.  The call synchronises the stream once.
 * Errors: SPX_ERR_INVALID, SPX_ERR_TOO_LARGE (ELL width x rows beyond the
 * device budget), SPX_ERR_OOM. */
int spx_matrix_create(spx_ctx *ctx, spx_matrix **out, int format, int dtype, int64_t nrows,
                      int64_t ncols, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                      const void *values, int values_dtype, int64_t hyb_width, unsigned flags);
/* Free a matrix and all its device arrays (ordered on the creating context's
 * stream).  Work on A issued on another context's stream must have completed
 * first (synchronise that stream). */
int spx_matrix_destroy(spx_matrix *A);

typedef struct {
    int32_t format, dtype;
    int64_t nrows, ncols, nnz;
    int64_t ell_width;    /* ELL / HYB-ELL width k (0 for CSR / COO) */
    int64_t ell_ld;       /* leading dimension of the column-major ELL arrays (multiple of 32, >= nrows) */
    int64_t coo_nnz;      /* entries in the COO (part) */
    int64_t max_row_len;
    double mean_row_len;
    int64_t device_bytes; /* bytes of all arrays the handle owns */
    int32_t kernel, kernel_param;
    int32_t has_f32_shadow;
} spx_matrix_info;

/* Fill `info` (host) for matrix A.  Host-only, no device work. */
int spx_matrix_get_info(const spx_matrix *A, spx_matrix_info *info);

/* Parts of a matrix that spx_matrix_export can copy out. */
typedef enum {
    SPX_PART_ROW_PTR = 0, SPX_PART_COL = 1, SPX_PART_VAL = 2,        /* CSR (CSR format) */
    SPX_PART_ELL_COL = 3, SPX_PART_ELL_VAL = 4,                      /* ELL / HYB ELL part, [width][ld] */
    SPX_PART_COO_ROW = 5, SPX_PART_COO_COL = 6, SPX_PART_COO_VAL = 7, /* COO / HYB COO part */
    SPX_PART_VAL_F32 = 8                                             /* FP32 shadow of the primary values */
} spx_part;

/* Copy one internal array of A into the caller's device buffer dst of
 * dst_bytes bytes (synchronous).  *written receives the array size in bytes.
 * Used to check conversions byte for byte.  Errors: SPX_ERR_NOT_FOUND (the
 * format has no such part), SPX_ERR_INVALID (dst too small). */
int spx_matrix_export(spx_ctx *ctx, const spx_matrix *A, int part, void *dst, size_t dst_bytes,
                      size_t *written);

/* Select the SpMV kernel (spx_kernel) and its parameter for A; host-only.
 * Errors: SPX_ERR_UNSUPPORTED if the kernel does not apply to A's format. */
int spx_matrix_set_kernel(spx_matrix *A, int kernel, int param);

/* Autotune A's SpMV kernel: time every kernel variant spx_matrix_set_kernel
 * accepts for A's format and dtype (the automatic choice included) with CUDA
 * events on the context stream, `reps` back-to-back products y = A x each after
 * one warm-up (x = 0, in the handle's staging buffers), and keep the fastest.
 * Variants that do not fit A (SPX_ERR_TOO_LARGE, SPX_ERR_UNSUPPORTED) are
 * skipped.  Outputs (may be NULL): the chosen kernel, its parameter and its
 * time per product in microseconds.  Synchronous.  reps must be in [1, 1000];
 * on any other error A keeps its previous kernel.  The Python binding adds a
 * JSON cache of choices keyed by GPU name and the matrix's shape statistics. */
int spx_matrix_tune(spx_ctx *ctx, spx_matrix *A, int reps, int *kernel, int *param, float *best_us);

/* ------------------------------------------------------------------ SpMV */

/* y = A x (Section 5), x[ncols] and y[nrows] of A's dtype, device pointers,
 * asynchronous on the context stream.  x and y must not overlap. */
int spx_spmv(spx_ctx *ctx, const spx_matrix *A, const void *x, void *y);

/* y = alpha A x + beta y (same rules as spx_spmv; alpha, beta given in double
 * and applied in A's dtype). */
int spx_spmv_axpby(spx_ctx *ctx, const spx_matrix *A, double alpha, const void *x, double beta,
                   void *y);

/* End-to-end SpMV from HOST memory: copies x_host (ncols values) to the
 * device, computes y = A x and copies y back to y_host (nrows values);
 * returns after the result is in y_host.  Staging buffers are owned by the
 * handle.  Host buffers should be pinned for full copy bandwidth. */
int spx_spmv_host(spx_ctx *ctx, const spx_matrix *A, const void *x_host, void *y_host);

/* SpMV for callers that cannot allocate device memory.
 *
 * The paper has no counterpart for this entry point.  Some callers may not
 * call cudaMalloc, or any routine that allocates, at the moment they need a
 * product: a real-time loop whose memory is fixed before it starts (an
 * allocation can block, fail or synchronise the device at a bad moment), or a
 * host framework that owns all device memory and forbids libraries to take
 * their own.  This call computes y = A x with the merge-path CSR kernel
 * straight from the caller's CSR arrays (no matrix handle, no context) on
 * `stream` (a cudaStream_t) of the current device, and allocates nothing: the
 * kernel's scratch (tile map, per-tile carries, look-back flags, an error
 * word) lives in one fixed 1 MiB array that the library declares in device
 * global memory; every GPU that loads the library holds it until the process
 * exits.
 *   - Limit: nrows + nnz <= SPX_NOALLOC_MAX_TILES * 2048 (67,108,864);
 *     larger problems return SPX_ERR_TOO_LARGE and launch nothing.
 *   - row_ptr, col_idx and values must be 16-byte aligned (SPX_ERR_INVALID
 *     otherwise) and form a valid CSR matrix (not checked here).
 *   - The first call on a device sets that device up: it looks up the array's
 *     device address (cudaGetSymbolAddress) and opts the kernel in to its
 *     shared memory; make that first call before any stream capture.
 *   - Every call shares the one array, which keeps the previous call's
 *     contents; each call clears what must start at zero.  Calls whose kernels
 *     overlap on the GPU (different streams with no ordering between them)
 *     race on the array and give wrong results; order them on one stream.
 *   - The return code reports argument and launch errors only; the work runs
 *     asynchronously.  If one of the kernel's bounded waits gives up (about a
 *     second without progress, which a valid matrix never causes), every
 *     element of y is set to NaN, so the failure shows in the result without
 *     a host synchronisation.
 *   - dtype: SPX_F64 or SPX_F32 for values, x and y. */
#define SPX_NOALLOC_MAX_TILES 32768
int spx_spmv_csr_noalloc(void *stream, int dtype, int64_t nrows, int64_t ncols, int64_t nnz,
                         const int32_t *row_ptr, const int32_t *col_idx, const void *values, const void *x,
                         void *y);


/* ------------------------------------------------------------------ BLAS-1 */

/* *result = sum_i x_i y_i with a deterministic two-stage device reduction
 * (the global synchronisation that Section 6.2 notes for a dot product).
 * result is a device scalar of the dtype. */
int spx_dot(spx_ctx *ctx, int dtype, int64_t n, const void *x, const void *y, void *result);
/* y = alpha x + beta y (device vectors of the dtype). */
int spx_axpby(spx_ctx *ctx, int dtype, int64_t n, double alpha, const void *x, double beta,
              void *y);

/* ------------------------------------------------------------------ solvers */

typedef struct {
    int32_t status;            /* spx_solve_status */
    int32_t restarts;          /* restarts after a failed true-residual check (IR: outer cycles) */
    int64_t iterations;        /* Krylov iterations (one SpMV each for CG / GMRES, two for BiCGSTAB / CGS) */
    double relres_recurrence;  /* last recurrence (or estimated) relative residual */
    double relres_true;        /* ||b - A x|| / ||b|| formed at exit in FP64 */
    double time_ms;            /* wall time of the call */
    int64_t inner_iterations;  /* SPX_PREC_MIXED: total FP32 inner iterations */
} spx_solve_info;

/* Solve A x = b (Section 5's Krylov methods: CG, BiCGSTAB, CGS, GMRES(m);
 * CGS is Sonneveld's conjugate gradient squared with shadow residual r0).
 * b[n] and x[n] are device
 * vectors of A's dtype (double for SPX_PREC_MIXED, which needs an FP64 matrix
 * created with SPX_MIXED_SHADOW); x holds the initial guess on entry and the
 * solution on exit.  solver: spx_solver; restart: GMRES restart length m
 * (ignored otherwise); precision: spx_precision.  Stopping: recurrence
 * residual ||r|| / ||b|| <= tol, then the true residual is formed; if it is
 * above tol the method restarts from x (at most 3 times).  b = 0 gives x = 0.
 * Synchronous: returns after `info` (host) is filled.  Non-convergence is
 * reported in info->status, not as an error code.  Workspace is cached in the
 * matrix handle.  Errors: SPX_ERR_INVALID, SPX_ERR_UNSUPPORTED, SPX_ERR_OOM. */
int spx_solve(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, int solver, double tol,
              int64_t max_iter, int restart, int precision, spx_solve_info *info);

/* Run exactly `iterations` Krylov iterations without convergence checks
 * (fixed-work throughput mode, Section 6.4 runs 1,000 iterations).  Same
 * arguments as spx_solve; info->relres_true is formed at the end. */
int spx_solve_fixed(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, int solver,
                    int64_t iterations, int restart, int precision, spx_solve_info *info);

/* ------------------------------------------------------------------ batched */

/* A batch of nsys independent square CSR systems stored back to back.
 * row_off[nsys+1] and nnz_off[nsys+1] are HOST int64 prefix offsets;
 * row_ptr holds, for system s, its LOCAL row pointer (n_s + 1 entries,
 * starting at 0) at row_ptr[row_off[s] + s]; col_idx (local column indices)
 * and values (dtype) hold system s at [nnz_off[s], nnz_off[s+1]).
 * Device pointers (host pointers with flags SPX_HOST_INPUT), copied into the
 * handle; SPX_MIXED_SHADOW also keeps FP32 values for SPX_PREC_MIXED.  A
 * system's vector is held in shared memory by the kernel, so the largest
 * system may have about 28 000 rows (227 KB / 8 B); larger ones fail in
 * spx_batch_solve with SPX_ERR_TOO_LARGE.
 * Errors: SPX_ERR_INVALID, SPX_ERR_TOO_LARGE, SPX_ERR_OOM. */
int spx_batch_create(spx_ctx *ctx, spx_batch **out, int dtype, int64_t nsys, const int64_t *row_off,
                     const int64_t *nnz_off, const int32_t *row_ptr, const int32_t *col_idx,
                     const void *values, unsigned flags);
int spx_batch_destroy(spx_batch *B);

/* Solve all systems of B in one persistent kernel launch (CG, BiCGSTAB or CGS),
 * b and x concatenated by row_off (device, dtype of the batch; x is the
 * initial guess on entry).  infos: HOST array of nsys entries, or NULL.
 * precision SPX_PREC_MIXED as spx_precision describes it (CG with reliable
 * updates, BiCGSTAB and CGS with refinement cycles).  Synchronous. */
int spx_batch_solve(spx_ctx *ctx, spx_batch *B, const void *b, void *x, int solver, double tol,
                    int64_t max_iter, int precision, spx_solve_info *infos);

/* Time the candidate tile shapes of the batched kernel on B (threads per
 * system) and keep the fastest for later spx_batch_solve calls.
 * *chosen receives the threads per system picked.  Synchronous. */
int spx_batch_tune(spx_ctx *ctx, spx_batch *B, int solver, int precision, int *chosen);

/* ------------------------------------------------------------------ serving */

/* A continuous-batching solve server on ctx's device.  budget_bytes caps the
 * device memory of the requests running at once (<= 0: 90% of the free
 * memory at creation); max_slots is the number of large requests that may
 * run concurrently, each on its own stream (1..64).  Small and mid-size CG /
 * BiCGSTAB / CGS requests (unpreconditioned) (FP64 or MIXED, at most 24 576 rows by default,
 * see spx_server_set_batching) are instead gathered by four batch lanes: each
 * lane solves every queued small request of one kind (same solver, tol,
 * max_iter, precision and size class) in one launch of the batched kernel,
 * and the lanes run concurrently with each other and with the slots.  The
 * server owns worker threads and their contexts (allocating with
 * cudaMallocAsync); ctx is only used to pick the device.
 * Errors: SPX_ERR_INVALID, SPX_ERR_CUDA. */
int spx_server_create(spx_ctx *ctx, spx_server **out, int64_t budget_bytes, int max_slots);

/* Queue one solve A x = b.  row_ptr[n+1], col_idx[nnz], values[nnz] (double),
 * b[n] and x[n] are HOST buffers that must stay valid (and x untouched) until
 * the request completes; the operator is uploaded when the request is
 * admitted (FIFO, as soon as its device footprint fits in the budget) and
 * freed when it completes.  x receives the solution (initial guess 0).
 * solver / tol / max_iter / restart / precision as in spx_solve (MIXED keeps
 * an FP32 copy of the values).  The footprint counts a second, tile-transposed
 * copy of the nonzeros when the rows are heavy-tailed (longest row above four
 * times the mean plus 8), found by reading row_ptr during this call.  *req_id
 * receives the request id.  Returns at once.  Errors: SPX_ERR_INVALID,
 * SPX_ERR_TOO_LARGE (footprint > budget). */
int spx_server_submit(spx_server *S, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                      const double *values, const double *b, double *x, int solver, double tol, int64_t max_iter,
                      int restart, int precision, int64_t *req_id);

/* Queue one solve A x = b on a RESIDENT operator: A is a square FP64 matrix
 * handle (any format) on the server's device, created by the caller and
 * borrowed until the request completes (not destroyed, and not used by the
 * caller for spmv / solve meanwhile: a solve caches its workspace in the
 * handle).  Nothing of A is uploaded; b[n] and x[n] are HOST buffers as in
 * spx_server_submit.  Requests on the same handle run one at a time (later
 * ones wait while other requests are admitted past them); requests on
 * different handles overlap.  MIXED needs A created with SPX_MIXED_SHADOW.
 * Always solved on a slot (the batch lanes take host operators only), with the
 * one-cluster solve when spx_server_set_cluster_rows's rule selects it.
 * This is the submit call of the solve server in its resident-matrix form
 * (the paper's Section 5 solvers, served).  Errors: SPX_ERR_INVALID,
 * SPX_ERR_TOO_LARGE (workspace > budget). */
int spx_server_submit_matrix(spx_server *S, spx_matrix *A, const double *b, double *x, int solver, double tol,
                             int64_t max_iter, int restart, int precision, int64_t *req_id);

typedef struct {
    int64_t id;
    int32_t error;       /* spx_status of the request's own library calls (SPX_OK normally) */
    int32_t pad;
    spx_solve_info info; /* as filled by spx_solve */
    double submit_ms, admit_ms, done_ms;  /* host clock, milliseconds since spx_server_create */
    /* Where the time after admission went (host clock, milliseconds).  Slot
     * requests: upload of the operator and b, set-up (validation, statistics,
     * the library's copy of the operator; 0 for a resident operator), the
     * solve, the download of x.  Batched requests: the phases of the whole
     * batch they ran in (set-up = gathering the operators into pinned staging,
     * upload = copy and device build). */
    double upload_ms, setup_ms, solve_ms, download_ms;
    int32_t batched;     /* route: 1 a batch lane, 2 a slot with the one-cluster solve, 0 a slot */
    int32_t pad2;
} spx_server_result;

/* Collect up to max_results completed requests into results (host array),
 * waiting up to wait_ms milliseconds if none is ready; *count receives how
 * many were written.  Each completed request is reported once. */
int spx_server_poll(spx_server *S, spx_server_result *results, int max_results, int wait_ms, int *count);

/* Route requests of at most max_rows rows to the batch lanes from now on
 * (0: none; capped at 262 144 rows; negative: leave the limit unchanged, only
 * report it).  A batched request runs on one SM of the persistent batched
 * kernel, batched with queued requests of its size class.
 * *effective (may be NULL) receives the limit in force.  A request's result
 * does not depend on the route of others, but the same request may differ in
 * the last bits between the two routes (different reduction trees). */
int spx_server_set_batching(spx_server *S, int64_t max_rows, int64_t *effective);

/* Solve the slot requests of at most max_rows rows that are CG / BiCGSTAB /
 * CGS without preconditioner on a CSR operator whose rows hold at most 8
 * entries on average with SPX_SOLVE_ONE_CLUSTER (one launch on one
 * thread-block cluster per request) from now on; 0: none; capped at 2^30;
 * negative: leave the limit unchanged, only report it.  The default is 65 536
 * rows (measured: sixteen concurrent mixed CG solves of a 27 000-row 7-point
 * stencil completed 1.5-1.7x as many solves per second on clusters as on the
 * general path, whose one solve per matrix launches its kernels directly below
 * 50 000 rows; 97 000 rows broke even; longer rows with random columns were
 * slower on clusters).  The decision uses only the request's own matrix.  A request submitted with
 * SPX_SOLVE_ONE_CLUSTER
 * in its solver code takes that route whatever its size.  *effective (may be
 * NULL) receives the limit in force.  As with the batch lanes, a request's
 * result does not depend on other requests; the routes may differ in the last
 * bits. */
int spx_server_set_cluster_rows(spx_server *S, int64_t max_rows, int64_t *effective);

/* The grid share of the slots: every slot's context sizes its launch grids for
 * `sms` SMs (spx_ctx_set_grid_sms; 0: the whole device, the default; -1: a
 * rule that sizes a request's grids for a quarter of the device's SMs when its
 * operator has at most 8 entries per row on average and for half of them
 * otherwise; below -1: leave the setting unchanged, only report it), applied
 * from the next admitted request on.  Sixteen concurrent mixed solves of one
 * matrix completed up to 1.6x (250 000-row 7-point stencil, quarter grids) and
 * 1.2x (100 000 rows of 20 random columns, half grids) as many solves per
 * second as with whole-device grids, so workloads of similar concurrent solves
 * gain; on a mix of sizes from 10^3 to 10^6 rows no setting beat the whole
 * device beyond run-to-run variation, and a lone large solve is slower with
 * narrow grids.  The rule uses only the request's own matrix.  *effective (may
 * be NULL) receives the setting in force. */
int spx_server_set_slot_sms(spx_server *S, int sms, int *effective);

/* Requests waiting for admission, running, and the device bytes reserved. */
int spx_server_pending(spx_server *S, int64_t *queued, int64_t *running, int64_t *bytes_in_use);

/* Stop admitting, wait for running requests, join the workers, free all.
 * Requests still queued are dropped. */
int spx_server_destroy(spx_server *S);

/* ------------------------------------------------------------------ measurement and test aids */
/* Neither call is part of the method the paper describes: one measures a
 * floor for the SpMV kernels, the other exercises the failure path. */

/* A measurement aid (not part of the paper's method): stream col_idx[nnz]
 * and gather x (dtype SPX_F64 or SPX_F32) at every index, summing the
 * gathered values; nothing is stored except, practically never, out[0]
 * (device, one element).  Its time is the floor any SpMV kernel has on that
 * sparsity pattern: the gathers of x plus 4 bytes per nonzero.  Device
 * pointers; every index must lie inside x (not checked).  Asynchronous on the
 * context stream.  Errors: SPX_ERR_INVALID. */
int spx_probe_gather(spx_ctx *ctx, int64_t nnz, const int32_t *col_idx, const void *x, int dtype, void *out);

/* Test hook for the failure path: launch one wait that nothing will satisfy
 * (which = 0: a look-back flag; 1: an mbarrier phase), limited to about a
 * millisecond of SM clocks.  It gives up, records the error and returns, so
 * the following spx_ctx_check reports SPX_ERR_TIMEOUT.  Nothing hangs or
 * faults.  Asynchronous.  Errors: SPX_ERR_INVALID. */
int spx_selftest_wait_timeout(spx_ctx *ctx, int which);

/* ------------------------------------------------------------------ errors */

/* Message of the last failed call on this thread ("" if none). */
const char *spx_last_error(void);
/* Static name of a status code. */
const char *spx_status_str(int status);
/* Library version, major * 10000 + minor * 100 + patch. */
int spx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPX_H */
