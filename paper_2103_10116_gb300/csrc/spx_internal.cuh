// spx_internal.cuh -- types and helpers shared by the libspx CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/spx.h"

namespace spx {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define SPX_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return ::spx::cuda_fail(e_, #call);       \
    } while (0)

#define SPX_TRY(call)                                                    \
    do {                                                                 \
        int s_ = (call);                                                 \
        if (s_ != SPX_OK) return s_;                                     \
    } while (0)

// ------------------------------------------------------------------ shared-memory opt-in
// cudaFuncSetAttribute acts on the current device only, so the opt-in to more
// than 48 KB of dynamic shared memory is made once per (kernel, device) pair
// on the device current at the call.  bytes < 0 asks for the device's opt-in
// limit less the kernel's static shared memory.  *granted, if given, receives
// the limit set for this pair.
int smem_optin(const void *kernel, int bytes, int *granted = nullptr);

// ------------------------------------------------------------------ device error word
// Bit flags a kernel may set in ctx->dev_err instead of trapping.
enum : unsigned { DEVERR_MBAR_TIMEOUT = 1u, DEVERR_BOUNDS = 2u, DEVERR_QUEUE_TIMEOUT = 4u };

}  // namespace spx

// ------------------------------------------------------------------ context
struct spx_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    spx_alloc_fn alloc = nullptr;
    spx_free_fn free = nullptr;
    void *user = nullptr;
    int sm_count = 0;  // the device's SMs: every scratch buffer is sized for grids over all of them
    int grid_sms = 0;  // SMs the context's launch grids are sized for (<= sm_count; spx_ctx_set_grid_sms)
    int max_smem_optin = 0;
    int64_t l2_bytes = 0;
    // small always-resident device scratch: reduction tickets, flags
    unsigned *dev_err = nullptr;      // device error word
    unsigned *host_err = nullptr;     // pinned mirror
    // scratch of the stand-alone BLAS-1 reductions (spx_dot): block partials + ticket
    void *red = nullptr;
    int red_grid = 0;
    cudaStream_t capture_stream = nullptr;  // private stream used only to capture CUDA graphs
};

namespace spx {

void *dalloc(spx_ctx *ctx, size_t bytes);
void dfree(spx_ctx *ctx, void *p, size_t bytes);

// A device buffer owned by a handle.  It remembers the allocator that made it
// (the allocating context's callback, or none: cudaMallocAsync), so any
// context may free it: a matrix solved from several contexts (the server's
// slots) holds buffers from each.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    spx_free_fn free_fn = nullptr;
    void *free_user = nullptr;
    template <class T> T *as() const { return static_cast<T *>(p); }
};
int dbuf_alloc(spx_ctx *ctx, DBuf &b, size_t bytes);
void dbuf_free(spx_ctx *ctx, DBuf &b);

inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Padding added after every array the library owns, so that 16-byte aligned
// bulk copies that round a range outwards stay inside the allocation.
constexpr size_t kArrayPad = 64;

struct SolverWork;  // solvers.cu

}  // namespace spx

// ------------------------------------------------------------------ matrices
struct spx_matrix {
    spx_ctx *ctx = nullptr;   // allocating context
    int format = SPX_CSR;
    int dtype = SPX_F64;
    int64_t n = 0, ncols = 0, nnz = 0;
    int64_t max_len = 0;
    double mean_len = 0.0;
    // CSR (CSR format; also kept for the merge tile map)
    spx::DBuf rp, col, val, val32;
    // ELL (ELL format or HYB ELL part), column-major [width][ld]
    int64_t ell_w = 0, ell_ld = 0;
    spx::DBuf ell_col, ell_val, ell_val32;
    // COO (COO format or HYB COO part)
    int64_t coo_nnz = 0;
    spx::DBuf coo_row, coo_col, coo_val, coo_val32;
    // SpMV kernel selection
    int kernel = SPX_KERNEL_AUTO, kparam = 0;
    // merge-path tile map (CSR), rebuilt when the tile size changes
    spx::DBuf tiles;          // int2 per tile boundary
    int64_t tiles_items = 0;  // items per tile the map was built for
    int64_t ntiles = 0;
    int64_t nsplit = 0;       // boundaries that split a row (need the look-back)
    // row-block CSR: the most nonzeros in a tile of 128 rows (-1: not measured yet)
    int64_t rows_cap = -1;
    // row hints of the nnz-split CSR kernel (row holding nonzero g * hint_ipt)
    spx::DBuf hint;
    int hint_ipt = 0;
    // tiled nnz-split CSR: tile-transposed nonzeros (values per value array) and
    // granule descriptors, built on first use for granules of tc_ipt nonzeros
    spx::DBuf tc_col, tc_val, tc_val32, tc_row, tc_mask, empty_rows;
    int tc_ipt = 0, tc_val_ipt = 0, tc_val32_ipt = 0;
    int64_t n_empty = -1;
    // tiled nnz-split COO (COO format / HYB COO part): tile-transposed row, column and value arrays
    spx::DBuf ct_row, ct_col, ct_val, ct_val32;
    int ct_ipt = 0, ct_val_ipt = 0, ct_val32_ipt = 0;
    // COO tile map (COO format / HYB COO part)
    spx::DBuf coo_tiles;      // int per tile boundary
    int64_t coo_tiles_items = 0, coo_ntiles = 0, coo_nsplit = 0;
    // COO row-block kernel: first entry of each tile of 128 rows, and the most entries in a tile
    spx::DBuf coo_rowtiles;
    int64_t coo_rows_cap = -1;
    // per-tile carries, look-back flags, reduction scratch of the SpMV kernels
    spx::DBuf carry_row, carry_val, flags, partials;
    spx::DBuf ticket;  // unsigned counters for last-block detection
    // host staging for spx_spmv_host
    spx::DBuf stage_x, stage_y;
    // solver workspace (solvers.cu)
    spx::SolverWork *work = nullptr;
    // small systems: the matrix as a batch of one for the one-block solve route (solvers.cu)
    spx_batch *batch1 = nullptr;
    bool batch1_shadow = false;
    spx::DBuf small_out;  // result record of the cluster solves (cluster.cu)
    spx::DBuf cl_work;    // workspace of the one-cluster solve of a mid-size system (cluster.cu)
    int64_t solves = 0;   // spx_solve calls made on this matrix (solvers.cu: when to capture graphs)
};

namespace spx {

// ------------------------------------------------------------------ SpMV epilogue
// The SpMV kernels compute t_i = (A x)_i and store
//     y_i = alpha * t_i + beta * z_i          (z may be y itself or null: beta ignored)
// and, optionally, two dot products over the stored y:
//     d0 = sum_i w_i * y_i   (w != null)      d1 = sum_i y_i * y_i   (want_yy)
// reduced deterministically; the last block writes them to dots[0..1] and
// then runs the scalar update `fin` (solver bookkeeping, see solvers.cu).
template <class T> struct Epi {
    T alpha = T(1), beta = T(0);
    const T *z = nullptr;
    T *y = nullptr;
    const T *w = nullptr;
    bool want_yy = false;
    T *dots = nullptr;        // device, 2 entries; null = no dots
    int fin = 0;              // scalar update id (0 = none)
    void *fin_state = nullptr;
    const int *skip = nullptr;  // device flag: if *skip != 0 the kernel returns at once
};

// Launchers (spmv.cu).  All asynchronous on ctx->stream.
template <class T>
int spmv_launch(spx_ctx *ctx, const spx_matrix *A, const T *x, const Epi<T> &epi, bool use32 = false);

// Deterministic reductions and vector kernels (blas1.cu).
template <class T> int dot_launch(spx_ctx *ctx, int64_t n, const T *x, const T *y, T *result);
template <class T> int axpby_launch(spx_ctx *ctx, int64_t n, T alpha, const T *x, T beta, T *y);

// Tile map for merge-path CSR (spmv.cu).
int ensure_merge_tiles(spx_ctx *ctx, spx_matrix *A, int64_t tile_items, int64_t slack);

// Solver code of the ABI -> method, Jacobi flag, block-Jacobi block size (0: none),
// block-Jacobi adaptive storage.
int parse_solver_code(int code, int *solver, bool *jacobi, int *bs, bool *adaptive);

// Iterative refinement: FP32 inner iterations per outer cycle are capped, so an
// inner solve that stagnates (FP32 CGS on large systems) hands its correction
// back to the FP64 outer loop instead of running to the global limit.
constexpr int kIrInnerCap = 500;
// An inner CGS cycle also ends once its recurrence residual has gone this many
// iterations without falling below half of the level it last halved to
// (starting from 1 at x0 = 0).  CGS squares its residual polynomial, so a
// cycle that starts from a residual mixing smooth and rough components can
// grow it by orders of magnitude in FP32 and never recover; the outer FP64
// residual then restarts the inner solve from the true residual.
constexpr int kIrCgsStall = 20;

// Batched solves without graph capture, at a given block size (batch.cu), and
// the largest system the batched kernel holds (rows).
int batch_solve_direct(spx_ctx *ctx, spx_batch *B, const void *b, void *x, int solver, double tol, int64_t max_iter,
                       int precision, int block, spx_solve_info *infos);
int batch_max_rows(const spx_ctx *ctx);

// CG on one thread-block cluster for small CSR systems (cluster.cu); synchronous.
int cluster_cg_max_rows();
int cluster_cg_solve(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, double tol, int64_t maxit,
                     spx_solve_info *info);
// A whole solve (CG, BiCGSTAB or CGS; F64, F32 or MIXED) of a CSR system in one
// launch on one thread-block cluster, vectors in global memory (cluster.cu);
// synchronous.  SPX_ERR_UNSUPPORTED when no cluster fits the device.
int cluster_solve(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, int solver, double tol, int64_t maxit,
                  int precision, spx_solve_info *info);

}  // namespace spx
