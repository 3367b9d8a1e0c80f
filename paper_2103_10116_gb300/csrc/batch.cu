// batch.cu -- many independent small sparse systems solved by one persistent
// kernel launch (CG, BiCGSTAB or CGS, FP64, FP32, or FP32 inner iterations inside
// FP64 iterative refinement).
//
// Each thread block takes the next system from a device work queue (largest
// systems first, for load balance), solves it completely with block-level
// reductions (warp shuffles + shared memory, fixed order: deterministic), and
// writes the system's status.  Blocks never wait on one another, so no
// grid-wide synchronisation exists.  The vector that the SpMV gathers from
// (p for CG; p and s for BiCGSTAB, staged in turn) lives in shared memory;
// the other vectors live in a global workspace that stays in L2 while the
// block works on the system.  The launch sequence (queue reset, kernel,
// status read-back) is captured once as a CUDA graph and replayed.  The block
// size is chosen per batch by timing the candidates (spx_batch_tune).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "dev_common.cuh"
#include "krylov_rows.cuh"
#include "spx_internal.cuh"

struct spx_batch {
    spx_ctx *ctx = nullptr;
    int dtype = SPX_F64;
    int64_t nsys = 0, nrows = 0, nnz = 0, max_n = 0;
    std::vector<int64_t> row_off, nnz_off;
    spx::DBuf d_row_off, d_nnz_off, rp, col, val, val32, order;
    spx::DBuf work;      // 4 vectors of nrows doubles
    spx::DBuf out;       // per system: status (int), iters (long long), relres (double)
    spx::DBuf queue;     // work-queue counter
    void *host_out = nullptr;          // pinned copy of `out` for the captured graph (made on first use)
    std::vector<char> host_out_pageable;  // the same for one-shot solves, which copy synchronously
    int block = 0;       // chosen threads per system (0 = not tuned: heuristic)
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey[10] = {0};
};

namespace spx {

struct BOut {
    int *status;
    long long *iters;
    double *relres;
    int *cycles;  // refinement cycles (mixed precision), else 0
};

// per-system results on the device and in the host copy: status | iterations | residual | cycles
inline size_t bout_off_iters(int64_t nsys) { return round_up((size_t)nsys * 4, 256); }
inline size_t bout_off_relres(int64_t nsys) { return bout_off_iters(nsys) + round_up((size_t)nsys * 8, 256); }
inline size_t bout_off_cycles(int64_t nsys) { return bout_off_relres(nsys) + round_up((size_t)nsys * 8, 256); }
inline size_t bout_bytes(int64_t nsys) { return bout_off_cycles(nsys) + round_up((size_t)nsys * 4, 256); }

// The persistent kernel: each block takes the next system from the queue and
// solves it alone (krylov_rows.cuh, one block owning all rows).  The vector
// the products gather from lives in shared memory (smem_vec) or, for systems
// too large for it, in the global workspace (slots 6 and 7 of the eight per
// row; read through L1, the block being the only reader).  Launch bounds of
// 1024 threads per SM hold every variant at 64 registers without spills
// (without the bound, ptxas gave some variants 32 registers and spilled).
template <class T, int BLOCK, int SOLVER, bool MIXED>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK)
    k_batch(int64_t nsys, const int64_t *__restrict__ row_off, const int64_t *__restrict__ nnz_off,
            const int *__restrict__ rp_all, const int *__restrict__ col_all, const T *__restrict__ val_all,
            const float *__restrict__ val32_all, const int *__restrict__ order, const T *__restrict__ b_all,
            T *__restrict__ x_all, T *__restrict__ work, int64_t nrows, T tol, long long maxit, unsigned *queue,
            BOut out, int smem_vec)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ T red[BLOCK / 32];
    __shared__ float redf[BLOCK / 32];
    __shared__ int s_sys;
    for (;;) {
        if (threadIdx.x == 0) s_sys = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int q = s_sys;
        __syncthreads();
        if (q >= nsys) break;
        const int s = order[q];
        const int64_t ro = row_off[s];
        BlockRows<BLOCK> g((int)(row_off[s + 1] - ro));
        const SysOut o = solve_rows<T, BLOCK, SOLVER, MIXED>(
            g, rp_all + ro + s, col_all + nnz_off[s], val_all + nnz_off[s], MIXED ? val32_all + nnz_off[s] : nullptr,
            b_all + ro, x_all + ro, work, nrows, ro, smem_vec ? smem : nullptr, red, redf, tol, maxit);
        if (threadIdx.x == 0) {
            out.status[s] = o.status;
            out.iters[s] = o.iters;
            out.relres[s] = o.relres;
            out.cycles[s] = o.cycles;
        }
    }
}

namespace {

template <class T, int BLOCK, int SOLVER, bool MIXED>
int launch_batch_t(spx_ctx *ctx, spx_batch *B, const T *b, T *x, double tol, int64_t maxit, BOut out,
                   unsigned *queue)
{
    auto kern = k_batch<T, BLOCK, SOLVER, MIXED>;
    int smem = (int)(B->max_n * (MIXED ? 8 : sizeof(T)));
    const int smem_vec = smem <= ctx->max_smem_optin - 1024 ? 1 : 0;  // else the vector stays in global memory
    if (!smem_vec) smem = 0;
    // the opt-in only ever grows (smem_optin): the server's batch lanes launch this
    // kernel from several threads with different sizes, and lowering the limit
    // between another thread's opt-in and its launch got that launch refused
    SPX_TRY(smem_optin(reinterpret_cast<const void *>(kern), smem));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t grid = (int64_t)per_sm * ctx->grid_sms;
    if (grid > B->nsys) grid = B->nsys;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)BLOCK);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = ctx->stream;
    SPX_CUDA(cudaLaunchKernelEx(&cfg, kern, B->nsys, (const int64_t *)B->d_row_off.as<int64_t>(),
                                (const int64_t *)B->d_nnz_off.as<int64_t>(), (const int *)B->rp.as<int>(),
                                (const int *)B->col.as<int>(), (const T *)B->val.as<T>(),
                                (const float *)B->val32.as<float>(), (const int *)B->order.as<int>(), b, x,
                                B->work.as<T>(), B->nrows, (T)tol, (long long)maxit, queue, out, smem_vec));
    return SPX_OK;
}

template <class T, int SOLVER, bool MIXED>
int launch_batch_b(spx_ctx *ctx, spx_batch *B, int block, const T *b, T *x, double tol, int64_t maxit, BOut out,
                   unsigned *queue)
{
    switch (block) {
    case 128: return launch_batch_t<T, 128, SOLVER, MIXED>(ctx, B, b, x, tol, maxit, out, queue);
    case 256: return launch_batch_t<T, 256, SOLVER, MIXED>(ctx, B, b, x, tol, maxit, out, queue);
    case 512: return launch_batch_t<T, 512, SOLVER, MIXED>(ctx, B, b, x, tol, maxit, out, queue);
    case 1024: return launch_batch_t<T, 1024, SOLVER, MIXED>(ctx, B, b, x, tol, maxit, out, queue);
    default: return fail(SPX_ERR_INVALID, "batched block size must be 128, 256, 512 or 1024");
    }
}

int launch_batch(spx_ctx *ctx, spx_batch *B, int block, int solver, int precision, const void *b, void *x,
                 double tol, int64_t maxit)
{
    BOut out;
    out.status = B->out.as<int>();
    out.iters = reinterpret_cast<long long *>(B->out.as<char>() + bout_off_iters(B->nsys));
    out.relres = reinterpret_cast<double *>(B->out.as<char>() + bout_off_relres(B->nsys));
    out.cycles = reinterpret_cast<int *>(B->out.as<char>() + bout_off_cycles(B->nsys));
    unsigned *queue = B->queue.as<unsigned>();
    SPX_CUDA(cudaMemsetAsync(queue, 0, 4, ctx->stream));
    if (precision == SPX_PREC_MIXED) {
        const double *bd = static_cast<const double *>(b);
        double *xd = static_cast<double *>(x);
        if (solver == SPX_CG) return launch_batch_b<double, SPX_CG, true>(ctx, B, block, bd, xd, tol, maxit, out, queue);
        if (solver == SPX_CGS) return launch_batch_b<double, SPX_CGS, true>(ctx, B, block, bd, xd, tol, maxit, out, queue);
        return launch_batch_b<double, SPX_BICGSTAB, true>(ctx, B, block, bd, xd, tol, maxit, out, queue);
    }
    if (B->dtype == SPX_F64) {
        const double *bd = static_cast<const double *>(b);
        double *xd = static_cast<double *>(x);
        if (solver == SPX_CG) return launch_batch_b<double, SPX_CG, false>(ctx, B, block, bd, xd, tol, maxit, out, queue);
        if (solver == SPX_CGS) return launch_batch_b<double, SPX_CGS, false>(ctx, B, block, bd, xd, tol, maxit, out, queue);
        return launch_batch_b<double, SPX_BICGSTAB, false>(ctx, B, block, bd, xd, tol, maxit, out, queue);
    }
    const float *bf = static_cast<const float *>(b);
    float *xf = static_cast<float *>(x);
    if (solver == SPX_CG) return launch_batch_b<float, SPX_CG, false>(ctx, B, block, bf, xf, tol, maxit, out, queue);
    if (solver == SPX_CGS) return launch_batch_b<float, SPX_CGS, false>(ctx, B, block, bf, xf, tol, maxit, out, queue);
    return launch_batch_b<float, SPX_BICGSTAB, false>(ctx, B, block, bf, xf, tol, maxit, out, queue);
}

int default_block(const spx_batch *B)
{
    const double mean = B->nsys ? (double)B->nrows / (double)B->nsys : 0.0;
    if (mean <= 1500) return 128;
    if (mean <= 4000) return 256;
    return 512;
}

struct DevGuardB {
    int prev = -1;
    explicit DevGuardB(int d)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
        else prev = -1;
    }
    ~DevGuardB()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void batch_free(spx_batch *B)
{
    spx_ctx *c = B->ctx;
    DBuf *bufs[] = {&B->d_row_off, &B->d_nnz_off, &B->rp, &B->col, &B->val, &B->val32, &B->order,
                    &B->work,      &B->out,       &B->queue};
    for (DBuf *b : bufs) dbuf_free(c, *b);
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    if (B->host_out) cudaFreeHost(B->host_out);
}

__global__ void k_cast_f32(int64_t m, const double *__restrict__ a, float *__restrict__ o)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        o[k] = (float)a[k];
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" int spx_batch_create(spx_ctx *ctx, spx_batch **out, int dtype, int64_t nsys, const int64_t *row_off,
                                const int64_t *nnz_off, const int32_t *row_ptr, const int32_t *col_idx,
                                const void *values, unsigned flags)
{
    if (!ctx || !out || !row_off || !nnz_off || nsys < 0) return fail(SPX_ERR_INVALID, "spx_batch_create: bad argument");
    *out = nullptr;
    if (dtype != SPX_F64 && dtype != SPX_F32) return fail(SPX_ERR_INVALID, "spx_batch_create: bad dtype");
    if (row_off[0] != 0 || nnz_off[0] != 0) return fail(SPX_ERR_INVALID, "offsets must start at 0");
    int64_t max_n = 0;
    for (int64_t s = 0; s < nsys; ++s) {
        const int64_t n = row_off[s + 1] - row_off[s], z = nnz_off[s + 1] - nnz_off[s];
        if (n < 0 || z < 0) return fail(SPX_ERR_INVALID, "offsets must be non-decreasing");
        max_n = std::max(max_n, n);
    }
    const int64_t nrows = row_off[nsys], nnz = nnz_off[nsys];
    if (nrows + nsys > INT32_MAX || nnz > INT32_MAX) return fail(SPX_ERR_TOO_LARGE, "batch too large for int32 indices");
    if ((nrows > 0 && !row_ptr) || (nnz > 0 && (!col_idx || !values))) return fail(SPX_ERR_INVALID, "NULL array");
    DevGuardB g(ctx->device);
    spx_batch *B = new spx_batch();
    B->ctx = ctx;
    B->dtype = dtype;
    B->nsys = nsys;
    B->nrows = nrows;
    B->nnz = nnz;
    B->max_n = max_n;
    B->row_off.assign(row_off, row_off + nsys + 1);
    B->nnz_off.assign(nnz_off, nnz_off + nsys + 1);
    const size_t V = dtype == SPX_F64 ? 8 : 4;
    int st = SPX_OK;
    auto chk = [&](int s) {
        if (st == SPX_OK) st = s;
    };
    chk(dbuf_alloc(ctx, B->d_row_off, (size_t)(nsys + 1) * 8));
    chk(dbuf_alloc(ctx, B->d_nnz_off, (size_t)(nsys + 1) * 8));
    chk(dbuf_alloc(ctx, B->rp, (size_t)(nrows + nsys) * 4));
    chk(dbuf_alloc(ctx, B->col, (size_t)nnz * 4));
    chk(dbuf_alloc(ctx, B->val, (size_t)nnz * V));
    chk(dbuf_alloc(ctx, B->order, (size_t)nsys * 4));
    chk(dbuf_alloc(ctx, B->work, (size_t)nrows * 8 * 8));
    chk(dbuf_alloc(ctx, B->out, bout_bytes(nsys)));
    chk(dbuf_alloc(ctx, B->queue, 64));
    if (st == SPX_OK && (flags & SPX_MIXED_SHADOW) && dtype == SPX_F64) chk(dbuf_alloc(ctx, B->val32, (size_t)nnz * 4));
    // largest systems first
    std::vector<int> order((size_t)nsys);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return row_off[a + 1] - row_off[a] > row_off[c + 1] - row_off[c];
    });
    if (st == SPX_OK) {
        cudaError_t e = cudaMemcpyAsync(B->d_row_off.p, row_off, (size_t)(nsys + 1) * 8, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_nnz_off.p, nnz_off, (size_t)(nsys + 1) * 8, cudaMemcpyHostToDevice, ctx->stream);
        const cudaMemcpyKind kind = (flags & SPX_HOST_INPUT) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        if (e == cudaSuccess && nrows + nsys > 0)
            e = cudaMemcpyAsync(B->rp.p, row_ptr, (size_t)(nrows + nsys) * 4, kind, ctx->stream);
        if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(B->col.p, col_idx, (size_t)nnz * 4, kind, ctx->stream);
        if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(B->val.p, values, (size_t)nnz * V, kind, ctx->stream);
        if (e == cudaSuccess && nsys > 0) e = cudaMemcpyAsync(B->order.p, order.data(), (size_t)nsys * 4, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess && B->val32.p && nnz > 0) {
            k_cast_f32<<<ctx->grid_sms * 8, 256, 0, ctx->stream>>>(nnz, B->val.as<double>(), B->val32.as<float>());
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "spx_batch_create");
    }
    if (st != SPX_OK) {
        std::string msg = spx_last_error();
        batch_free(B);
        cudaStreamSynchronize(ctx->stream);
        delete B;
        set_error(msg);
        return st;
    }
    *out = B;
    return SPX_OK;
}

extern "C" int spx_batch_destroy(spx_batch *B)
{
    if (!B) return SPX_OK;
    DevGuardB g(B->ctx->device);
    cudaStreamSynchronize(B->ctx->stream);
    batch_free(B);
    cudaStreamSynchronize(B->ctx->stream);
    delete B;
    return SPX_OK;
}

namespace {
int batch_solve_impl(spx_ctx *ctx, spx_batch *B, const void *b, void *x, int solver, double tol, int64_t max_iter,
                     int precision, spx_solve_info *infos, int block, bool use_graph)
{
    if (precision == SPX_PREC_MIXED && (B->dtype != SPX_F64 || !B->val32.p))
        return fail(SPX_ERR_UNSUPPORTED, "mixed precision needs an FP64 batch created with SPX_MIXED_SHADOW");
    if (precision == SPX_PREC_F64 && B->dtype != SPX_F64) return fail(SPX_ERR_UNSUPPORTED, "precision must match dtype");
    if (precision == SPX_PREC_F32 && B->dtype != SPX_F32) return fail(SPX_ERR_UNSUPPORTED, "precision must match dtype");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t out_bytes = bout_bytes(B->nsys);
    uint64_t key[10] = {(uint64_t)(uintptr_t)b, (uint64_t)(uintptr_t)x, (uint64_t)solver, (uint64_t)precision, 0,
                        (uint64_t)max_iter, (uint64_t)block, (uint64_t)(uintptr_t)ctx->stream,
                        (uint64_t)ctx->grid_sms, 0};
    std::memcpy(&key[4], &tol, 8);
    bool same = use_graph && B->gexec;
    for (int i = 0; i < 10 && same; ++i) same = B->gkey[i] == key[i];
    // the result read-back: into pinned memory when it is part of a captured graph;
    // a one-shot batch (the request server builds one per launch) copies into
    // pageable memory and spares a pinned allocation per batch
    if (use_graph && !B->host_out) SPX_CUDA(cudaMallocHost(&B->host_out, out_bytes + 64));
    if (!use_graph) B->host_out_pageable.resize(out_bytes + 64);
    void *hout = use_graph ? B->host_out : static_cast<void *>(B->host_out_pageable.data());
    auto body = [&]() -> int {
        SPX_TRY(launch_batch(ctx, B, block, solver, precision, b, x, tol, max_iter));
        SPX_CUDA(cudaMemcpyAsync(hout, B->out.p, out_bytes, cudaMemcpyDeviceToHost, ctx->stream));
        return SPX_OK;
    };
    if (same) {
        SPX_CUDA(cudaGraphLaunch(B->gexec, ctx->stream));
    } else if (use_graph) {
        // capture the launch sequence on the private stream, replay it on ctx->stream
        if (B->gexec) {
            cudaGraphExecDestroy(B->gexec);
            B->gexec = nullptr;
        }
        cudaStream_t user = ctx->stream;
        ctx->stream = ctx->capture_stream;
        cudaError_t e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeRelaxed);
        int st = e == cudaSuccess ? body() : SPX_OK;
        cudaGraph_t g = nullptr;
        cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ctx->capture_stream, &g) : e;
        ctx->stream = user;
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        if (st != SPX_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&B->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        std::memcpy(B->gkey, key, sizeof(key));
        SPX_CUDA(cudaGraphLaunch(B->gexec, ctx->stream));
    } else {
        SPX_TRY(body());
    }
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (infos) {
        const char *h = static_cast<const char *>(hout);
        const int *stv = reinterpret_cast<const int *>(h);
        const long long *itv = reinterpret_cast<const long long *>(h + bout_off_iters(B->nsys));
        const double *rv = reinterpret_cast<const double *>(h + bout_off_relres(B->nsys));
        const int *cyv = reinterpret_cast<const int *>(h + bout_off_cycles(B->nsys));
        for (int64_t s = 0; s < B->nsys; ++s) {
            std::memset(&infos[s], 0, sizeof(infos[s]));
            infos[s].status = stv[s];
            infos[s].iterations = itv[s];
            infos[s].relres_recurrence = rv[s];
            infos[s].relres_true = rv[s];
            infos[s].time_ms = ms;
            if (precision == SPX_PREC_MIXED) {
                infos[s].inner_iterations = itv[s];
                infos[s].restarts = cyv[s];  // refinement cycles, as the per-system path reports them
            }
        }
    }
    return SPX_OK;
}
}  // namespace

namespace spx {
// One-shot batches (the request server builds a new batch per launch): no
// graph capture, block size given by the caller.
int batch_solve_direct(spx_ctx *ctx, spx_batch *B, const void *b, void *x, int solver, double tol, int64_t max_iter,
                       int precision, int block, spx_solve_info *infos)
{
    if (B->nsys == 0) return SPX_OK;
    return batch_solve_impl(ctx, B, b, x, solver, tol, max_iter, precision, infos, block, false);
}

int batch_max_rows(const spx_ctx *ctx) { return (ctx->max_smem_optin - 1024) / 8; }
}  // namespace spx

extern "C" int spx_batch_solve(spx_ctx *ctx, spx_batch *B, const void *b, void *x, int solver, double tol,
                               int64_t max_iter, int precision, spx_solve_info *infos)
{
    if (!ctx || !B || (B->nrows > 0 && (!b || !x))) return fail(SPX_ERR_INVALID, "spx_batch_solve: NULL argument");
    if (solver != SPX_CG && solver != SPX_BICGSTAB && solver != SPX_CGS)
        return fail(SPX_ERR_UNSUPPORTED, "batched solver must be CG, BiCGSTAB or CGS");
    if (!(tol >= 0.0) || max_iter < 0) return fail(SPX_ERR_INVALID, "spx_batch_solve: bad tol or max_iter");
    if (B->nsys == 0) return SPX_OK;
    DevGuardB g(ctx->device);
    const int block = B->block ? B->block : default_block(B);
    return batch_solve_impl(ctx, B, b, x, solver, tol, max_iter, precision, infos, block, true);
}

extern "C" int spx_batch_tune(spx_ctx *ctx, spx_batch *B, int solver, int precision, int *chosen)
{
    if (!ctx || !B) return fail(SPX_ERR_INVALID, "spx_batch_tune: NULL argument");
    if (solver != SPX_CG && solver != SPX_BICGSTAB && solver != SPX_CGS)
        return fail(SPX_ERR_UNSUPPORTED, "batched solver must be CG, BiCGSTAB or CGS");
    if (B->nsys == 0) {
        if (chosen) *chosen = default_block(B);
        return SPX_OK;
    }
    DevGuardB g(ctx->device);
    // time every candidate on the batch itself: b = A 1 (built on the fly from a
    // ones vector would need an SpMV; a unit right-hand side is enough to time)
    const size_t V = precision == SPX_PREC_F32 ? 4 : 8;
    DBuf bb, xx;
    SPX_TRY(dbuf_alloc(ctx, bb, (size_t)B->nrows * V));
    SPX_TRY(dbuf_alloc(ctx, xx, (size_t)B->nrows * V));
    if (V == 8) {
        std::vector<double> ones((size_t)B->nrows, 1.0);
        SPX_CUDA(cudaMemcpyAsync(bb.p, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
        SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    } else {
        std::vector<float> ones((size_t)B->nrows, 1.0f);
        SPX_CUDA(cudaMemcpyAsync(bb.p, ones.data(), ones.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
        SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    const int cands[4] = {128, 256, 512, 1024};
    double best = 1e300;
    int best_b = default_block(B);
    cudaEvent_t e0, e1;
    SPX_CUDA(cudaEventCreate(&e0));
    SPX_CUDA(cudaEventCreate(&e1));
    for (int c : cands) {
        float msum = 0.f;
        int ok = SPX_OK;
        for (int rep = 0; rep < 2 && ok == SPX_OK; ++rep) {
            SPX_CUDA(cudaMemsetAsync(xx.p, 0, (size_t)B->nrows * V, ctx->stream));
            SPX_CUDA(cudaEventRecord(e0, ctx->stream));
            ok = launch_batch(ctx, B, c, solver, precision, bb.p, xx.p, 1e-10, 10000);
            SPX_CUDA(cudaEventRecord(e1, ctx->stream));
            SPX_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) msum += ms;
        }
        if (ok != SPX_OK) continue;  // e.g. a block shape that does not fit
        if (msum < best) {
            best = msum;
            best_b = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dbuf_free(ctx, bb);
    dbuf_free(ctx, xx);
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    B->block = best_b;
    if (B->gexec) {
        cudaGraphExecDestroy(B->gexec);
        B->gexec = nullptr;
    }
    if (chosen) *chosen = best_b;
    return SPX_OK;
}
