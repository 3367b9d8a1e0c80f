// server.cu -- continuous-batching solve server.
//
// Requests (a CSR operator in host memory, a right-hand side, an output
// buffer, solver settings) enter a FIFO queue.  A request is admitted to a
// free slot as soon as its device footprint (the uploaded matrix arrays and
// the library's copy, FP32 shadow, the tiled copy of heavy-tailed rows, solver
// workspace, b and x) fits in what the byte budget has left; while it
// runs, later requests keep being admitted into the other slots, so solves
// of different sizes overlap on the GPU.  Each slot is a worker thread with
// its own context and CUDA stream: the operator is uploaded, solved on the
// device (the same spx_solve path a single caller uses) and the solution is
// copied back; then the slot's memory returns to the budget and the next
// queued request is admitted.  Completion records (status, iterations,
// residual, submit / admit / finish times) are collected with
// spx_server_poll.
//
// Small and mid-size CG / BiCGSTAB / CGS requests (up to batch_rows rows) do
// not take a slot of their own: batch
// lanes (further worker threads, each with its own context and stream) take
// every queued small request with the same solver settings and size class
// that fits the budget, stage them back to back in pinned host memory, and
// solve them all with one launch of the persistent batched kernel.  A request
// arriving while such a batch runs is picked up by the next free lane, so
// batches overlap each other and the large solves.
//
// Slot requests of CG / BiCGSTAB / CGS (unpreconditioned) on CSR operators of
// at most cluster_rows rows whose rows hold at most 8 entries on average (the
// 7-point stencil's class) may run the whole solve in one launch on one
// thread-block cluster (SPX_SOLVE_ONE_CLUSTER): on the general path such a
// solve is hundreds of dependent launches of kernels with a few microseconds
// of work each (and a request solves its matrix once, too few times to repay
// capturing CUDA graphs).  Sixteen concurrent solves of a 27 000-row 7-point
// stencil (mixed CG to 1e-8) completed 1.5-1.7x as many solves per second on
// clusters as on the general path launching its kernels directly; on the
// serving trace the solve phases of the 25 000 - 100 000-row requests summed to
// 128 s with the route and 187 s without.  At 97 000 rows the two broke even,
// and for longer rows with random columns the cluster route was slower at every
// size measured, so the rule takes short rows of at most 65 536 rows.  The
// decision reads the row statistics of the request's own matrix, so it does not
// depend on other requests.
//
// Results do not depend on what else runs: every kernel of a solve uses only
// its own matrix's and slot's scratch, with fixed-order reductions; a
// batched request always runs at the block size of its size class, with
// block-local reductions, whatever it is batched with.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "spx_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kBatchLanes = 4;
constexpr int64_t kServeBatchRows = 24576;     // default size limit of batched requests
constexpr int64_t kServeBatchRowsMax = 262144; // the largest limit spx_server_set_batching accepts
constexpr int64_t kServeClusterRows = 65536;    // default size limit of one-cluster requests
constexpr int64_t kServeClusterRowsMax = 1 << 30;
constexpr double kServeClusterMeanLen = 8.0;    // ... and their largest mean row length
// Slot grids are sized for a share of the device's SMs, so that the kernels of
// concurrent slots run side by side (spx_ctx_set_grid_sms).  Sixteen concurrent
// mixed solves to 1e-8 of one matrix (solves per second at whole-device / half /
// quarter / eighth grids): 7-point stencils of 250 000 rows 534 / 750 / 839 /
// 743, of 512 000 rows 292 / 376 / 391 / 353, of 10^6 rows 154 / 175 / 179 /
// 166; rows of 20 random columns, 10^5 rows 1092 / 1277 / 1233 / 1039,
// 3 x 10^5 rows 506 / 521 / 490 / 414.  The rule (-1) takes a quarter for short
// rows and a half for long ones.  On the mixed serving trace no setting beat
// whole-device grids beyond run-to-run variation (whole device 397-403 solves
// per second, the rule 382, a half 414, a quarter 374), so the default is 0.
constexpr int kServeShortRowShare = 4;
constexpr int kServeLongRowShare = 2;
constexpr size_t kMaxBatchSystems = 4096;
constexpr int64_t kMaxBatchRows = 16 << 20;

struct Request {
    int64_t id;
    bool batched;
    bool one_cluster;  // a slot request solved on one thread-block cluster
    bool cluster_auto; // ... if its matrix's mean row length allows (not asked for by the caller)
    int block;  // threads per system when batched
    int64_t n, nnz;
    const int32_t *rp, *col;
    const double *val, *b;
    double *x;
    spx_matrix *A;  // resident operator (spx_server_submit_matrix), else null
    int solver, precision, restart;
    double tol;
    int64_t max_iter;
    size_t tiled;  // the general path's tile-transposed copy of the nonzeros (heavy-tailed rows), else 0
    size_t footprint;
    Clock::time_point t_submit, t_admit, t_done;
    double upload_ms, setup_ms, solve_ms, download_ms;  // phases after admission
    spx_solve_info info;
    int error;
};

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct spx_server {
    int device = 0;
    size_t budget = 0, in_use = 0;
    int slots = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;   // requests that take a slot of their own
    std::deque<Request *> bqueue;  // requests for the batch lanes
    int64_t batch_rows = 0, batch_rows_limit = 0;
    int64_t cluster_rows = 0;
    int slot_sms = 0;  // grid share of the slots' contexts (spx_ctx_set_grid_sms; 0: the whole device;
                       // -1: by the request's mean row length, kServeShortRowShare / kServeLongRowShare)
    std::vector<Request *> done;
    std::vector<std::thread> workers;
    std::vector<const spx_matrix *> busy;  // resident operators with a request running
    std::atomic<bool> stop{false};
    int64_t next_id = 1;
    int active = 0;
    Clock::time_point t0 = Clock::now();
    std::string worker_error;
};

namespace spx {

// Device bytes a request needs while it runs (upper estimate).  An uploaded
// operator counts twice: the worker's upload buffers and the library's own
// copy of the matrix coexist while the matrix is built (the upload buffers are
// freed before the solve allocates its workspace; counting both at once keeps
// the estimate an upper bound).  A resident operator (uploaded = false) is the
// caller's and counts nothing.
size_t request_footprint(int64_t n, int64_t nnz, bool uploaded, int solver, int precision, int restart)
{
    const size_t csr = uploaded ? 2 * ((size_t)nnz * 12 + (size_t)(n + 1) * 4) : 0;
    const size_t shadow = uploaded && precision == SPX_PREC_MIXED ? (size_t)nnz * 4 : 0;
    size_t vecs;
    const size_t V = precision == SPX_PREC_F32 ? 4 : 8;
    const int nv = solver == SPX_CG ? 4 : solver == SPX_BICGSTAB ? 7 : solver == SPX_CGS ? 8 : restart + 2;
    if (precision == SPX_PREC_MIXED) vecs = (size_t)n * (8 * 4 + 4 * (nv + 2)) + (size_t)n * 16;
    else vecs = (size_t)n * V * nv;
    return csr + shadow + vecs + (size_t)n * 16 /* b, x */ + (1u << 20);
}

// Device bytes of the tile-transposed copy of the nonzeros that the SpMV of a
// CSR matrix with heavy-tailed rows builds on first use (the automatic kernel
// choice takes the tiled nnz-split kernel when the longest row exceeds four
// times the mean plus 8): column indices and FP64 values, the FP32 values as
// well in mixed precision, padded to whole chunks of 32 x 32 nonzeros, plus the
// granule descriptors and the list of empty rows.  0 for other matrices, whose
// kernels read the CSR arrays in place.  row_ptr: the request's n + 1 host row
// offsets (read only here, before the request is queued).
size_t tiled_copy_bytes(int64_t n, int64_t nnz, const int32_t *row_ptr, int precision)
{
    if (n <= 0 || nnz <= 0) return 0;
    int64_t mx = 0;
    for (int64_t i = 0; i < n; ++i) mx = std::max<int64_t>(mx, (int64_t)row_ptr[i + 1] - (int64_t)row_ptr[i]);
    const double mean = (double)nnz / (double)n;
    if ((double)mx <= 4.0 * mean + 8.0) return 0;
    constexpr int64_t kChunk = 32 * 32;
    const size_t total = (size_t)((nnz + kChunk - 1) / kChunk * kChunk);
    const size_t per_nz = 4 + 8 + (precision == SPX_PREC_MIXED ? 4 : 0);
    return total * per_nz + (total / 32 + 1) * 8 + (size_t)n * 4 + 64;
}

// the same for a request solved on one cluster: its workspace is 64 bytes per row
size_t cluster_footprint(int64_t n, int64_t nnz, bool uploaded, int precision)
{
    const size_t csr = uploaded ? 2 * ((size_t)nnz * 12 + (size_t)(n + 1) * 4) : 0;
    const size_t shadow = uploaded && precision == SPX_PREC_MIXED ? (size_t)nnz * 4 : 0;
    return csr + shadow + (size_t)n * 64 + (size_t)n * 16 + (1u << 20);
}

// Route of a request: the batch lanes, a slot with the one-cluster solve, or a
// slot with the general path.  code: the solver code with SPX_SOLVE_ONE_CLUSTER
// removed; asked: the caller set that flag.
void route_request(spx_server *S, Request *R, int code, bool asked, bool csr)
{
    const bool plain = code == SPX_CG || code == SPX_BICGSTAB || code == SPX_CGS;  // unpreconditioned
    std::lock_guard<std::mutex> lk(S->mu);
    R->batched = !asked && R->A == nullptr && plain &&
                 (R->precision == SPX_PREC_F64 || R->precision == SPX_PREC_MIXED) && R->n <= S->batch_rows;
    R->one_cluster = asked || (!R->batched && plain && csr && R->n <= S->cluster_rows);
    R->cluster_auto = R->one_cluster && !asked;
}

// Device bytes of a routed request: the route's workspace; a request whose
// route waits for its row statistics reserves the larger of the two.
size_t routed_footprint(const Request *R, int base_solver, bool jacobi, int bs, bool adaptive, bool resident)
{
    const size_t general = request_footprint(R->n, R->nnz, !resident, base_solver, R->precision, R->restart) +
                           (resident ? 0 : R->tiled) +
                           (jacobi ? (size_t)R->n * 24 : 0) +                     // M^-1 and the preconditioned vectors
                           (size_t)R->n * (size_t)bs * (adaptive ? 12 : 8);       // block-Jacobi inverses
    if (!R->one_cluster) return general;
    const size_t cl = cluster_footprint(R->n, R->nnz, !resident, R->precision);
    return R->cluster_auto ? std::max(cl, general) : cl;
}

// The request a free slot admits next: the first queued request whose resident
// operator (if any) is not in use by a running request -- two solves on one
// handle would share its workspace -- provided its footprint fits what the
// budget has left (FIFO: a request that does not fit blocks the ones after it).
// Null if none can start now.  Called with S->mu held.
static std::deque<Request *>::iterator next_admissible(spx_server *S)
{
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        const Request *R = *it;
        if (R->A && std::find(S->busy.begin(), S->busy.end(), R->A) != S->busy.end()) continue;
        return S->in_use + R->footprint <= S->budget ? it : S->queue.end();
    }
    return S->queue.end();
}

static void worker_main(spx_server *S)
{
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    spx_ctx *ctx = nullptr;
    if (spx_ctx_create(&ctx, S->device, st, nullptr, nullptr, nullptr) != SPX_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->worker_error = spx_last_error();
        return;
    }
    for (;;) {
        Request *R = nullptr;
        int sms = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop.load() || next_admissible(S) != S->queue.end(); });
            if (S->stop.load()) break;
            auto it = next_admissible(S);
            if (it == S->queue.end()) continue;
            R = *it;
            S->queue.erase(it);
            S->in_use += R->footprint;
            S->active += 1;
            if (R->A) S->busy.push_back(R->A);
            R->t_admit = Clock::now();
            sms = S->slot_sms;
        }
        S->cv_work.notify_all();  // another slot may admit the next request too
        int err = SPX_OK;
        spx_matrix *A = R->A;
        void *bd = nullptr, *xd = nullptr, *rpd = nullptr, *cold = nullptr, *vald = nullptr;
        std::memset(&R->info, 0, sizeof(R->info));
        const size_t vb = (size_t)R->n * 8;
        // upload: the operator (unless resident) and b
        if (!R->A) {
            if (cudaMallocAsync(&rpd, (size_t)(R->n + 1) * 4 + 16, st) != cudaSuccess ||
                cudaMallocAsync(&cold, (size_t)R->nnz * 4 + 16, st) != cudaSuccess ||
                cudaMallocAsync(&vald, (size_t)R->nnz * 8 + 16, st) != cudaSuccess)
                err = SPX_ERR_OOM;
            if (err == SPX_OK &&
                (cudaMemcpyAsync(rpd, R->rp, (size_t)(R->n + 1) * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                 (R->nnz > 0 && cudaMemcpyAsync(cold, R->col, (size_t)R->nnz * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
                 (R->nnz > 0 && cudaMemcpyAsync(vald, R->val, (size_t)R->nnz * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)))
                err = SPX_ERR_CUDA;
        }
        if (err == SPX_OK && cudaMallocAsync(&bd, vb + 16, st) != cudaSuccess) err = SPX_ERR_OOM;
        if (err == SPX_OK && cudaMallocAsync(&xd, vb + 16, st) != cudaSuccess) err = SPX_ERR_OOM;
        if (err == SPX_OK && cudaMemcpyAsync(bd, R->b, vb, cudaMemcpyHostToDevice, st) != cudaSuccess) err = SPX_ERR_CUDA;
        if (err == SPX_OK && cudaMemsetAsync(xd, 0, vb, st) != cudaSuccess) err = SPX_ERR_CUDA;
        cudaStreamSynchronize(st);
        const auto t_up = Clock::now();
        // set-up: validation, statistics and the library's own copy of the operator
        if (err == SPX_OK && !R->A)
            err = spx_matrix_create(ctx, &A, SPX_CSR, SPX_F64, R->n, R->n, R->nnz, (const int32_t *)rpd,
                                    (const int32_t *)cold, vald, SPX_F64, -1,
                                    R->precision == SPX_PREC_MIXED ? SPX_MIXED_SHADOW : 0u);
        cudaStreamSynchronize(st);
        if (rpd) cudaFreeAsync(rpd, st);
        if (cold) cudaFreeAsync(cold, st);
        if (vald) cudaFreeAsync(vald, st);
        const auto t_setup = Clock::now();
        if (err == SPX_OK && R->cluster_auto) R->one_cluster = A->mean_len <= kServeClusterMeanLen;
        if (err == SPX_OK) {  // the grid share: the server's setting, else by the operator's row length
            const bool short_rows = A->mean_len <= kServeClusterMeanLen;
            spx_ctx_set_grid_sms(ctx, sms >= 0 ? sms : ctx->sm_count / (short_rows ? kServeShortRowShare : kServeLongRowShare),
                                 nullptr);
        }
        if (err == SPX_OK)
            err = spx_solve(ctx, A, bd, xd, R->solver | (R->one_cluster ? SPX_SOLVE_ONE_CLUSTER : 0), R->tol,
                            R->max_iter, R->restart, R->precision, &R->info);
        cudaStreamSynchronize(st);
        const auto t_solve = Clock::now();
        if (err == SPX_OK && cudaMemcpyAsync(R->x, xd, vb, cudaMemcpyDeviceToHost, st) != cudaSuccess) err = SPX_ERR_CUDA;
        cudaStreamSynchronize(st);
        const auto t_down = Clock::now();
        if (A && !R->A) spx_matrix_destroy(A);
        if (bd) cudaFreeAsync(bd, st);
        if (xd) cudaFreeAsync(xd, st);
        cudaStreamSynchronize(st);
        R->error = err;
        R->upload_ms = ms_between(R->t_admit, t_up);
        R->setup_ms = ms_between(t_up, t_setup);
        R->solve_ms = ms_between(t_setup, t_solve);
        R->download_ms = ms_between(t_solve, t_down);
        R->t_done = Clock::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->in_use -= R->footprint;
            S->active -= 1;
            if (R->A) S->busy.erase(std::find(S->busy.begin(), S->busy.end(), R->A));
            S->done.push_back(R);
        }
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    spx_ctx_destroy(ctx);
    cudaStreamDestroy(st);
}

// threads per system of a batched request and its size class: functions of
// its own size only.  Requests are batched within a class, so a small request
// does not wait for a large one in the same launch; above 24 576 rows (a
// limit raised by spx_server_set_batching) the batched kernel keeps its
// gathered vector in global memory instead of shared memory.  The default
// stays at 24 576: on the serving trace, batching requests of up to 131 072
// rows (one SM each, their operators gathered into pinned staging by the
// lane's thread) took 147 s to drain against 50 s.
static int batch_block_for(int64_t n) { return n <= 1024 ? 128 : n <= 4096 ? 256 : n <= 8192 ? 512 : 1024; }
static int batch_class_for(int64_t n)
{
    return n <= 1024 ? 0 : n <= 4096 ? 1 : n <= 8192 ? 2 : n <= 24576 ? 3 : n <= 65536 ? 4 : 5;
}

static bool same_batch_key(const Request *a, const Request *b)
{
    return a->solver == b->solver && a->precision == b->precision && a->tol == b->tol &&
           a->max_iter == b->max_iter && a->block == b->block && batch_class_for(a->n) == batch_class_for(b->n);
}

// row_ptr monotone from 0 to nnz, columns in [0, n)
static bool csr_ok(const Request *R)
{
    if (R->rp[0] != 0 || R->rp[R->n] != R->nnz) return false;
    for (int64_t i = 0; i < R->n; ++i)
        if (R->rp[i + 1] < R->rp[i]) return false;
    for (int64_t k = 0; k < R->nnz; ++k)
        if (R->col[k] < 0 || R->col[k] >= R->n) return false;
    return true;
}

struct Pinned {
    void *p = nullptr;
    size_t cap = 0;
    bool reserve(size_t bytes)
    {
        if (bytes <= cap) return true;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        const size_t want = std::max(bytes, cap + cap / 2);
        if (cudaHostAlloc(&p, want, cudaHostAllocDefault) != cudaSuccess) return false;
        cap = want;
        return true;
    }
    ~Pinned()
    {
        if (p) cudaFreeHost(p);
    }
};

// Solve the requests rs (same solver settings) as one batch; per-request
// errors (an invalid operator) are set in R->error, the batch's own error is
// returned.
static int run_batch(spx_ctx *ctx, cudaStream_t st, Pinned &stage, std::vector<Request *> &rs, double *phase_ms)
{
    const auto t_start = Clock::now();
    std::vector<Request *> ok;
    for (Request *R : rs) {
        std::memset(&R->info, 0, sizeof(R->info));
        R->error = csr_ok(R) ? SPX_OK : SPX_ERR_INVALID;
        if (R->error == SPX_OK) ok.push_back(R);
    }
    if (ok.empty()) return SPX_OK;
    const int64_t ns = (int64_t)ok.size();
    int64_t rows = 0, nnz = 0;
    for (Request *R : ok) {
        rows += R->n;
        nnz += R->nnz;
    }
    const size_t o_row = 0, o_nnz = round_up((size_t)(ns + 1) * 8, 256);
    const size_t o_rp = o_nnz + round_up((size_t)(ns + 1) * 8, 256);
    const size_t o_col = o_rp + round_up((size_t)(rows + ns) * 4, 256);
    const size_t o_val = o_col + round_up((size_t)nnz * 4, 256);
    const size_t o_b = o_val + round_up((size_t)nnz * 8, 256);
    const size_t total = o_b + round_up((size_t)rows * 8, 256);
    if (!stage.reserve(total)) return fail(SPX_ERR_OOM, "pinned staging for a batch");
    char *h = static_cast<char *>(stage.p);
    int64_t *row_off = reinterpret_cast<int64_t *>(h + o_row), *nnz_off = reinterpret_cast<int64_t *>(h + o_nnz);
    int32_t *rp = reinterpret_cast<int32_t *>(h + o_rp), *col = reinterpret_cast<int32_t *>(h + o_col);
    double *val = reinterpret_cast<double *>(h + o_val), *b = reinterpret_cast<double *>(h + o_b);
    row_off[0] = nnz_off[0] = 0;
    for (int64_t s = 0; s < ns; ++s) {
        const Request *R = ok[(size_t)s];
        std::memcpy(rp + row_off[s] + s, R->rp, (size_t)(R->n + 1) * 4);
        std::memcpy(col + nnz_off[s], R->col, (size_t)R->nnz * 4);
        std::memcpy(val + nnz_off[s], R->val, (size_t)R->nnz * 8);
        std::memcpy(b + row_off[s], R->b, (size_t)R->n * 8);
        row_off[s + 1] = row_off[s] + R->n;
        nnz_off[s + 1] = nnz_off[s] + R->nnz;
    }
    const Request *h0 = ok[0];
    const auto t_staged = Clock::now();
    spx_batch *B = nullptr;
    int err = spx_batch_create(ctx, &B, SPX_F64, ns, row_off, nnz_off, rp, col, val,
                               SPX_HOST_INPUT | (h0->precision == SPX_PREC_MIXED ? SPX_MIXED_SHADOW : 0u));
    void *bd = nullptr, *xd = nullptr;
    const size_t vb = (size_t)rows * 8;
    if (err == SPX_OK && cudaMallocAsync(&bd, vb + 16, st) != cudaSuccess) err = fail(SPX_ERR_OOM, "batch b");
    if (err == SPX_OK && cudaMallocAsync(&xd, vb + 16, st) != cudaSuccess) err = fail(SPX_ERR_OOM, "batch x");
    if (err == SPX_OK && cudaMemcpyAsync(bd, b, vb, cudaMemcpyHostToDevice, st) != cudaSuccess) err = SPX_ERR_CUDA;
    if (err == SPX_OK && cudaMemsetAsync(xd, 0, vb, st) != cudaSuccess) err = SPX_ERR_CUDA;
    cudaStreamSynchronize(st);
    const auto t_up = Clock::now();
    std::vector<spx_solve_info> infos((size_t)ns);
    if (err == SPX_OK)
        err = batch_solve_direct(ctx, B, bd, xd, h0->solver, h0->tol, h0->max_iter, h0->precision, h0->block,
                                 infos.data());
    const auto t_solved = Clock::now();
    // the solve has synchronised the stream: b's staging is free for x
    if (err == SPX_OK && cudaMemcpyAsync(b, xd, vb, cudaMemcpyDeviceToHost, st) != cudaSuccess) err = SPX_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess && err == SPX_OK) err = SPX_ERR_CUDA;
    // phases of the whole batch, reported for each of its requests: gathering the
    // operators into pinned staging (set-up), upload and device build, the solve,
    // the download
    phase_ms[1] = ms_between(t_start, t_staged);
    phase_ms[0] = ms_between(t_staged, t_up);
    phase_ms[2] = ms_between(t_up, t_solved);
    phase_ms[3] = ms_between(t_solved, Clock::now());
    if (err == SPX_OK) {
        for (int64_t s = 0; s < ns; ++s) {
            Request *R = ok[(size_t)s];
            std::memcpy(R->x, b + row_off[s], (size_t)R->n * 8);
            R->info = infos[(size_t)s];
        }
    }
    if (B) spx_batch_destroy(B);
    if (bd) cudaFreeAsync(bd, st);
    if (xd) cudaFreeAsync(xd, st);
    cudaStreamSynchronize(st);
    return err;
}

static void lane_main(spx_server *S)
{
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    spx_ctx *ctx = nullptr;
    if (spx_ctx_create(&ctx, S->device, st, nullptr, nullptr, nullptr) != SPX_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->worker_error = spx_last_error();
        return;
    }
    Pinned stage;
    for (;;) {
        std::vector<Request *> take;
        size_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                return S->stop.load() ||
                       (!S->bqueue.empty() && S->in_use + S->bqueue.front()->footprint <= S->budget);
            });
            if (S->stop.load()) break;
            if (S->bqueue.empty() || S->in_use + S->bqueue.front()->footprint > S->budget) continue;
            // the head request and every later one of its kind that still fits, in arrival order
            const Request *head = S->bqueue.front();
            int64_t rows = 0;
            for (auto it = S->bqueue.begin(); it != S->bqueue.end();) {
                Request *R = *it;
                if (!same_batch_key(R, head)) {
                    ++it;
                    continue;
                }
                if (take.size() >= kMaxBatchSystems || rows + R->n > kMaxBatchRows ||
                    S->in_use + bytes + R->footprint > S->budget)
                    break;
                take.push_back(R);
                bytes += R->footprint;
                rows += R->n;
                it = S->bqueue.erase(it);
            }
            S->in_use += bytes;
            S->active += (int)take.size();
            const auto now = Clock::now();
            for (Request *R : take) R->t_admit = now;
        }
        S->cv_work.notify_all();
        double ph[4] = {0, 0, 0, 0};
        const int err = run_batch(ctx, st, stage, take, ph);
        const auto now = Clock::now();
        for (Request *R : take) {
            if (err != SPX_OK && R->error == SPX_OK) R->error = err;
            R->upload_ms = ph[0];
            R->setup_ms = ph[1];
            R->solve_ms = ph[2];
            R->download_ms = ph[3];
            R->t_done = now;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->in_use -= bytes;
            S->active -= (int)take.size();
            for (Request *R : take) S->done.push_back(R);
        }
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    spx_ctx_destroy(ctx);
    cudaStreamDestroy(st);
}

}  // namespace spx

using namespace spx;

extern "C" int spx_server_create(spx_ctx *ctx, spx_server **out, int64_t budget_bytes, int max_slots)
{
    if (!ctx || !out || max_slots < 1 || max_slots > 64) return fail(SPX_ERR_INVALID, "spx_server_create: bad argument");
    *out = nullptr;
    size_t freeb = 0, total = 0;
    {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(ctx->device);
        cudaError_t e = cudaMemGetInfo(&freeb, &total);
        cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    }
    spx_server *S = new spx_server();
    S->device = ctx->device;
    S->budget = budget_bytes > 0 ? (size_t)budget_bytes : (size_t)(0.9 * (double)freeb);
    S->slots = max_slots;
    S->batch_rows_limit = kServeBatchRowsMax;
    S->batch_rows = std::min<int64_t>(kServeBatchRows, S->batch_rows_limit);
    S->cluster_rows = kServeClusterRows;
    S->slot_sms = 0;
    for (int i = 0; i < max_slots; ++i) S->workers.emplace_back(worker_main, S);
    for (int i = 0; i < kBatchLanes; ++i) S->workers.emplace_back(lane_main, S);
    *out = S;
    return SPX_OK;
}

extern "C" int spx_server_submit_matrix(spx_server *S, spx_matrix *A, const double *b, double *x, int solver,
                                        double tol, int64_t max_iter, int restart, int precision, int64_t *req_id)
{
    if (!S || !A || !b || !x || !req_id) return fail(SPX_ERR_INVALID, "spx_server_submit_matrix: bad argument");
    if (A->dtype != SPX_F64 || A->n != A->ncols || A->n <= 0)
        return fail(SPX_ERR_INVALID, "spx_server_submit_matrix: A must be a square FP64 matrix");
    if (A->ctx->device != S->device) return fail(SPX_ERR_INVALID, "spx_server_submit_matrix: A is on another device");
    if (precision == SPX_PREC_MIXED && !A->val32.p && !A->ell_val32.p && !A->coo_val32.p)
        return fail(SPX_ERR_INVALID, "spx_server_submit_matrix: MIXED needs A created with SPX_MIXED_SHADOW");
    const bool asked = (solver & SPX_SOLVE_ONE_CLUSTER) != 0;
    solver &= ~SPX_SOLVE_ONE_CLUSTER;
    int base_solver = 0, bs = 0;
    bool jacobi = false, adaptive = false;
    if (parse_solver_code(solver, &base_solver, &jacobi, &bs, &adaptive) != SPX_OK)
        return fail(SPX_ERR_INVALID, "spx_server_submit_matrix: bad solver");
    Request *R = new Request();
    R->n = A->n;
    R->nnz = A->nnz;
    R->rp = nullptr;
    R->col = nullptr;
    R->val = nullptr;
    R->A = A;
    R->b = b;
    R->x = x;
    R->solver = solver;
    R->precision = precision;
    R->restart = restart;
    R->tol = tol;
    R->max_iter = max_iter;
    R->block = 0;
    R->tiled = 0;  // a resident matrix's own buffers are the caller's
    route_request(S, R, solver, asked, A->format == SPX_CSR && A->rp.p != nullptr);
    // the operator is resident (the caller's); the workspace, b and x are the request's
    R->footprint = routed_footprint(R, base_solver, jacobi, bs, adaptive, true);
    R->error = SPX_OK;
    R->t_submit = Clock::now();
    if (R->footprint > S->budget) {
        delete R;
        return fail(SPX_ERR_TOO_LARGE, "request footprint exceeds the server's byte budget");
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        R->id = S->next_id++;
        S->queue.push_back(R);
    }
    *req_id = R->id;
    S->cv_work.notify_all();
    return SPX_OK;
}

extern "C" int spx_server_submit(spx_server *S, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                                 const double *values, const double *b, double *x, int solver, double tol,
                                 int64_t max_iter, int restart, int precision, int64_t *req_id)
{
    if (!S || !row_ptr || !b || !x || !req_id || n <= 0 || nnz < 0 || (nnz > 0 && (!col_idx || !values)))
        return fail(SPX_ERR_INVALID, "spx_server_submit: bad argument");
    const bool asked = (solver & SPX_SOLVE_ONE_CLUSTER) != 0;
    solver &= ~SPX_SOLVE_ONE_CLUSTER;
    int base_solver = 0, bs = 0;
    bool jacobi = false, adaptive = false;
    if (parse_solver_code(solver, &base_solver, &jacobi, &bs, &adaptive) != SPX_OK)
        return fail(SPX_ERR_INVALID, "spx_server_submit: bad solver");
    Request *R = new Request();
    R->A = nullptr;
    R->n = n;
    R->nnz = nnz;
    R->rp = row_ptr;
    R->col = col_idx;
    R->val = values;
    R->b = b;
    R->x = x;
    R->solver = solver;
    R->precision = precision;
    R->restart = restart;
    R->tol = tol;
    R->max_iter = max_iter;
    route_request(S, R, solver, asked, true);
    R->tiled = R->batched || (R->one_cluster && !R->cluster_auto) ? 0 : tiled_copy_bytes(n, nnz, row_ptr, precision);
    R->footprint = routed_footprint(R, base_solver, jacobi, bs, adaptive, false);
    R->error = SPX_OK;
    R->t_submit = Clock::now();
    R->block = batch_block_for(n);
    if (R->footprint > S->budget) {
        delete R;
        return fail(SPX_ERR_TOO_LARGE, "request footprint exceeds the server's byte budget");
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        R->id = S->next_id++;
        (R->batched ? S->bqueue : S->queue).push_back(R);
    }
    *req_id = R->id;
    S->cv_work.notify_all();
    return SPX_OK;
}

extern "C" int spx_server_poll(spx_server *S, spx_server_result *results, int max_results, int wait_ms, int *count)
{
    if (!S || !count || (max_results > 0 && !results)) return fail(SPX_ERR_INVALID, "spx_server_poll: bad argument");
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
    const int k = std::min<int>(max_results, (int)S->done.size());
    spx_server_result *out = results;
    auto ms = [&](Clock::time_point t) { return std::chrono::duration<double, std::milli>(t - S->t0).count(); };
    for (int i = 0; i < k; ++i) {
        Request *R = S->done[(size_t)i];
        out[i].id = R->id;
        out[i].error = R->error;
        out[i].pad = 0;
        out[i].info = R->info;
        out[i].submit_ms = ms(R->t_submit);
        out[i].admit_ms = ms(R->t_admit);
        out[i].done_ms = ms(R->t_done);
        out[i].upload_ms = R->upload_ms;
        out[i].setup_ms = R->setup_ms;
        out[i].solve_ms = R->solve_ms;
        out[i].download_ms = R->download_ms;
        out[i].batched = R->batched ? 1 : R->one_cluster ? 2 : 0;
        out[i].pad2 = 0;
        delete R;
    }
    S->done.erase(S->done.begin(), S->done.begin() + k);
    *count = k;
    return SPX_OK;
}

extern "C" int spx_server_pending(spx_server *S, int64_t *queued, int64_t *running, int64_t *bytes_in_use)
{
    if (!S) return fail(SPX_ERR_INVALID, "spx_server_pending: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = (int64_t)(S->queue.size() + S->bqueue.size());
    if (running) *running = S->active;
    if (bytes_in_use) *bytes_in_use = (int64_t)S->in_use;
    return SPX_OK;
}

extern "C" int spx_server_destroy(spx_server *S)
{
    if (!S) return SPX_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop.store(true);
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    for (Request *R : S->queue) delete R;
    for (Request *R : S->bqueue) delete R;
    for (Request *R : S->done) delete R;
    delete S;
    return SPX_OK;
}

extern "C" int spx_server_set_batching(spx_server *S, int64_t max_rows, int64_t *effective)
{
    if (!S) return fail(SPX_ERR_INVALID, "spx_server_set_batching: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (max_rows >= 0) S->batch_rows = std::min<int64_t>(max_rows, S->batch_rows_limit);
    if (effective) *effective = S->batch_rows;
    return SPX_OK;
}

extern "C" int spx_server_set_cluster_rows(spx_server *S, int64_t max_rows, int64_t *effective)
{
    if (!S) return fail(SPX_ERR_INVALID, "spx_server_set_cluster_rows: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (max_rows >= 0) S->cluster_rows = std::min<int64_t>(max_rows, kServeClusterRowsMax);
    if (effective) *effective = S->cluster_rows;
    return SPX_OK;
}

extern "C" int spx_server_set_slot_sms(spx_server *S, int sms, int *effective)
{
    if (!S) return fail(SPX_ERR_INVALID, "spx_server_set_slot_sms: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (sms >= -1) S->slot_sms = sms;
    if (effective) *effective = S->slot_sms;
    return SPX_OK;
}
