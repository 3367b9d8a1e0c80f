// api.cu -- C ABI of libspx: context, errors, matrix creation (validation,
// statistics, CSR -> CSR/ELL/COO/HYB conversion on the device), export,
// SpMV entry points.
#include <climits>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dev_common.cuh"
#include "kstate.cuh"
#include "spx_internal.cuh"

namespace spx {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
int fail(int status, const std::string &msg)
{
    g_last_error = msg;
    return status;
}
int cuda_fail(cudaError_t e, const char *what)
{
    // clear the runtime's record of a non-sticky error (a launch refused for its
    // resources, an invalid argument), so the thread's next call does not report it
    cudaGetLastError();
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SPX_ERR_OOM : SPX_ERR_CUDA;
}

void *dalloc(spx_ctx *ctx, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (ctx->alloc) return ctx->alloc(bytes, ctx->stream, ctx->user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dfree(spx_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    if (ctx->free) ctx->free(p, bytes, ctx->stream, ctx->user);
    else cudaFreeAsync(p, ctx->stream);
}

int dbuf_alloc(spx_ctx *ctx, DBuf &b, size_t bytes)
{
    const size_t padded = round_up(bytes, 16) + kArrayPad;
    b.p = dalloc(ctx, padded);
    if (!b.p) {
        b.bytes = 0;
        return fail(SPX_ERR_OOM, "device allocation of " + std::to_string(padded) + " bytes failed");
    }
    b.bytes = bytes;
    b.free_fn = ctx->alloc ? ctx->free : nullptr;
    b.free_user = ctx->user;
    return SPX_OK;
}

void dbuf_free(spx_ctx *ctx, DBuf &b)
{
    if (b.p) {
        const size_t padded = round_up(b.bytes, 16) + kArrayPad;
        if (b.free_fn) b.free_fn(b.p, padded, ctx->stream, b.free_user);
        else cudaFreeAsync(b.p, ctx->stream);
    }
    b.p = nullptr;
    b.bytes = 0;
    b.free_fn = nullptr;
    b.free_user = nullptr;
}

// Sets the context's device for the lifetime of a call, restores the caller's.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// ------------------------------------------------------------------ validation / statistics
__global__ void k_validate_rows(int64_t n, int64_t nnz, const int *__restrict__ rp, unsigned *flags,
                                int *maxlen)
{
    int ml = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = rp[i], b = rp[i + 1];
        if (a < 0 || b < a || (int64_t)b > nnz) atomicOr(flags, 1u);
        else ml = max(ml, b - a);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || (int64_t)rp[n] != nnz))
        atomicOr(flags, 1u);
    ml = max(ml, __reduce_max_sync(0xffffffffu, ml));
    if ((threadIdx.x & 31) == 0 && ml > 0) atomicMax(maxlen, ml);
}

__global__ void k_validate_cols(int64_t nnz, int64_t ncols, const int *__restrict__ col,
                                unsigned *flags)
{
    bool bad = false;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int c = col[k];
        bad |= (c < 0 || (int64_t)c >= ncols);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, 2u);
}

// Row-length histogram.  Lengths below kHistShared are counted in a block-local
// shared histogram first (one global atomic per bin per block instead of one
// per row: most rows fall in a handful of bins); longer rows go straight to
// the global bins.
constexpr int kHistShared = 2048;

__global__ void k_len_hist(int64_t n, const int *__restrict__ rp, unsigned long long *hist, int64_t bins)
{
    __shared__ unsigned sh[kHistShared];
    const int nb = bins < kHistShared ? (int)bins : kHistShared;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int len = rp[i + 1] - rp[i];
        if (len < nb) atomicAdd(sh + len, 1u);
        else atomicAdd(hist + len, 1ull);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (sh[b]) atomicAdd(hist + b, (unsigned long long)sh[b]);
}

// ------------------------------------------------------------------ conversions
template <class S, class D>
__global__ void k_cast(int64_t m, const S *__restrict__ src, D *__restrict__ dst)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = static_cast<D>(src[k]);
}

// COO row indices: one warp per row writes row i over [rp[i], rp[i+1]).
__global__ void k_expand_rows(int64_t n, const int *__restrict__ rp, int *__restrict__ row)
{
    const int lane = threadIdx.x & 31;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5)
        for (int k = rp[i] + lane; k < rp[i + 1]; k += 32) row[k] = (int)i;
}

// ELL width w, slot (i, j) at j*ld + i: the first min(len_i, w) entries of
// row i in CSR order, then padding (col -1, value +0.0).  Rows n..ld-1 are
// padding too.  Value bytes are copied unchanged.
template <class T>
__global__ void k_to_ell(int64_t n, int64_t ld, int w, const int *__restrict__ rp,
                         const int *__restrict__ col, const T *__restrict__ val, int *__restrict__ ecol,
                         T *__restrict__ eval)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ld;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = i < n ? rp[i] : 0;
        const int len = i < n ? rp[i + 1] - a : 0;
        for (int j = 0; j < w; ++j) {
            const int64_t s = (int64_t)j * ld + i;
            if (j < len) {
                ecol[s] = col[a + j];
                eval[s] = val[a + j];
            } else {
                ecol[s] = -1;
                eval[s] = T(0);
            }
        }
    }
}

constexpr int kHybRows = 1024;  // rows per block of the HYB COO builder

__global__ void k_hyb_block_counts(int64_t n, const int *__restrict__ rp, int w,
                                   long long *__restrict__ block_tot)
{
    __shared__ long long red[32];
    const int64_t i = blockIdx.x * (int64_t)kHybRows + threadIdx.x;
    long long c = 0;
    if (i < n) c = max(0, rp[i + 1] - rp[i] - w);
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long s = red[threadIdx.x];
        s = warp_sum(s);
        if (threadIdx.x == 0) block_tot[blockIdx.x] = s;
    }
}

template <class T>
__global__ void k_hyb_coo(int64_t n, const int *__restrict__ rp, const int *__restrict__ col,
                          const T *__restrict__ val, int w, const long long *__restrict__ block_off,
                          int *__restrict__ crow, int *__restrict__ ccol, T *__restrict__ cval)
{
    __shared__ long long scan[kHybRows];
    const int64_t i = blockIdx.x * (int64_t)kHybRows + threadIdx.x;
    long long c = 0;
    if (i < n) c = max(0, rp[i + 1] - rp[i] - w);
    scan[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < kHybRows; o <<= 1) {  // inclusive Hillis-Steele scan (integers: exact)
        const long long v = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
    }
    if (i < n && c > 0) {
        long long o = block_off[blockIdx.x] + scan[threadIdx.x] - c;
        for (int k = rp[i] + w; k < rp[i + 1]; ++k, ++o) {
            crow[o] = (int)i;
            ccol[o] = col[k];
            cval[o] = val[k];
        }
    }
}

}  // namespace spx

using namespace spx;

// ------------------------------------------------------------------ context
extern "C" int spx_ctx_create(spx_ctx **out, int device, void *stream, spx_alloc_fn alloc,
                              spx_free_fn freefn, void *user)
{
    if (!out) return fail(SPX_ERR_INVALID, "spx_ctx_create: out is NULL");
    *out = nullptr;
    if ((alloc == nullptr) != (freefn == nullptr))
        return fail(SPX_ERR_INVALID, "spx_ctx_create: give both alloc and free, or neither");
    int ndev = 0;
    SPX_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(SPX_ERR_INVALID, "spx_ctx_create: bad device");
    DeviceGuard g(device);
    spx_ctx *c = new (std::nothrow) spx_ctx();
    if (!c) return fail(SPX_ERR_OOM, "host allocation failed");
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    c->alloc = alloc;
    c->free = freefn;
    c->user = user;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaGetDeviceProperties");
    }
    c->sm_count = prop.multiProcessorCount;
    c->grid_sms = c->sm_count;
    c->max_smem_optin = (int)prop.sharedMemPerBlockOptin;
    c->l2_bytes = prop.l2CacheSize;
    c->red_grid = c->sm_count * 4;
    const size_t red_bytes = (size_t)(2 * c->red_grid + 16) * 8;
    c->dev_err = static_cast<unsigned *>(dalloc(c, 64));
    c->red = dalloc(c, red_bytes);
    if (!c->dev_err || !c->red) {
        dfree(c, c->dev_err, 64);
        dfree(c, c->red, red_bytes);
        delete c;
        return fail(SPX_ERR_OOM, "spx_ctx_create: device scratch allocation failed");
    }
    e = cudaMemsetAsync(c->dev_err, 0, 64, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->red, 0, red_bytes, c->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(&c->host_err, 64);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        dfree(c, c->dev_err, 64);
        delete c;
        return cuda_fail(e, "spx_ctx_create");
    }
    *out = c;
    return SPX_OK;
}

extern "C" int spx_ctx_set_grid_sms(spx_ctx *ctx, int sms, int *effective)
{
    if (!ctx) return fail(SPX_ERR_INVALID, "spx_ctx_set_grid_sms: NULL context");
    ctx->grid_sms = sms <= 0 ? ctx->sm_count : std::min(sms, ctx->sm_count);
    if (effective) *effective = ctx->grid_sms;
    return SPX_OK;
}

extern "C" int spx_ctx_check(spx_ctx *ctx)
{
    if (!ctx) return fail(SPX_ERR_INVALID, "spx_ctx_check: NULL context");
    DeviceGuard g(ctx->device);
    unsigned h = 0;
    SPX_CUDA(cudaMemcpyAsync(&h, ctx->dev_err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    if (h == 0) return SPX_OK;
    SPX_CUDA(cudaMemsetAsync(ctx->dev_err, 0, sizeof(unsigned), ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    return fail(SPX_ERR_TIMEOUT, "a bounded device-side wait gave up (error word " + std::to_string(h) + ")");
}

extern "C" int spx_ctx_destroy(spx_ctx *ctx)
{
    if (!ctx) return SPX_OK;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    dfree(ctx, ctx->dev_err, 64);
    dfree(ctx, ctx->red, (size_t)(2 * ctx->red_grid + 16) * 8);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->host_err) cudaFreeHost(ctx->host_err);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    delete ctx;
    return SPX_OK;
}

extern "C" int spx_ctx_set_stream(spx_ctx *ctx, void *stream)
{
    if (!ctx) return fail(SPX_ERR_INVALID, "spx_ctx_set_stream: ctx is NULL");
    ctx->stream = static_cast<cudaStream_t>(stream);
    return SPX_OK;
}

// ------------------------------------------------------------------ matrices
namespace {

void free_matrix_arrays(spx_matrix *A)
{
    spx_ctx *c = A->ctx;
    DBuf *bufs[] = {&A->rp,       &A->col,       &A->val,      &A->val32,     &A->ell_col,
                    &A->ell_val,  &A->ell_val32, &A->coo_row,  &A->coo_col,   &A->coo_val,
                    &A->coo_val32, &A->tiles,    &A->carry_row, &A->carry_val, &A->partials,
                    &A->ticket,   &A->stage_x,   &A->stage_y,   &A->coo_tiles, &A->flags,
                    &A->hint,     &A->coo_rowtiles, &A->tc_col, &A->tc_val, &A->tc_val32, &A->tc_row,
                    &A->tc_mask,  &A->empty_rows, &A->ct_row, &A->ct_col, &A->ct_val, &A->ct_val32,
                    &A->small_out, &A->cl_work};
    for (DBuf *b : bufs) dbuf_free(c, *b);
}

int grid1d(spx_ctx *ctx, int64_t work, int block = 256)
{
    int64_t g = ceil_div(work, block);
    const int64_t cap = (int64_t)ctx->grid_sms * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

template <class S, class D> int cast_into(spx_ctx *ctx, const void *src, DBuf &dst, int64_t m)
{
    SPX_TRY(dbuf_alloc(ctx, dst, (size_t)m * sizeof(D)));
    if (m > 0) {
        k_cast<S, D><<<grid1d(ctx, m), 256, 0, ctx->stream>>>(m, static_cast<const S *>(src), dst.as<D>());
        SPX_CUDA(cudaGetLastError());
    }
    return SPX_OK;
}

int copy_into(spx_ctx *ctx, const void *src, DBuf &dst, size_t bytes)
{
    SPX_TRY(dbuf_alloc(ctx, dst, bytes));
    if (bytes) SPX_CUDA(cudaMemcpyAsync(dst.p, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    return SPX_OK;
}

template <class T> int build_ell(spx_ctx *ctx, spx_matrix *A, int64_t w, const DBuf &val, DBuf &ecol, DBuf &ev)
{
    const int64_t slots = w * A->ell_ld;
    if (!ecol.p) SPX_TRY(dbuf_alloc(ctx, ecol, (size_t)slots * 4));
    SPX_TRY(dbuf_alloc(ctx, ev, (size_t)slots * sizeof(T)));
    if (slots > 0) {
        k_to_ell<T><<<grid1d(ctx, A->ell_ld), 256, 0, ctx->stream>>>(
            A->n, A->ell_ld, (int)w, A->rp.as<int>(), A->col.as<int>(), val.as<T>(), ecol.as<int>(),
            ev.as<T>());
        SPX_CUDA(cudaGetLastError());
    }
    return SPX_OK;
}

template <class T>
int build_hyb_coo(spx_ctx *ctx, spx_matrix *A, int64_t w, const DBuf &val, const DBuf &block_off,
                  int64_t nblocks, bool first, DBuf &cv)
{
    if (first) {
        SPX_TRY(dbuf_alloc(ctx, A->coo_row, (size_t)A->coo_nnz * 4));
        SPX_TRY(dbuf_alloc(ctx, A->coo_col, (size_t)A->coo_nnz * 4));
    }
    SPX_TRY(dbuf_alloc(ctx, cv, (size_t)A->coo_nnz * sizeof(T)));
    if (A->coo_nnz > 0) {
        k_hyb_coo<T><<<(int)nblocks, kHybRows, 0, ctx->stream>>>(
            A->n, A->rp.as<int>(), A->col.as<int>(), val.as<T>(), (int)w, block_off.as<long long>(),
            A->coo_row.as<int>(), A->coo_col.as<int>(), cv.as<T>());
        SPX_CUDA(cudaGetLastError());
    }
    return SPX_OK;
}

int matrix_build(spx_ctx *ctx, spx_matrix *A, const int32_t *rp_in, const int32_t *col_in,
                 const void *val_in, int vdt, int64_t hyb_width, unsigned flags)
{
    const int64_t n = A->n, nnz = A->nnz;
    const size_t V = A->dtype == SPX_F64 ? 8 : 4;
    // 1. owned copies of the CSR arrays, values in the matrix dtype
    SPX_TRY(copy_into(ctx, rp_in, A->rp, (size_t)(n + 1) * 4));
    SPX_TRY(copy_into(ctx, col_in, A->col, (size_t)nnz * 4));
    if (vdt == A->dtype) SPX_TRY(copy_into(ctx, val_in, A->val, (size_t)nnz * V));
    else if (A->dtype == SPX_F64) SPX_TRY((cast_into<float, double>(ctx, val_in, A->val, nnz)));
    else SPX_TRY((cast_into<double, float>(ctx, val_in, A->val, nnz)));

    // 2. validation and row statistics (one synchronisation)
    DBuf scratch;
    SPX_TRY(dbuf_alloc(ctx, scratch, 64));
    SPX_CUDA(cudaMemsetAsync(scratch.p, 0, 64, ctx->stream));
    unsigned *flags_d = scratch.as<unsigned>();
    int *maxlen_d = reinterpret_cast<int *>(scratch.as<unsigned char>() + 16);
    k_validate_rows<<<grid1d(ctx, n), 256, 0, ctx->stream>>>(n, nnz, A->rp.as<int>(), flags_d, maxlen_d);
    SPX_CUDA(cudaGetLastError());
    if (nnz > 0) {
        k_validate_cols<<<grid1d(ctx, nnz), 256, 0, ctx->stream>>>(nnz, A->ncols, A->col.as<int>(), flags_d);
        SPX_CUDA(cudaGetLastError());
    }
    unsigned hv[8] = {0};
    SPX_CUDA(cudaMemcpyAsync(hv, scratch.p, 32, cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    dbuf_free(ctx, scratch);
    if (hv[0] & 1u) return fail(SPX_ERR_INVALID, "invalid CSR row pointers (need rp[0]=0, non-decreasing, rp[n]=nnz)");
    if (hv[0] & 2u) return fail(SPX_ERR_INVALID, "column index out of range [0, ncols)");
    A->max_len = (int64_t)(int)hv[4];
    A->mean_len = n > 0 ? (double)nnz / (double)n : 0.0;

    const bool shadow = (flags & SPX_MIXED_SHADOW) && A->dtype == SPX_F64;
    if (A->format == SPX_CSR) {
        if (shadow) SPX_TRY((cast_into<double, float>(ctx, A->val.p, A->val32, nnz)));
        return SPX_OK;
    }
    if (A->format == SPX_COO) {
        A->coo_nnz = nnz;
        SPX_TRY(dbuf_alloc(ctx, A->coo_row, (size_t)nnz * 4));
        if (nnz > 0) {
            k_expand_rows<<<grid1d(ctx, n * 32), 256, 0, ctx->stream>>>(n, A->rp.as<int>(), A->coo_row.as<int>());
            SPX_CUDA(cudaGetLastError());
        }
        A->coo_col = A->col;
        A->coo_val = A->val;
        A->col = DBuf();
        A->val = DBuf();
        if (shadow) SPX_TRY((cast_into<double, float>(ctx, A->coo_val.p, A->coo_val32, nnz)));
        dbuf_free(ctx, A->rp);
        return SPX_OK;
    }
    // ELL / HYB
    int64_t w = A->max_len;
    if (A->format == SPX_HYB) {
        if (hyb_width >= 0) {
            w = hyb_width < A->max_len ? hyb_width : A->max_len;
        } else {
            // footprint-optimal width: smallest k with (V+8) #{len > k} <= (V+4) n
            DBuf hist;
            const int64_t bins = A->max_len + 1;
            SPX_TRY(dbuf_alloc(ctx, hist, (size_t)bins * 8));
            SPX_CUDA(cudaMemsetAsync(hist.p, 0, (size_t)bins * 8, ctx->stream));
            k_len_hist<<<grid1d(ctx, n), 256, 0, ctx->stream>>>(n, A->rp.as<int>(), hist.as<unsigned long long>(),
                                                                bins);
            SPX_CUDA(cudaGetLastError());
            std::vector<unsigned long long> h((size_t)bins);
            SPX_CUDA(cudaMemcpyAsync(h.data(), hist.p, (size_t)bins * 8, cudaMemcpyDeviceToHost, ctx->stream));
            SPX_CUDA(cudaStreamSynchronize(ctx->stream));
            dbuf_free(ctx, hist);
            int64_t longer = n;  // rows with len > k, k = -1
            w = A->max_len;
            for (int64_t k = 0; k <= A->max_len; ++k) {
                longer -= (int64_t)h[(size_t)k];
                if ((int64_t)(V + 8) * longer <= (int64_t)(V + 4) * n) {
                    w = k;
                    break;
                }
            }
        }
    }
    A->ell_ld = (int64_t)round_up((size_t)(n > 0 ? n : 1), 32);
    const double ell_bytes = (double)w * (double)A->ell_ld * (double)(4 + V + (shadow ? 4 : 0));
    size_t free_b = 0, total_b = 0;
    SPX_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (ell_bytes > 0.9 * (double)free_b || w * A->ell_ld > (int64_t)1 << 40)
        return fail(SPX_ERR_TOO_LARGE, "ELL footprint (" + std::to_string((long long)(ell_bytes / 1e9)) +
                                           " GB for width " + std::to_string((long long)w) +
                                           ") exceeds the device budget");
    A->ell_w = w;
    if (A->dtype == SPX_F64) {
        SPX_TRY(build_ell<double>(ctx, A, w, A->val, A->ell_col, A->ell_val));
        if (shadow) SPX_TRY((cast_into<double, float>(ctx, A->ell_val.p, A->ell_val32, w * A->ell_ld)));
    } else {
        SPX_TRY(build_ell<float>(ctx, A, w, A->val, A->ell_col, A->ell_val));
    }
    if (A->format == SPX_HYB) {
        const int64_t nblocks = ceil_div(n, kHybRows);
        DBuf tot;
        SPX_TRY(dbuf_alloc(ctx, tot, (size_t)(nblocks > 0 ? nblocks : 1) * 8));
        std::vector<long long> h((size_t)(nblocks > 0 ? nblocks : 1), 0);
        if (nblocks > 0) {
            k_hyb_block_counts<<<(int)nblocks, kHybRows, 0, ctx->stream>>>(n, A->rp.as<int>(), (int)w, tot.as<long long>());
            SPX_CUDA(cudaGetLastError());
            SPX_CUDA(cudaMemcpyAsync(h.data(), tot.p, (size_t)nblocks * 8, cudaMemcpyDeviceToHost, ctx->stream));
            SPX_CUDA(cudaStreamSynchronize(ctx->stream));
        }
        long long run = 0;
        for (auto &v : h) {
            const long long c = v;
            v = run;
            run += c;
        }
        A->coo_nnz = run;
        if (nblocks > 0)
            SPX_CUDA(cudaMemcpyAsync(tot.p, h.data(), (size_t)nblocks * 8, cudaMemcpyHostToDevice, ctx->stream));
        if (A->dtype == SPX_F64) {
            SPX_TRY(build_hyb_coo<double>(ctx, A, w, A->val, tot, nblocks, true, A->coo_val));
            if (shadow) SPX_TRY((cast_into<double, float>(ctx, A->coo_val.p, A->coo_val32, A->coo_nnz)));
        } else {
            SPX_TRY(build_hyb_coo<float>(ctx, A, w, A->val, tot, nblocks, true, A->coo_val));
        }
        SPX_CUDA(cudaStreamSynchronize(ctx->stream));  // the host offsets must outlive the copy
        dbuf_free(ctx, tot);
    }
    dbuf_free(ctx, A->rp);
    dbuf_free(ctx, A->col);
    dbuf_free(ctx, A->val);
    return SPX_OK;
}

}  // namespace

extern "C" int spx_matrix_create(spx_ctx *ctx, spx_matrix **out, int format, int dtype, int64_t nrows,
                                 int64_t ncols, int64_t nnz, const int32_t *row_ptr,
                                 const int32_t *col_idx, const void *values, int values_dtype,
                                 int64_t hyb_width, unsigned flags)
{
    if (!ctx || !out) return fail(SPX_ERR_INVALID, "spx_matrix_create: ctx or out is NULL");
    *out = nullptr;
    if (format < SPX_CSR || format > SPX_HYB) return fail(SPX_ERR_INVALID, "unknown format");
    if ((dtype != SPX_F64 && dtype != SPX_F32) || (values_dtype != SPX_F64 && values_dtype != SPX_F32))
        return fail(SPX_ERR_INVALID, "dtype must be SPX_F64 or SPX_F32");
    if (nrows < 0 || ncols < 0 || nnz < 0) return fail(SPX_ERR_INVALID, "negative size");
    if (nrows >= INT_MAX || ncols > INT_MAX || nnz > INT_MAX)
        return fail(SPX_ERR_TOO_LARGE, "sizes must fit int32 indices");
    if (!row_ptr || (nnz > 0 && (!col_idx || !values)))
        return fail(SPX_ERR_INVALID, "NULL input array");
    DeviceGuard g(ctx->device);
    spx_matrix *A = new (std::nothrow) spx_matrix();
    if (!A) return fail(SPX_ERR_OOM, "host allocation failed");
    A->ctx = ctx;
    A->format = format;
    A->dtype = dtype;
    A->n = nrows;
    A->ncols = ncols;
    A->nnz = nnz;
    const size_t vin = values_dtype == SPX_F64 ? 8 : 4;
    DBuf hrp, hcol, hval;
    const int32_t *rp_d = row_ptr, *col_d = col_idx;
    const void *val_d = values;
    int st = SPX_OK;
    if (flags & SPX_HOST_INPUT) {
        st = dbuf_alloc(ctx, hrp, (size_t)(nrows + 1) * 4);
        if (st == SPX_OK) st = dbuf_alloc(ctx, hcol, (size_t)nnz * 4);
        if (st == SPX_OK) st = dbuf_alloc(ctx, hval, (size_t)nnz * vin);
        if (st == SPX_OK) {
            cudaError_t e = cudaMemcpyAsync(hrp.p, row_ptr, (size_t)(nrows + 1) * 4, cudaMemcpyHostToDevice, ctx->stream);
            if (e == cudaSuccess && nnz)
                e = cudaMemcpyAsync(hcol.p, col_idx, (size_t)nnz * 4, cudaMemcpyHostToDevice, ctx->stream);
            if (e == cudaSuccess && nnz)
                e = cudaMemcpyAsync(hval.p, values, (size_t)nnz * vin, cudaMemcpyHostToDevice, ctx->stream);
            if (e != cudaSuccess) st = cuda_fail(e, "spx_matrix_create: host copy");
        }
        rp_d = hrp.as<int32_t>();
        col_d = hcol.as<int32_t>();
        val_d = hval.p;
    }
    if (st == SPX_OK) st = matrix_build(ctx, A, rp_d, col_d, val_d, values_dtype, hyb_width, flags);
    if (st == SPX_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "spx_matrix_create");
    }
    dbuf_free(ctx, hrp);
    dbuf_free(ctx, hcol);
    dbuf_free(ctx, hval);
    if (st != SPX_OK) {
        std::string msg = spx_last_error();
        free_matrix_arrays(A);
        cudaStreamSynchronize(ctx->stream);
        delete A;
        set_error(msg);
        return st;
    }
    A->kernel = SPX_KERNEL_AUTO;
    *out = A;
    return SPX_OK;
}

namespace spx {
void solver_work_free(spx_matrix *A);  // solvers.cu
}

extern "C" int spx_matrix_destroy(spx_matrix *A)
{
    if (!A) return SPX_OK;
    DeviceGuard g(A->ctx->device);
    solver_work_free(A);
    if (A->batch1) spx_batch_destroy(A->batch1);
    free_matrix_arrays(A);
    cudaStreamSynchronize(A->ctx->stream);
    delete A;
    return SPX_OK;
}

extern "C" int spx_matrix_get_info(const spx_matrix *A, spx_matrix_info *info)
{
    if (!A || !info) return fail(SPX_ERR_INVALID, "spx_matrix_get_info: NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->format = A->format;
    info->dtype = A->dtype;
    info->nrows = A->n;
    info->ncols = A->ncols;
    info->nnz = A->nnz;
    info->ell_width = A->ell_w;
    info->ell_ld = A->ell_ld;
    info->coo_nnz = A->coo_nnz;
    info->max_row_len = A->max_len;
    info->mean_row_len = A->mean_len;
    const DBuf *bufs[] = {&A->rp,      &A->col,     &A->val,       &A->val32,   &A->ell_col,
                          &A->ell_val, &A->ell_val32, &A->coo_row, &A->coo_col, &A->coo_val,
                          &A->coo_val32};
    int64_t b = 0;
    for (const DBuf *x : bufs) b += (int64_t)x->bytes;
    info->device_bytes = b;
    info->kernel = A->kernel;
    info->kernel_param = A->kparam;
    info->has_f32_shadow = (A->val32.p || A->ell_val32.p || A->coo_val32.p) ? 1 : 0;
    return SPX_OK;
}

extern "C" int spx_matrix_export(spx_ctx *ctx, const spx_matrix *A, int part, void *dst,
                                 size_t dst_bytes, size_t *written)
{
    if (!ctx || !A) return fail(SPX_ERR_INVALID, "spx_matrix_export: NULL argument");
    const DBuf *b = nullptr;
    switch (part) {
    case SPX_PART_ROW_PTR: b = &A->rp; break;
    case SPX_PART_COL: b = &A->col; break;
    case SPX_PART_VAL: b = &A->val; break;
    case SPX_PART_ELL_COL: b = &A->ell_col; break;
    case SPX_PART_ELL_VAL: b = &A->ell_val; break;
    case SPX_PART_COO_ROW: b = &A->coo_row; break;
    case SPX_PART_COO_COL: b = &A->coo_col; break;
    case SPX_PART_COO_VAL: b = &A->coo_val; break;
    case SPX_PART_VAL_F32:
        b = A->val32.p ? &A->val32 : (A->ell_val32.p ? &A->ell_val32 : &A->coo_val32);
        break;
    default: return fail(SPX_ERR_NOT_FOUND, "unknown part");
    }
    if (!b->p) return fail(SPX_ERR_NOT_FOUND, "the matrix format has no such part");
    if (written) *written = b->bytes;
    if (dst_bytes < b->bytes) return fail(SPX_ERR_INVALID, "export buffer too small");
    DeviceGuard g(ctx->device);
    if (b->bytes) SPX_CUDA(cudaMemcpyAsync(dst, b->p, b->bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    return SPX_OK;
}

extern "C" int spx_matrix_set_kernel(spx_matrix *A, int kernel, int param)
{
    if (!A) return fail(SPX_ERR_INVALID, "spx_matrix_set_kernel: A is NULL");
    bool okk = false;
    switch (A->format) {
    case SPX_CSR:
        okk = kernel == SPX_KERNEL_AUTO || kernel == SPX_KERNEL_CSR_VECTOR || kernel == SPX_KERNEL_CSR_MERGE ||
              kernel == SPX_KERNEL_CSR_SPLIT || kernel == SPX_KERNEL_CSR_ROWS || kernel == SPX_KERNEL_CSR_TILED;
        break;
    case SPX_ELL: okk = kernel == SPX_KERNEL_AUTO || kernel == SPX_KERNEL_ELL; break;
    case SPX_COO: okk = kernel == SPX_KERNEL_AUTO || kernel == SPX_KERNEL_COO; break;
    case SPX_HYB: okk = kernel == SPX_KERNEL_AUTO || kernel == SPX_KERNEL_ELL || kernel == SPX_KERNEL_COO; break;
    }
    if (!okk) return fail(SPX_ERR_UNSUPPORTED, "kernel does not apply to the matrix format");
    if (kernel == SPX_KERNEL_CSR_VECTOR && param != 0 &&
        !(param == 1 || param == 2 || param == 4 || param == 8 || param == 16 || param == 32))
        return fail(SPX_ERR_INVALID, "CSR vector width must be 0 (auto) or 1..32, a power of 2");
    if (kernel == SPX_KERNEL_CSR_TILED && param != 0 && !(param == 16 || param == 32))
        return fail(SPX_ERR_INVALID, "tiled CSR nonzeros per lane must be 0 (auto: 32), 16 or 32");
    if (kernel == SPX_KERNEL_CSR_MERGE && param != 0 && !(param == 4 || param == 8 || param == 16))
        return fail(SPX_ERR_INVALID, "merge items per thread must be 0 (auto), 4, 8 or 16");
    if (kernel == SPX_KERNEL_COO && param != 0 &&
        !(param == 1 || param == 8 || param == 16 || param == 216 || param == 232 || param == 104 || param == 108 ||
          param == 116))
        return fail(SPX_ERR_INVALID, "COO parameter must be 0 (auto), 1 (row-block), 8, 16 (split), 216, 232 "
                                     "(tiled split) or 104, 108, 116 (tiled segmented reduction)");
    if (kernel == SPX_KERNEL_CSR_ROWS && param != 0 &&
        !(param == 1 || param == 2 || param == 12 || param == 22 || param == 42))
        return fail(SPX_ERR_INVALID, "row-block parameter must be 0 (auto), 1, 2, 12, 22 or 42");
    if (kernel == SPX_KERNEL_CSR_SPLIT && param != 0 && !(param == 8 || param == 16))
        return fail(SPX_ERR_INVALID, "split nonzeros per lane must be 0 (auto), 8 or 16");
    if (kernel == SPX_KERNEL_ELL && param != 0 && !(param == 1 || param == 2 || (param == 4 && A->dtype == SPX_F32)))
        return fail(SPX_ERR_INVALID, "ELL rows per thread must be 0 (auto), 1, 2 (or 4 for FP32)");
    A->kernel = kernel;
    A->kparam = param;
    return SPX_OK;
}

// ------------------------------------------------------------------ kernel autotuning
namespace {
// Kernel variants worth timing for a matrix (those spx_matrix_set_kernel accepts).
std::vector<std::pair<int, int>> tune_candidates(const spx_matrix *A)
{
    std::vector<std::pair<int, int>> c;
    switch (A->format) {
    case SPX_CSR:
        c = {{SPX_KERNEL_CSR_ROWS, 1}, {SPX_KERNEL_CSR_ROWS, 2}, {SPX_KERNEL_CSR_ROWS, 22},
             {SPX_KERNEL_CSR_ROWS, 42}, {SPX_KERNEL_CSR_MERGE, 4},
             {SPX_KERNEL_CSR_MERGE, 8}, {SPX_KERNEL_CSR_MERGE, 16}, {SPX_KERNEL_CSR_SPLIT, 8},
             {SPX_KERNEL_CSR_SPLIT, 16}, {SPX_KERNEL_CSR_TILED, 16}, {SPX_KERNEL_CSR_TILED, 32}};
        for (int sw = 1; sw <= 32; sw *= 2) c.push_back({SPX_KERNEL_CSR_VECTOR, sw});
        break;
    case SPX_ELL:
        c = {{SPX_KERNEL_ELL, 1}, {SPX_KERNEL_ELL, 2}};
        if (A->dtype == SPX_F32) c.push_back({SPX_KERNEL_ELL, 4});
        break;
    case SPX_COO:
        c = {{SPX_KERNEL_COO, 1},   {SPX_KERNEL_COO, 8},   {SPX_KERNEL_COO, 16},  {SPX_KERNEL_COO, 216},
             {SPX_KERNEL_COO, 232}, {SPX_KERNEL_COO, 104}, {SPX_KERNEL_COO, 108}, {SPX_KERNEL_COO, 116}};
        break;
    default:  // HYB: its ELL part's rows per thread, or its COO part's kernel
        c = {{SPX_KERNEL_ELL, 1},   {SPX_KERNEL_ELL, 2},   {SPX_KERNEL_COO, 8},   {SPX_KERNEL_COO, 16},
             {SPX_KERNEL_COO, 216}, {SPX_KERNEL_COO, 232}, {SPX_KERNEL_COO, 104}, {SPX_KERNEL_COO, 116}};
        if (A->dtype == SPX_F32) c.push_back({SPX_KERNEL_ELL, 4});
        break;
    }
    c.insert(c.begin(), {SPX_KERNEL_AUTO, 0});
    return c;
}

template <class T> int time_spmv(spx_ctx *ctx, spx_matrix *A, int reps, cudaEvent_t e0, cudaEvent_t e1, float *us)
{
    const T *x = A->stage_x.as<T>();
    T *y = A->stage_y.as<T>();
    Epi<T> e;
    e.y = y;
    SPX_TRY(spmv_launch<T>(ctx, A, x, e, false));  // warm-up; builds the variant's tile maps
    SPX_CUDA(cudaEventRecord(e0, ctx->stream));
    for (int r = 0; r < reps; ++r) SPX_TRY(spmv_launch<T>(ctx, A, x, e, false));
    SPX_CUDA(cudaEventRecord(e1, ctx->stream));
    SPX_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    SPX_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *us = ms * 1000.f / (float)reps;
    return SPX_OK;
}
}  // namespace

extern "C" int spx_matrix_tune(spx_ctx *ctx, spx_matrix *A, int reps, int *kernel, int *param, float *best_us)
{
    if (!ctx || !A) return fail(SPX_ERR_INVALID, "spx_matrix_tune: ctx or A is NULL");
    if (reps < 1 || reps > 1000) return fail(SPX_ERR_INVALID, "spx_matrix_tune: reps must be in [1, 1000]");
    DeviceGuard g(ctx->device);
    const size_t V = A->dtype == SPX_F64 ? 8 : 4;
    if (!A->stage_x.p) SPX_TRY(dbuf_alloc(ctx, A->stage_x, (size_t)(A->ncols > 0 ? A->ncols : 1) * V));
    if (!A->stage_y.p) SPX_TRY(dbuf_alloc(ctx, A->stage_y, (size_t)(A->n > 0 ? A->n : 1) * V));
    if (A->ncols) SPX_CUDA(cudaMemsetAsync(A->stage_x.p, 0, (size_t)A->ncols * V, ctx->stream));
    const int k0 = A->kernel, p0 = A->kparam;
    cudaEvent_t e0, e1;
    SPX_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(SPX_ERR_CUDA, "cudaEventCreate");
    }
    int bk = k0, bp = p0, st = SPX_OK;
    float best = -1.f;
    for (const auto &kp : tune_candidates(A)) {
        if (spx_matrix_set_kernel(A, kp.first, kp.second) != SPX_OK) continue;
        float us = 0.f;
        const int r = A->dtype == SPX_F64 ? time_spmv<double>(ctx, A, reps, e0, e1, &us)
                                          : time_spmv<float>(ctx, A, reps, e0, e1, &us);
        if (r == SPX_ERR_TOO_LARGE || r == SPX_ERR_UNSUPPORTED) continue;  // variant does not fit this matrix
        if (r != SPX_OK) {
            st = r;
            break;
        }
        if (best < 0.f || us < best) {
            best = us;
            bk = kp.first;
            bp = kp.second;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SPX_OK || best < 0.f) {
        A->kernel = k0;
        A->kparam = p0;
        return st != SPX_OK ? st : fail(SPX_ERR_UNSUPPORTED, "spx_matrix_tune: no kernel variant ran");
    }
    A->kernel = bk;
    A->kparam = bp;
    if (kernel) *kernel = bk;
    if (param) *param = bp;
    if (best_us) *best_us = best;
    return SPX_OK;
}

// ------------------------------------------------------------------ SpMV entry points
namespace {
template <class T>
int spmv_common(spx_ctx *ctx, const spx_matrix *A, double alpha, const void *x, double beta, void *y,
                bool use_beta)
{
    Epi<T> e;
    e.alpha = (T)alpha;
    e.beta = (T)beta;
    e.z = use_beta && beta != 0.0 ? static_cast<const T *>(y) : nullptr;
    e.y = static_cast<T *>(y);
    return spmv_launch<T>(ctx, A, static_cast<const T *>(x), e, false);
}

int spmv_args(spx_ctx *ctx, const spx_matrix *A, const void *x, void *y)
{
    if (!ctx || !A) return fail(SPX_ERR_INVALID, "spx_spmv: ctx or A is NULL");
    if ((A->n > 0 && !y) || (A->ncols > 0 && A->nnz > 0 && !x)) return fail(SPX_ERR_INVALID, "spx_spmv: NULL vector");
    if (A->ctx->device != ctx->device) return fail(SPX_ERR_INVALID, "matrix and context on different devices");
    const size_t V = A->dtype == SPX_F64 ? 8 : 4;
    const char *xb = static_cast<const char *>(x), *yb = static_cast<const char *>(y);
    if (x && y && xb < yb + (size_t)A->n * V && yb < xb + (size_t)A->ncols * V)
        return fail(SPX_ERR_INVALID, "spx_spmv: x and y overlap");
    return SPX_OK;
}
}  // namespace

extern "C" int spx_spmv(spx_ctx *ctx, const spx_matrix *A, const void *x, void *y)
{
    SPX_TRY(spmv_args(ctx, A, x, y));
    DeviceGuard g(ctx->device);
    return A->dtype == SPX_F64 ? spmv_common<double>(ctx, A, 1.0, x, 0.0, y, false)
                               : spmv_common<float>(ctx, A, 1.0, x, 0.0, y, false);
}

extern "C" int spx_spmv_axpby(spx_ctx *ctx, const spx_matrix *A, double alpha, const void *x, double beta,
                              void *y)
{
    SPX_TRY(spmv_args(ctx, A, x, y));
    DeviceGuard g(ctx->device);
    return A->dtype == SPX_F64 ? spmv_common<double>(ctx, A, alpha, x, beta, y, true)
                               : spmv_common<float>(ctx, A, alpha, x, beta, y, true);
}

extern "C" int spx_spmv_host(spx_ctx *ctx, const spx_matrix *Ac, const void *x_host, void *y_host)
{
    if (!ctx || !Ac || (Ac->ncols > 0 && !x_host) || (Ac->n > 0 && !y_host))
        return fail(SPX_ERR_INVALID, "spx_spmv_host: NULL argument");
    spx_matrix *A = const_cast<spx_matrix *>(Ac);
    DeviceGuard g(ctx->device);
    const size_t V = A->dtype == SPX_F64 ? 8 : 4;
    if (!A->stage_x.p) SPX_TRY(dbuf_alloc(ctx, A->stage_x, (size_t)A->ncols * V));
    if (!A->stage_y.p) SPX_TRY(dbuf_alloc(ctx, A->stage_y, (size_t)A->n * V));
    if (A->ncols) SPX_CUDA(cudaMemcpyAsync(A->stage_x.p, x_host, (size_t)A->ncols * V, cudaMemcpyHostToDevice, ctx->stream));
    SPX_TRY(A->dtype == SPX_F64 ? spmv_common<double>(ctx, A, 1.0, A->stage_x.p, 0.0, A->stage_y.p, false)
                                : spmv_common<float>(ctx, A, 1.0, A->stage_x.p, 0.0, A->stage_y.p, false));
    if (A->n) SPX_CUDA(cudaMemcpyAsync(y_host, A->stage_y.p, (size_t)A->n * V, cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    return SPX_OK;
}

// ------------------------------------------------------------------ BLAS-1
extern "C" int spx_dot(spx_ctx *ctx, int dtype, int64_t n, const void *x, const void *y, void *result)
{
    if (!ctx || n < 0 || (n > 0 && (!x || !y)) || !result) return fail(SPX_ERR_INVALID, "spx_dot: bad argument");
    DeviceGuard g(ctx->device);
    if (dtype == SPX_F64)
        return dot_launch<double>(ctx, n, static_cast<const double *>(x), static_cast<const double *>(y),
                                  static_cast<double *>(result));
    if (dtype == SPX_F32)
        return dot_launch<float>(ctx, n, static_cast<const float *>(x), static_cast<const float *>(y),
                                 static_cast<float *>(result));
    return fail(SPX_ERR_INVALID, "spx_dot: bad dtype");
}

extern "C" int spx_axpby(spx_ctx *ctx, int dtype, int64_t n, double alpha, const void *x, double beta, void *y)
{
    if (!ctx || n < 0 || (n > 0 && (!x || !y))) return fail(SPX_ERR_INVALID, "spx_axpby: bad argument");
    DeviceGuard g(ctx->device);
    if (dtype == SPX_F64)
        return axpby_launch<double>(ctx, n, alpha, static_cast<const double *>(x), beta, static_cast<double *>(y));
    if (dtype == SPX_F32)
        return axpby_launch<float>(ctx, n, (float)alpha, static_cast<const float *>(x), (float)beta,
                                   static_cast<float *>(y));
    return fail(SPX_ERR_INVALID, "spx_axpby: bad dtype");
}

// ------------------------------------------------------------------ errors
extern "C" const char *spx_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *spx_status_str(int status)
{
    switch (status) {
    case SPX_OK: return "SPX_OK";
    case SPX_ERR_INVALID: return "SPX_ERR_INVALID";
    case SPX_ERR_TOO_LARGE: return "SPX_ERR_TOO_LARGE";
    case SPX_ERR_OOM: return "SPX_ERR_OOM";
    case SPX_ERR_CUDA: return "SPX_ERR_CUDA";
    case SPX_ERR_UNSUPPORTED: return "SPX_ERR_UNSUPPORTED";
    case SPX_ERR_TIMEOUT: return "SPX_ERR_TIMEOUT";
    case SPX_ERR_NOT_FOUND: return "SPX_ERR_NOT_FOUND";
    default: return "SPX_ERR_UNKNOWN";
    }
}

extern "C" int spx_version(void) { return 100; }
