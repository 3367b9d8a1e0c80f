// blas1.cu -- vector kernels: deterministic dot product and axpby.
//
// The dot product needs one device-wide reduction (Section 6.2 notes that
// the Dot kernel, which needs a global synchronisation, runs below streaming
// bandwidth).  Here it is one launch: a fixed grid, block partials in a fixed
// order, and the last block to finish sums the partials in index order, so
// the result does not depend on scheduling.
#include "dev_common.cuh"
#include "spx_internal.cuh"

namespace spx {

constexpr int kDotBlock = 256;

template <class T>
__global__ void __launch_bounds__(kDotBlock)
    k_dot(int64_t n, const T *__restrict__ x, const T *__restrict__ y, T *partials, unsigned *ticket,
          T *result)
{
    __shared__ T red[kDotBlock / 32];
    T s = T(0);
    for (int64_t i = blockIdx.x * (int64_t)kDotBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kDotBlock)
        s = fma(x[i], y[i], s);
    s = block_sum<T, kDotBlock>(s, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (!last_block(ticket, gridDim.x)) return;
    T t = T(0);
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kDotBlock) t += ldcg(partials + b);
    t = block_sum<T, kDotBlock>(t, red);
    if (threadIdx.x == 0) *result = t;
}

template <class T>
__global__ void k_axpby(int64_t n, T alpha, const T *__restrict__ x, T beta, T *__restrict__ y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = beta == T(0) ? alpha * x[i] : fma(alpha, x[i], beta * y[i]);
}

template <class T> int dot_launch(spx_ctx *ctx, int64_t n, const T *x, const T *y, T *result)
{
    int64_t g = ceil_div(n, kDotBlock * 4);
    if (g > ctx->red_grid) g = ctx->red_grid;
    if (g > (int64_t)ctx->grid_sms * 4) g = (int64_t)ctx->grid_sms * 4;
    if (g < 1) g = 1;
    T *partials = static_cast<T *>(ctx->red);
    unsigned *ticket = reinterpret_cast<unsigned *>(static_cast<char *>(ctx->red) +
                                                    (size_t)(2 * ctx->red_grid) * 8);
    k_dot<T><<<(int)g, kDotBlock, 0, ctx->stream>>>(n, x, y, partials, ticket, result);
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

template <class T> int axpby_launch(spx_ctx *ctx, int64_t n, T alpha, const T *x, T beta, T *y)
{
    if (n == 0) return SPX_OK;
    int64_t g = ceil_div(n, 256);
    if (g > (int64_t)ctx->grid_sms * 8) g = (int64_t)ctx->grid_sms * 8;
    k_axpby<T><<<(int)g, 256, 0, ctx->stream>>>(n, alpha, x, beta, y);
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

template int dot_launch<double>(spx_ctx *, int64_t, const double *, const double *, double *);
template int dot_launch<float>(spx_ctx *, int64_t, const float *, const float *, float *);
template int axpby_launch<double>(spx_ctx *, int64_t, double, const double *, double, double *);
template int axpby_launch<float>(spx_ctx *, int64_t, float, const float *, float, float *);

}  // namespace spx
