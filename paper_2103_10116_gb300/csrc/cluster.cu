// cluster.cu -- CG on one thread-block cluster for small systems.
//
// A system of at most 8 * 4096 rows is solved by one cluster of 8 thread
// blocks on 8 SMs, launched once for the whole solve.  Block k owns rows
// [k R, (k+1) R) (R a power of two) and keeps its slices of x, r, p and q in
// its shared memory; the product A p reads the entries of p it needs from
// the other blocks' shared memory through the cluster's distributed shared
// memory, and the dot products are summed by every block from the eight block
// partials in rank order, so all blocks take the same decisions and the
// result does not depend on timing.  An iteration costs three cluster
// barriers and no kernel launch.  The textbook CG recurrences (Hestenes and
// Stiefel, the form the Krylov solvers of Section 5 follow), then the true
// residual at exit with at most three restarts, as the general path does.
//
// Why a cluster: one SM alone is bound by its two FP64 lanes (the 2D
// Laplacian on a 64 x 64 grid, about 40 thousand FMAs per CG iteration, takes
// 20 us per iteration on one block); the general path spreads an iteration
// over the whole GPU but pays three launches and a device-wide reduction
// (23 us per iteration).
#include <cooperative_groups.h>

#include "dev_common.cuh"
#include "spx_internal.cuh"

namespace cg = cooperative_groups;

namespace spx {
namespace {

constexpr int kCl = 8;         // blocks per cluster (the portable maximum)
constexpr int kClBlock = 512;  // threads per block
constexpr int kClMaxRowsPerBlock = 4096;

struct ClOut {
    int status;
    int restarts;
    long long iters;
    double relres;
};

// Sum of v over the cluster: block sums, then every block adds the kCl
// block partials in rank order (the same bits in every block).  `slot`
// alternates between the reductions of an iteration; see the barrier
// argument in k_cluster_cg.
template <class T>
__device__ __forceinline__ T cluster_sum(cg::cluster_group &cl, T v, T *red, T *part, int slot)
{
    v = block_sum<T, kClBlock>(v, red);
    if (threadIdx.x == 0) part[slot] = v;
    cl.sync();
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kCl; ++k) s += *cl.map_shared_rank(part + slot, k);
    return s;
}

// (A v)_i for the local row i (global row g) with v distributed over the
// cluster's shared memory (slices of R = 2^lg entries).
template <class T>
__device__ __forceinline__ T dist_row_dot(cg::cluster_group &cl, const int *__restrict__ rp,
                                          const int *__restrict__ col, const T *__restrict__ val, T *vs, int lg,
                                          int g)
{
    const int mask = (1 << lg) - 1;
    T s = T(0);
    const int a = rp[g], b = rp[g + 1];
    for (int k = a; k < b; ++k) {
        const int c = col[k];
        const T *src = cl.map_shared_rank(vs, c >> lg);
        s = fma(val[k], src[c & mask], s);
    }
    return s;
}

template <class T>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClBlock)
    k_cluster_cg(int n, int lg, const int *__restrict__ rp, const int *__restrict__ col, const T *__restrict__ val,
                 const T *__restrict__ b, T *__restrict__ x, T tol, long long maxit, ClOut *out)
{
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int R = 1 << lg;
    const int r0 = rank * R;
    const int nr = max(0, min(n - r0, R));
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ps = reinterpret_cast<T *>(smem_raw);  // p (also x while the residual is formed)
    T *rs = ps + R;
    T *xs = rs + R;
    T *qs = xs + R;
    __shared__ T red[kClBlock / 32];
    __shared__ T part[4];
    __shared__ T sc[2];  // alpha and beta, computed by thread 0 (a division is many FP64 instructions)
    const int tid = threadIdx.x;

    T bb = T(0);
    for (int i = tid; i < nr; i += kClBlock) {
        const T bi = b[r0 + i];
        bb = fma(bi, bi, bb);
        xs[i] = x[r0 + i];
    }
    bb = cluster_sum<T>(cl, bb, red, part, 2);
    ClOut res{SPX_MAX_ITER, 0, 0, 0.0};
    if (bb == T(0)) {
        for (int i = tid; i < nr; i += kClBlock) xs[i] = T(0);
        res.status = SPX_CONVERGED;
    } else {
        const T tol2 = tol * tol * bb;
        long long iters = 0;
        for (int restart = 0;; ++restart) {
            // r = b - A x, p = r, rho = r.r  (x is exchanged through ps)
            for (int i = tid; i < nr; i += kClBlock) ps[i] = xs[i];
            cl.sync();
            T rho = T(0);
            for (int i = tid; i < nr; i += kClBlock) {
                const T ri = b[r0 + i] - dist_row_dot<T>(cl, rp, col, val, ps, lg, r0 + i);
                rs[i] = ri;
                rho = fma(ri, ri, rho);
            }
            rho = cluster_sum<T>(cl, rho, red, part, 3);  // every block is past its reads of ps
            for (int i = tid; i < nr; i += kClBlock) ps[i] = rs[i];
            cl.sync();
            T last = rho;  // the last recurrence residual, squared
            int status = rho <= tol2 ? SPX_CONVERGED : SPX_MAX_ITER;
            // Per iteration: A p reads remote p; barrier S1 (in the pq sum); x, r
            // updates; S2 (in the rr sum); p update; S3.  A block rewrites part[0]
            // only after S3 of the previous iteration, when every block has read
            // it (right after S1); likewise part[1] (read after S2).  p changes
            // only between S2 and S3, when no block reads it.
            while (status == SPX_MAX_ITER && iters < maxit) {
                T pq = T(0);
                for (int i = tid; i < nr; i += kClBlock) {
                    const T qi = dist_row_dot<T>(cl, rp, col, val, ps, lg, r0 + i);
                    qs[i] = qi;
                    pq = fma(ps[i], qi, pq);
                }
                pq = cluster_sum<T>(cl, pq, red, part, 0);
                if (pq == T(0)) {
                    status = SPX_BREAKDOWN;
                    break;
                }
                if (tid == 0) sc[0] = rho / pq;
                __syncthreads();
                const T alpha = sc[0];
                T rr = T(0);
                for (int i = tid; i < nr; i += kClBlock) {
                    xs[i] = fma(alpha, ps[i], xs[i]);
                    const T ri = fma(-alpha, qs[i], rs[i]);
                    rs[i] = ri;
                    rr = fma(ri, ri, rr);
                }
                rr = cluster_sum<T>(cl, rr, red, part, 1);
                ++iters;
                last = rr;
                if (rr <= tol2) {
                    status = SPX_CONVERGED;
                    break;
                }
                if (tid == 0) sc[1] = rr / rho;
                __syncthreads();
                const T beta = sc[1];
                rho = rr;
                for (int i = tid; i < nr; i += kClBlock) ps[i] = fma(beta, ps[i], rs[i]);
                cl.sync();
            }
            res.status = status;
            res.relres = (double)sqrt(last / bb);
            res.iters = iters;
            res.restarts = restart;
            if (status != SPX_CONVERGED) break;
            // the true residual ||b - A x|| / ||b||
            cl.sync();  // every block is past its reads of ps
            for (int i = tid; i < nr; i += kClBlock) ps[i] = xs[i];
            cl.sync();
            T rt = T(0);
            for (int i = tid; i < nr; i += kClBlock) {
                const T ri = b[r0 + i] - dist_row_dot<T>(cl, rp, col, val, ps, lg, r0 + i);
                rt = fma(ri, ri, rt);
            }
            rt = cluster_sum<T>(cl, rt, red, part, 2);
            res.relres = (double)sqrt(rt / bb);
            if (rt <= tol2) break;
            if (restart == 3) {
                res.status = SPX_STAGNATED;
                break;
            }
            cl.sync();
        }
    }
    for (int i = tid; i < nr; i += kClBlock) x[r0 + i] = xs[i];
    if (rank == 0 && tid == 0) *out = res;
    cl.sync();  // no block leaves while another may still read its shared memory
}

}  // namespace

int cluster_cg_max_rows() { return kCl * kClMaxRowsPerBlock; }

// CG on one cluster (see the file comment); synchronous.  b, x: device, dtype
// of A (FP64 or FP32); x holds the initial guess.  SPX_ERR_UNSUPPORTED when
// the matrix is not a CSR matrix of at most cluster_cg_max_rows() rows.
int cluster_cg_solve(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, double tol, int64_t maxit,
                     spx_solve_info *info)
{
    if (A->format != SPX_CSR || !A->rp.p || A->n < 1 || A->n > cluster_cg_max_rows()) return SPX_ERR_UNSUPPORTED;
    int lg = 0;
    while ((int64_t)kCl << lg < A->n) ++lg;
    const size_t V = A->dtype == SPX_F64 ? 8 : 4;
    const int smem = (int)(4 * ((size_t)1 << lg) * V);
    if (!A->small_out.p) SPX_TRY(dbuf_alloc(A->ctx, A->small_out, sizeof(ClOut)));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCl);
    cfg.blockDim = dim3(kClBlock);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = ctx->stream;
    ClOut *out = A->small_out.as<ClOut>();
    if (A->dtype == SPX_F64) {
        auto kern = k_cluster_cg<double>;
        SPX_TRY(smem_optin(reinterpret_cast<const void *>(kern), smem));
        SPX_CUDA(cudaLaunchKernelEx(&cfg, kern, (int)A->n, lg, (const int *)A->rp.as<int>(),
                                    (const int *)A->col.as<int>(), (const double *)A->val.as<double>(),
                                    static_cast<const double *>(b), static_cast<double *>(x), tol,
                                    (long long)maxit, out));
    } else {
        auto kern = k_cluster_cg<float>;
        SPX_TRY(smem_optin(reinterpret_cast<const void *>(kern), smem));
        SPX_CUDA(cudaLaunchKernelEx(&cfg, kern, (int)A->n, lg, (const int *)A->rp.as<int>(),
                                    (const int *)A->col.as<int>(), (const float *)A->val.as<float>(),
                                    static_cast<const float *>(b), static_cast<float *>(x), (float)tol,
                                    (long long)maxit, out));
    }
    ClOut h;
    SPX_CUDA(cudaMemcpyAsync(&h, out, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    info->status = h.status;
    info->iterations = h.iters;
    info->restarts = h.restarts;
    info->relres_recurrence = h.relres;
    info->relres_true = h.relres;
    return SPX_OK;
}

}  // namespace spx
