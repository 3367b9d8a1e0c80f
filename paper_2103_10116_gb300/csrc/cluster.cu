// cluster.cu -- CG on one thread-block cluster for small systems.
//
// A system of at most 16 * 4096 rows is solved by one cluster of 16 thread
// blocks on 16 SMs (8 where the device runs no cluster of 16), launched once
// for the whole solve.  Block k owns rows
// [k R, (k+1) R) (R a power of two) and keeps its slices of x, r, p and q in
// its shared memory; the product A p reads the entries of p it needs from
// the other blocks' shared memory through the cluster's distributed shared
// memory, and the dot products are summed by every block from the block
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

constexpr int kClMaxRowsPerBlock = 4096;

struct ClOut {
    int status;
    int restarts;
    long long iters;
    double relres;
};

// Sum of v over the cluster: block sums, then every block adds the CL
// block partials in rank order (the same bits in every block).  `slot`
// alternates between the reductions of an iteration; see the barrier
// argument in k_cluster_cg.
template <class T, int CL, int BLOCK>
__device__ __forceinline__ T cluster_sum(cg::cluster_group &cl, T v, T *red, T *part, int slot)
{
    v = block_sum<T, BLOCK>(v, red);
    if (threadIdx.x == 0) part[slot] = v;
    cl.sync();
    T s = T(0);
#pragma unroll
    for (int k = 0; k < CL; ++k) s += *cl.map_shared_rank(part + slot, k);
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

template <class T, int CL, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
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
    __shared__ T red[BLOCK / 32];
    __shared__ T part[4];
    __shared__ T sc[2];  // alpha and beta, computed by thread 0 (a division is many FP64 instructions)
    const int tid = threadIdx.x;

    T bb = T(0);
    for (int i = tid; i < nr; i += BLOCK) {
        const T bi = b[r0 + i];
        bb = fma(bi, bi, bb);
        xs[i] = x[r0 + i];
    }
    bb = cluster_sum<T, CL, BLOCK>(cl, bb, red, part, 2);
    ClOut res{SPX_MAX_ITER, 0, 0, 0.0};
    if (bb == T(0)) {
        for (int i = tid; i < nr; i += BLOCK) xs[i] = T(0);
        res.status = SPX_CONVERGED;
    } else {
        const T tol2 = tol * tol * bb;
        long long iters = 0;
        for (int restart = 0;; ++restart) {
            // r = b - A x, p = r, rho = r.r  (x is exchanged through ps)
            for (int i = tid; i < nr; i += BLOCK) ps[i] = xs[i];
            cl.sync();
            T rho = T(0);
            for (int i = tid; i < nr; i += BLOCK) {
                const T ri = b[r0 + i] - dist_row_dot<T>(cl, rp, col, val, ps, lg, r0 + i);
                rs[i] = ri;
                rho = fma(ri, ri, rho);
            }
            rho = cluster_sum<T, CL, BLOCK>(cl, rho, red, part, 3);  // every block is past its reads of ps
            for (int i = tid; i < nr; i += BLOCK) ps[i] = rs[i];
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
                for (int i = tid; i < nr; i += BLOCK) {
                    const T qi = dist_row_dot<T>(cl, rp, col, val, ps, lg, r0 + i);
                    qs[i] = qi;
                    pq = fma(ps[i], qi, pq);
                }
                pq = cluster_sum<T, CL, BLOCK>(cl, pq, red, part, 0);
                if (pq == T(0)) {
                    status = SPX_BREAKDOWN;
                    break;
                }
                if (tid == 0) sc[0] = rho / pq;
                __syncthreads();
                const T alpha = sc[0];
                T rr = T(0);
                for (int i = tid; i < nr; i += BLOCK) {
                    xs[i] = fma(alpha, ps[i], xs[i]);
                    const T ri = fma(-alpha, qs[i], rs[i]);
                    rs[i] = ri;
                    rr = fma(ri, ri, rr);
                }
                rr = cluster_sum<T, CL, BLOCK>(cl, rr, red, part, 1);
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
                for (int i = tid; i < nr; i += BLOCK) ps[i] = fma(beta, ps[i], rs[i]);
                cl.sync();
            }
            res.status = status;
            res.relres = (double)sqrt(last / bb);
            res.iters = iters;
            res.restarts = restart;
            if (status != SPX_CONVERGED) break;
            // the true residual ||b - A x|| / ||b||
            cl.sync();  // every block is past its reads of ps
            for (int i = tid; i < nr; i += BLOCK) ps[i] = xs[i];
            cl.sync();
            T rt = T(0);
            for (int i = tid; i < nr; i += BLOCK) {
                const T ri = b[r0 + i] - dist_row_dot<T>(cl, rp, col, val, ps, lg, r0 + i);
                rt = fma(ri, ri, rt);
            }
            rt = cluster_sum<T, CL, BLOCK>(cl, rt, red, part, 2);
            res.relres = (double)sqrt(rt / bb);
            if (rt <= tol2) break;
            if (restart == 3) {
                res.status = SPX_STAGNATED;
                break;
            }
            cl.sync();
        }
    }
    for (int i = tid; i < nr; i += BLOCK) x[r0 + i] = xs[i];
    if (rank == 0 && tid == 0) *out = res;
    cl.sync();  // no block leaves while another may still read its shared memory
}

}  // namespace

int cluster_cg_max_rows() { return 16 * kClMaxRowsPerBlock; }

namespace {

// The largest cluster (16 blocks, a non-portable size, else the portable 8)
// this device can run for the kernel's shared memory; 0 if none.
template <class T, int CL, int BLOCK> int cluster_fits(int smem)
{
    auto kern = k_cluster_cg<T, CL, BLOCK>;
    if (smem_optin(reinterpret_cast<const void *>(kern), smem) != SPX_OK) return 0;
    if (CL > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(BLOCK);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

template <class T, int CL, int BLOCK>
int launch_cluster_cg(spx_ctx *ctx, spx_matrix *A, int lg, const T *b, T *x, double tol, int64_t maxit, ClOut *out)
{
    const int smem = (int)(4 * ((size_t)1 << lg) * sizeof(T));
    auto kern = k_cluster_cg<T, CL, BLOCK>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(BLOCK);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    SPX_CUDA(cudaLaunchKernelEx(&cfg, kern, (int)A->n, lg, (const int *)A->rp.as<int>(),
                                (const int *)A->col.as<int>(), (const T *)A->val.as<T>(), b, x, (T)tol,
                                (long long)maxit, out));
    return SPX_OK;
}

template <class T>
int cluster_cg_typed(spx_ctx *ctx, spx_matrix *A, const T *b, T *x, double tol, int64_t maxit, ClOut *out)
{
    // 16 blocks of 256 threads where the device runs such a cluster, else 8 of 512
    int lg16 = 0, lg8 = 0;
    while ((int64_t)16 << lg16 < A->n) ++lg16;
    while ((int64_t)8 << lg8 < A->n) ++lg8;
    if ((1 << lg16) <= kClMaxRowsPerBlock && cluster_fits<T, 16, 256>((int)(4 * ((size_t)1 << lg16) * sizeof(T))) > 0)
        return launch_cluster_cg<T, 16, 256>(ctx, A, lg16, b, x, tol, maxit, out);
    if ((1 << lg8) <= kClMaxRowsPerBlock && cluster_fits<T, 8, 512>((int)(4 * ((size_t)1 << lg8) * sizeof(T))) > 0)
        return launch_cluster_cg<T, 8, 512>(ctx, A, lg8, b, x, tol, maxit, out);
    return SPX_ERR_UNSUPPORTED;
}

}  // namespace

// CG on one cluster (see the file comment); synchronous.  b, x: device, dtype
// of A (FP64 or FP32); x holds the initial guess.  SPX_ERR_UNSUPPORTED when
// the matrix is not a CSR matrix of at most cluster_cg_max_rows() rows or no
// cluster fits.
int cluster_cg_solve(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, double tol, int64_t maxit,
                     spx_solve_info *info)
{
    if (A->format != SPX_CSR || !A->rp.p || A->n < 1 || A->n > cluster_cg_max_rows()) return SPX_ERR_UNSUPPORTED;
    if (!A->small_out.p) SPX_TRY(dbuf_alloc(A->ctx, A->small_out, sizeof(ClOut)));
    ClOut *out = A->small_out.as<ClOut>();
    const int st = A->dtype == SPX_F64
                       ? cluster_cg_typed<double>(ctx, A, static_cast<const double *>(b), static_cast<double *>(x),
                                                  tol, maxit, out)
                       : cluster_cg_typed<float>(ctx, A, static_cast<const float *>(b), static_cast<float *>(x), tol,
                                                 maxit, out);
    if (st != SPX_OK) return st;
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
