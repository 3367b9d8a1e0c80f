// cluster.cu -- whole solves in one launch on one thread-block cluster: CG for
// small systems with its vectors in shared memory (this part), and CG, BiCGSTAB
// or CGS of any size with its vectors in global memory (k_cluster_solve, below).
//
// A system of at most 16 * 4096 rows is solved by one cluster of 16 thread
// blocks on 16 SMs (8 where the device runs no cluster of 16), launched once
// for the whole solve.  Block k owns rows
// [k R, (k+1) R) (R a power of two) and keeps its slices of x, r, p and q in
// its shared memory; the product A p reads the entries of p it needs from
// the other blocks' shared memory through the cluster's distributed shared
// memory, and the dot products are summed by every block from the block
// partials in one fixed order, so all blocks take the same decisions and the
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

#include <map>
#include <mutex>

#include "dev_common.cuh"
#include "krylov_rows.cuh"
#include "spx_internal.cuh"

namespace cg = cooperative_groups;

namespace spx {
namespace {

constexpr int kClMaxRowsPerBlock = 4096;
constexpr size_t kOutBytes = 64;  // the result record of either cluster solve

struct ClOut {
    int status;
    int restarts;
    long long iters;
    double relres;
};

// Sum of v over the cluster: block sums, then in every block warp 0 adds the CL
// block partials in one fixed shuffle order (the same bits in every block) and
// shares the total through shared memory.  (Every thread reading all CL remote
// partials took CL distributed-shared-memory loads per thread per sum.)  `slot`
// alternates between the reductions of an iteration; see the barrier argument
// in k_cluster_cg.  bc is rewritten by the next sum only after its block
// barriers, which every thread reaches after reading it.
template <class T, int CL, int BLOCK>
__device__ __forceinline__ T cluster_sum(cg::cluster_group &cl, T v, T *red, T *part, int slot)
{
    __shared__ T bc;
    v = block_sum<T, BLOCK>(v, red);
    if (threadIdx.x == 0) part[slot] = v;
    cl.sync();
    if (threadIdx.x < 32) {
        T p = threadIdx.x < CL ? *cl.map_shared_rank(part + slot, (unsigned)threadIdx.x) : T(0);
        p = warp_sum(p);
        if (threadIdx.x == 0) bc = p;
    }
    __syncthreads();
    return bc;
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
__global__ void __launch_bounds__(BLOCK, 1)  // one block per SM: no register cap, no spills
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
// Asked once per (device, shared-memory size).
template <class T, int CL, int BLOCK> int cluster_fits(int smem)
{
    auto kern = k_cluster_cg<T, CL, BLOCK>;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> known;  // (device, smem) -> clusters
    std::lock_guard<std::mutex> lk(mu);
    auto it = known.find({dev, smem});
    if (it != known.end()) return it->second;
    int &nc = known[{dev, smem}];
    nc = 0;
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
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        nc = 0;
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
    if (!A->small_out.p) SPX_TRY(dbuf_alloc(ctx, A->small_out, kOutBytes));  // stream-ordered with its use
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

// ------------------------------------------------------------------ one system per cluster, any size
// The solve of a mid-size system (tens of thousands to about a million rows)
// on the general path is a chain of hundreds of launches of kernels with a
// few microseconds of work each: launch and drain latency, not memory, bound
// it (a 97 336-row 7-point stencil: 20.6 us per FP32 CG iteration for about
// 1.5 us of HBM traffic).  Here one cluster of CL blocks runs the whole solve
// in one launch (krylov_rows.cuh with the cluster group): block k owns rows
// [k R, (k+1) R), the vectors live in a global workspace of 8 doubles per row
// that stays in L2 for such sizes, the gathered vector is read through L2
// after a cluster barrier, and the group sums go through distributed shared
// memory.  One cluster uses 16 (or 8) SMs, so a lone large solve is faster on
// the general path; many such solves on separate streams (the request server)
// run side by side with no launch between iterations, though sixteen at once
// completed only three to four times the solves per second of one, and each
// thread walking its own row makes rows of many random columns costly (one
// warp's column and value loads touch up to 32 lines).  Measured faster than
// the general path for short rows up to a few tens of thousands of rows.
template <class T, int CL, int BLOCK, int SOLVER, bool MIXED>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK)
    k_cluster_solve(int n, const int *__restrict__ rp, const int *__restrict__ col, const T *__restrict__ val,
                    const float *__restrict__ val32, const T *__restrict__ b, T *__restrict__ x, T *__restrict__ work,
                    T tol, long long maxit, SysOut *out)
{
    __shared__ T red[BLOCK / 32];
    __shared__ float redf[BLOCK / 32];
    __shared__ double part[8];
    __shared__ double bc[2];
    const int rank = (int)cg::this_cluster().block_rank();
    const int R = ((n + CL - 1) / CL + 31) & ~31;  // n <= 2^30: no overflow
    ClusterRows<CL, BLOCK> g;
    g.lo = min(n, rank * R);
    g.hi = min(n, g.lo + R);
    g.part = part;
    g.bc = bc;
    const SysOut o = solve_rows<T, BLOCK, SOLVER, MIXED>(g, rp, col, val, val32, b, x, work, n, 0, nullptr, red,
                                                         redf, tol, maxit);
    if (rank == 0 && threadIdx.x == 0) *out = o;
    cg::this_cluster().sync();  // no block exits while another may still read its shared memory
}

namespace {

constexpr int kClSolveBlock = 512;

template <class T, int CL, int SOLVER, bool MIXED> cudaLaunchConfig_t cl_cfg(cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kClSolveBlock);
    cfg.dynamicSmemBytes = 0;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// Clusters of CL blocks of this kernel the device can hold at once (0: none),
// asked once per (kernel, device): the query takes driver locks, and the
// request server's slots launch this kernel from many threads at once.
template <class T, int CL, int SOLVER, bool MIXED> int cl_solve_fits()
{
    auto kern = k_cluster_solve<T, CL, kClSolveBlock, SOLVER, MIXED>;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    static std::mutex mu;
    static std::map<int, int> known;  // device -> clusters
    std::lock_guard<std::mutex> lk(mu);
    auto it = known.find(dev);
    if (it != known.end()) return it->second;
    int nc = 0;
    if (CL > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
    } else {
        cudaLaunchAttribute at[1];
        cudaLaunchConfig_t cfg = cl_cfg<T, CL, SOLVER, MIXED>(at);
        if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
            cudaGetLastError();
            nc = 0;
        }
    }
    known[dev] = nc;
    return nc;
}

template <class T, int CL, int SOLVER, bool MIXED>
int cl_solve_launch(spx_ctx *ctx, spx_matrix *A, const T *b, T *x, double tol, int64_t maxit, SysOut *out)
{
    auto kern = k_cluster_solve<T, CL, kClSolveBlock, SOLVER, MIXED>;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cl_cfg<T, CL, SOLVER, MIXED>(at);
    cfg.stream = ctx->stream;
    const float *v32 = MIXED ? A->val32.as<float>() : nullptr;
    SPX_CUDA(cudaLaunchKernelEx(&cfg, kern, (int)A->n, (const int *)A->rp.as<int>(), (const int *)A->col.as<int>(),
                                (const T *)A->val.as<T>(), v32, b, x, A->cl_work.as<T>(), (T)tol, (long long)maxit,
                                out));
    return SPX_OK;
}

// Clusters of 16 blocks for systems of at least 65 536 rows (8 rows per thread),
// where the device runs such clusters; else 8 blocks.
constexpr int64_t kClSolve16Rows = 65536;

template <class T, int SOLVER, bool MIXED>
int cl_solve_typed(spx_ctx *ctx, spx_matrix *A, const T *b, T *x, double tol, int64_t maxit, SysOut *out)
{
    if (A->n >= kClSolve16Rows && cl_solve_fits<T, 16, SOLVER, MIXED>() > 0)
        return cl_solve_launch<T, 16, SOLVER, MIXED>(ctx, A, b, x, tol, maxit, out);
    if (cl_solve_fits<T, 8, SOLVER, MIXED>() > 0) return cl_solve_launch<T, 8, SOLVER, MIXED>(ctx, A, b, x, tol, maxit, out);
    return SPX_ERR_UNSUPPORTED;
}

template <class T, bool MIXED>
int cl_solve_solver(spx_ctx *ctx, spx_matrix *A, int solver, const T *b, T *x, double tol, int64_t maxit, SysOut *out)
{
    if (solver == SPX_CG) return cl_solve_typed<T, SPX_CG, MIXED>(ctx, A, b, x, tol, maxit, out);
    if (solver == SPX_CGS) return cl_solve_typed<T, SPX_CGS, MIXED>(ctx, A, b, x, tol, maxit, out);
    return cl_solve_typed<T, SPX_BICGSTAB, MIXED>(ctx, A, b, x, tol, maxit, out);
}

}  // namespace

int cluster_solve(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, int solver, double tol, int64_t maxit,
                  int precision, spx_solve_info *info)
{
    if (A->format != SPX_CSR || !A->rp.p)
        return fail(SPX_ERR_UNSUPPORTED, "the one-cluster solve runs on CSR matrices");
    if (solver != SPX_CG && solver != SPX_BICGSTAB && solver != SPX_CGS)
        return fail(SPX_ERR_UNSUPPORTED, "the one-cluster solve runs CG, BiCGSTAB or CGS");
    const bool mixed = precision == SPX_PREC_MIXED;
    if (mixed && (A->dtype != SPX_F64 || !A->val32.p))
        return fail(SPX_ERR_UNSUPPORTED, "mixed precision needs an FP64 matrix created with SPX_MIXED_SHADOW");
    if (!mixed && (precision == SPX_PREC_F64 ? SPX_F64 : SPX_F32) != A->dtype)
        return fail(SPX_ERR_UNSUPPORTED, "precision must match the matrix dtype (or use MIXED)");
    if (A->n > (int64_t)1 << 30) return fail(SPX_ERR_TOO_LARGE, "the one-cluster solve takes at most 2^30 rows");
    if (!A->small_out.p) SPX_TRY(dbuf_alloc(ctx, A->small_out, kOutBytes));  // stream-ordered with its use
    if (!A->cl_work.p) SPX_TRY(dbuf_alloc(ctx, A->cl_work, (size_t)A->n * 64));
    SysOut *out = reinterpret_cast<SysOut *>(A->small_out.p);
    int st;
    if (mixed)
        st = cl_solve_solver<double, true>(ctx, A, solver, static_cast<const double *>(b), static_cast<double *>(x),
                                           tol, maxit, out);
    else if (A->dtype == SPX_F64)
        st = cl_solve_solver<double, false>(ctx, A, solver, static_cast<const double *>(b), static_cast<double *>(x),
                                            tol, maxit, out);
    else
        st = cl_solve_solver<float, false>(ctx, A, solver, static_cast<const float *>(b), static_cast<float *>(x), tol,
                                           maxit, out);
    if (st == SPX_ERR_UNSUPPORTED) return fail(st, "no thread-block cluster of 8 or 16 blocks fits this device");
    if (st != SPX_OK) return st;
    SysOut h;
    SPX_CUDA(cudaMemcpyAsync(&h, out, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    info->status = h.status;
    info->iterations = h.iters;
    info->relres_recurrence = h.relres;
    info->relres_true = h.relres;
    if (mixed) {
        info->inner_iterations = h.iters;
        info->restarts = h.cycles;
    }
    return SPX_OK;
}

}  // namespace spx
