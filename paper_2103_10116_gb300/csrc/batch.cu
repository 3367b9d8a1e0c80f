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
    void *host_out = nullptr;
    int block = 0;       // chosen threads per system (0 = not tuned: heuristic)
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey[10] = {0};
};

namespace spx {

constexpr int kBatchMaxRestarts = 3;

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

template <class T, int BLOCK> __device__ __forceinline__ T bsum(T v, T *red) { return block_sum<T, BLOCK>(v, red); }

// y_i = (A x)_i for the rows this thread owns, x in shared memory
template <class T, class V>
__device__ __forceinline__ T row_dot(const int *__restrict__ rp, const int *__restrict__ col,
                                     const V *__restrict__ val, const T *xs, int i)
{
    T s = T(0);
    const int a = rp[i], b = rp[i + 1];
    for (int k = a; k < b; ++k) s = fma((T)val[k], xs[col[k]], s);
    return s;
}

// The scalars of an iteration (alpha, beta, omega) are computed once per block,
// by thread 0, and read from shared memory: a division is a sequence of FP64
// instructions, and every thread of the block computing it cost as much FP64
// issue as a fifth of a small system's iteration (ncu: the FP64 pipe 78% busy
// on one 4096-row system).  Slot k is written once per iteration and read right
// after the barrier that follows the write; the block reductions between two
// writes of a slot end every read of it.
template <class T> __device__ __forceinline__ T share_scalar(T v, T *slot)
{
    if (threadIdx.x == 0) *slot = v;
    __syncthreads();
    return *slot;
}

// One system by CG in precision T on values V (V = T, or float values in the
// FP32 inner solve).  x: initial guess (zero_x0: start from 0).  check_true:
// form the true residual at exit and restart from x if it misses tol.
template <class T, class V, int BLOCK>
__device__ int cg_system(int n, const int *__restrict__ rp, const int *__restrict__ col, const V *__restrict__ val,
                         const T *__restrict__ b, T *__restrict__ x, T *__restrict__ r, T *__restrict__ q, T *ps,
                         T *red, T tol, long long maxit, bool zero_x0, bool check_true, long long &iters, T &relres)
{
    const int tid = threadIdx.x;
    __shared__ T sc[2];
    T bb = T(0);
    for (int i = tid; i < n; i += BLOCK) bb = fma(b[i], b[i], bb);
    bb = bsum<T, BLOCK>(bb, red);
    if (bb == T(0)) {
        for (int i = tid; i < n; i += BLOCK) x[i] = T(0);
        relres = T(0);
        return SPX_CONVERGED;
    }
    const T tol2 = tol * tol * bb;
    if (zero_x0)
        for (int i = tid; i < n; i += BLOCK) x[i] = T(0);
    int status = SPX_MAX_ITER;
    for (int restart = 0;; ++restart) {
        // r = b - A x ; p = r ; rho = r.r
        for (int i = tid; i < n; i += BLOCK) ps[i] = x[i];
        __syncthreads();
        T rho = T(0);
        for (int i = tid; i < n; i += BLOCK) {
            const T ri = b[i] - row_dot<T, V>(rp, col, val, ps, i);
            r[i] = ri;
            rho = fma(ri, ri, rho);
        }
        rho = bsum<T, BLOCK>(rho, red);  // (ends with a barrier: ps free)
        for (int i = tid; i < n; i += BLOCK) ps[i] = r[i];
        __syncthreads();
        T last = rho;  // the last recurrence residual, squared
        status = rho <= tol2 ? SPX_CONVERGED : SPX_MAX_ITER;
        while (status == SPX_MAX_ITER && iters < maxit) {
            T pq = T(0);
            for (int i = tid; i < n; i += BLOCK) {
                const T qi = row_dot<T, V>(rp, col, val, ps, i);
                q[i] = qi;
                pq = fma(ps[i], qi, pq);
            }
            pq = bsum<T, BLOCK>(pq, red);
            if (pq == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            const T alpha = share_scalar(tid == 0 ? rho / pq : T(0), &sc[0]);
            T rr = T(0);
            for (int i = tid; i < n; i += BLOCK) {
                x[i] = fma(alpha, ps[i], x[i]);
                const T ri = fma(-alpha, q[i], r[i]);
                r[i] = ri;
                rr = fma(ri, ri, rr);
            }
            rr = bsum<T, BLOCK>(rr, red);
            ++iters;
            last = rr;
            if (rr <= tol2) {
                status = SPX_CONVERGED;
                break;
            }
            const T beta = share_scalar(tid == 0 ? rr / rho : T(0), &sc[1]);
            rho = rr;
            for (int i = tid; i < n; i += BLOCK) ps[i] = fma(beta, ps[i], r[i]);
            __syncthreads();
        }
        if (tid == 0) relres = sqrt(last / bb);
        if (!check_true || status != SPX_CONVERGED) break;
        // true residual
        __syncthreads();
        for (int i = tid; i < n; i += BLOCK) ps[i] = x[i];
        __syncthreads();
        T rt = T(0);
        for (int i = tid; i < n; i += BLOCK) {
            const T ri = b[i] - row_dot<T, V>(rp, col, val, ps, i);
            rt = fma(ri, ri, rt);
        }
        rt = bsum<T, BLOCK>(rt, red);
        relres = sqrt(rt / bb);
        if (rt <= tol2) break;
        if (restart == kBatchMaxRestarts) {
            status = SPX_STAGNATED;
            break;
        }
    }
    __syncthreads();
    return status;
}

// One system by BiCGSTAB (r^ = r0), vectors r, rh, p, v, s, t in global
// workspace w[0..5]; the vector an SpMV gathers from is staged in ps.
template <class T, class V, int BLOCK>
__device__ int bicgstab_system(int n, const int *__restrict__ rp, const int *__restrict__ col,
                               const V *__restrict__ val, const T *__restrict__ b, T *__restrict__ x, T *const *w,
                               T *ps, T *red, T tol, long long maxit, bool zero_x0, bool check_true,
                               long long &iters, T &relres)
{
    const int tid = threadIdx.x;
    __shared__ T sc[3];
    T *r = w[0], *rh = w[1], *p = w[2], *v = w[3], *s = w[4], *t = w[5];
    T bb = T(0);
    for (int i = tid; i < n; i += BLOCK) bb = fma(b[i], b[i], bb);
    bb = bsum<T, BLOCK>(bb, red);
    if (bb == T(0)) {
        for (int i = tid; i < n; i += BLOCK) x[i] = T(0);
        relres = T(0);
        return SPX_CONVERGED;
    }
    const T tol2 = tol * tol * bb;
    if (zero_x0)
        for (int i = tid; i < n; i += BLOCK) x[i] = T(0);
    int status = SPX_MAX_ITER;
    for (int restart = 0;; ++restart) {
        for (int i = tid; i < n; i += BLOCK) ps[i] = x[i];
        __syncthreads();
        T rr0 = T(0);
        for (int i = tid; i < n; i += BLOCK) {
            const T ri = b[i] - row_dot<T, V>(rp, col, val, ps, i);
            r[i] = ri;
            rh[i] = ri;
            p[i] = T(0);
            v[i] = T(0);
            rr0 = fma(ri, ri, rr0);
        }
        rr0 = bsum<T, BLOCK>(rr0, red);
        T rho = T(1), alpha = T(1), omega = T(1), rho1 = rr0;
        T last = rr0;  // the last recurrence residual, squared
        status = rr0 <= tol2 ? SPX_CONVERGED : SPX_MAX_ITER;
        while (status == SPX_MAX_ITER && iters < maxit) {
            if (rho1 == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            const T beta = share_scalar(tid == 0 ? (rho1 / rho) * (alpha / omega) : T(0), &sc[0]);
            for (int i = tid; i < n; i += BLOCK) {
                const T pi = fma(beta, fma(-omega, v[i], p[i]), r[i]);
                p[i] = pi;
                ps[i] = pi;
            }
            __syncthreads();
            T rv = T(0);
            for (int i = tid; i < n; i += BLOCK) {
                const T vi = row_dot<T, V>(rp, col, val, ps, i);
                v[i] = vi;
                rv = fma(rh[i], vi, rv);
            }
            rv = bsum<T, BLOCK>(rv, red);
            if (rv == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            alpha = share_scalar(tid == 0 ? rho1 / rv : T(0), &sc[1]);
            T ss = T(0);
            for (int i = tid; i < n; i += BLOCK) {
                const T si = fma(-alpha, v[i], r[i]);
                s[i] = si;
                ps[i] = si;
                ss = fma(si, si, ss);
            }
            ss = bsum<T, BLOCK>(ss, red);
            ++iters;
            if (ss <= tol2) {
                for (int i = tid; i < n; i += BLOCK) {
                    x[i] = fma(alpha, p[i], x[i]);
                    r[i] = s[i];
                }
                last = ss;
                status = SPX_CONVERGED;
                __syncthreads();
                break;
            }
            T ts = T(0), tt = T(0);
            for (int i = tid; i < n; i += BLOCK) {
                const T ti = row_dot<T, V>(rp, col, val, ps, i);
                t[i] = ti;
                ts = fma(ti, s[i], ts);
                tt = fma(ti, ti, tt);
            }
            ts = bsum<T, BLOCK>(ts, red);
            tt = bsum<T, BLOCK>(tt, red);
            if (tt == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            omega = share_scalar(tid == 0 ? ts / tt : T(0), &sc[2]);
            T rr = T(0), rhr = T(0);
            for (int i = tid; i < n; i += BLOCK) {
                x[i] = fma(omega, s[i], fma(alpha, p[i], x[i]));
                const T ri = fma(-omega, t[i], s[i]);
                r[i] = ri;
                rr = fma(ri, ri, rr);
                rhr = fma(rh[i], ri, rhr);
            }
            rr = bsum<T, BLOCK>(rr, red);
            rhr = bsum<T, BLOCK>(rhr, red);
            last = rr;
            if (rr <= tol2) {
                status = SPX_CONVERGED;
                break;
            }
            if (omega == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            rho = rho1;
            rho1 = rhr;
        }
        if (tid == 0) relres = sqrt(last / bb);
        if (!check_true || status != SPX_CONVERGED) break;
        __syncthreads();
        for (int i = tid; i < n; i += BLOCK) ps[i] = x[i];
        __syncthreads();
        T rt = T(0);
        for (int i = tid; i < n; i += BLOCK) {
            const T ri = b[i] - row_dot<T, V>(rp, col, val, ps, i);
            rt = fma(ri, ri, rt);
        }
        rt = bsum<T, BLOCK>(rt, red);
        relres = sqrt(rt / bb);
        if (rt <= tol2) break;
        if (restart == kBatchMaxRestarts) {
            status = SPX_STAGNATED;
            break;
        }
    }
    __syncthreads();
    return status;
}

// One system by CGS (Sonneveld; shadow residual r^ = r0).  The SpMV operands
// (p, then u + q) are staged in turn through the shared-memory vector ps.
// stall > 0 (inner cycle of refinement, x0 = 0): also stop once the recurrence
// residual has gone `stall` iterations without halving.
template <class T, class V, int BLOCK>
__device__ int cgs_system(int n, const int *__restrict__ rp, const int *__restrict__ col, const V *__restrict__ val,
                          const T *__restrict__ b, T *__restrict__ x, T *const *w, T *ps, T *red, T tol,
                          long long maxit, bool zero_x0, bool check_true, long long &iters, T &relres,
                          int stall = 0)
{
    T mark2 = T(1);  // the squared relative residual the stall test measures against
    long long mark_it = iters;
    const int tid = threadIdx.x;
    __shared__ T sc[2];
    T *r = w[0], *rh = w[1], *p = w[2], *u = w[3], *q = w[4], *v = w[5];
    T bb = T(0);
    for (int i = tid; i < n; i += BLOCK) bb = fma(b[i], b[i], bb);
    bb = bsum<T, BLOCK>(bb, red);
    if (bb == T(0)) {
        for (int i = tid; i < n; i += BLOCK) x[i] = T(0);
        relres = T(0);
        return SPX_CONVERGED;
    }
    const T tol2 = tol * tol * bb;
    if (zero_x0)
        for (int i = tid; i < n; i += BLOCK) x[i] = T(0);
    int status = SPX_MAX_ITER;
    for (int restart = 0;; ++restart) {
        for (int i = tid; i < n; i += BLOCK) ps[i] = x[i];
        __syncthreads();
        T rr0 = T(0);
        for (int i = tid; i < n; i += BLOCK) {
            const T ri = b[i] - row_dot<T, V>(rp, col, val, ps, i);
            r[i] = ri;
            rh[i] = ri;
            p[i] = ri;
            u[i] = ri;
            rr0 = fma(ri, ri, rr0);
        }
        rr0 = bsum<T, BLOCK>(rr0, red);  // (its barrier also ends every read of ps)
        for (int i = tid; i < n; i += BLOCK) ps[i] = p[i];
        __syncthreads();
        T rho = rr0;
        T last = rr0;  // the last recurrence residual, squared
        status = rr0 <= tol2 ? SPX_CONVERGED : SPX_MAX_ITER;
        while (status == SPX_MAX_ITER && iters < maxit) {
            if (rho == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            T rv = T(0);
            for (int i = tid; i < n; i += BLOCK) {  // v = A p
                const T vi = row_dot<T, V>(rp, col, val, ps, i);
                v[i] = vi;
                rv = fma(rh[i], vi, rv);
            }
            rv = bsum<T, BLOCK>(rv, red);
            if (rv == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            const T alpha = share_scalar(tid == 0 ? rho / rv : T(0), &sc[0]);
            for (int i = tid; i < n; i += BLOCK) {
                const T qi = fma(-alpha, v[i], u[i]);
                q[i] = qi;
                const T wi = u[i] + qi;
                x[i] = fma(alpha, wi, x[i]);
                ps[i] = wi;
            }
            __syncthreads();
            T rr = T(0), rhr = T(0);
            for (int i = tid; i < n; i += BLOCK) {  // r -= alpha A (u + q)
                const T ri = fma(-alpha, row_dot<T, V>(rp, col, val, ps, i), r[i]);
                r[i] = ri;
                rr = fma(ri, ri, rr);
                rhr = fma(rh[i], ri, rhr);
            }
            rr = bsum<T, BLOCK>(rr, red);
            rhr = bsum<T, BLOCK>(rhr, red);
            ++iters;
            last = rr;
            if (rr <= tol2) {
                status = SPX_CONVERGED;
                break;
            }
            if (stall > 0) {  // ||r|| / ||b|| below half the mark, compared in squares
                if (rr < T(0.25) * mark2 * bb) {
                    mark2 = rr / bb;
                    mark_it = iters;
                } else if (iters - mark_it >= stall) {
                    status = SPX_STAGNATED;
                    break;
                }
            }
            const T beta = share_scalar(tid == 0 ? rhr / rho : T(0), &sc[1]);
            for (int i = tid; i < n; i += BLOCK) {
                const T ui = fma(beta, q[i], r[i]);
                u[i] = ui;
                const T pi = fma(beta, fma(beta, p[i], q[i]), ui);
                p[i] = pi;
                ps[i] = pi;
            }
            __syncthreads();
            rho = rhr;
        }
        if (tid == 0) relres = sqrt(last / bb);
        if (!check_true || status != SPX_CONVERGED) break;
        __syncthreads();
        for (int i = tid; i < n; i += BLOCK) ps[i] = x[i];
        __syncthreads();
        T rt = T(0);
        for (int i = tid; i < n; i += BLOCK) {
            const T ri = b[i] - row_dot<T, V>(rp, col, val, ps, i);
            rt = fma(ri, ri, rt);
        }
        rt = bsum<T, BLOCK>(rt, red);
        relres = sqrt(rt / bb);
        if (rt <= tol2) break;
        if (restart == kBatchMaxRestarts) {
            status = SPX_STAGNATED;
            break;
        }
    }
    __syncthreads();
    return status;
}

// The persistent kernel.  MIXED: FP64 refinement (r = b - A64 x, x += ||r|| d)
// around an FP32 inner solve of A32 d = r / ||r|| to 1e-4 on float values.
template <class T, int BLOCK, int SOLVER, bool MIXED>
__global__ void __launch_bounds__(BLOCK)
    k_batch(int64_t nsys, const int64_t *__restrict__ row_off, const int64_t *__restrict__ nnz_off,
            const int *__restrict__ rp_all, const int *__restrict__ col_all, const T *__restrict__ val_all,
            const float *__restrict__ val32_all, const int *__restrict__ order, const T *__restrict__ b_all,
            T *__restrict__ x_all, T *__restrict__ work, int64_t nrows, T tol, long long maxit, unsigned *queue,
            BOut out, int smem_vec)
{
    // The vector the products gather from lives in shared memory (smem_vec) or,
    // for systems too large for it, in the global workspace (slots 6 and 7 of
    // the eight per row; read through L1).
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
        const int n = (int)(row_off[s + 1] - ro);
        const int *rp = rp_all + ro + s;
        const int *col = col_all + nnz_off[s];
        const T *b = b_all + ro;
        T *x = x_all + ro;
        long long iters = 0;
        T relres = T(0);
        int status;
        int outer = 0;
        if (!MIXED) {
            const T *val = val_all + nnz_off[s];
            T *ps = smem_vec ? reinterpret_cast<T *>(smem) : work + 6 * nrows + ro;
            if (SOLVER == SPX_CG) {
                status = cg_system<T, T, BLOCK>(n, rp, col, val, b, x, work + ro, work + nrows + ro, ps, red, tol,
                                                maxit, false, true, iters, relres);
            } else if (SOLVER == SPX_CGS) {
                T *w[6];
                for (int k = 0; k < 6; ++k) w[k] = work + (int64_t)k * nrows + ro;
                status = cgs_system<T, T, BLOCK>(n, rp, col, val, b, x, w, ps, red, tol, maxit, false, true, iters,
                                                 relres);
            } else {
                T *w[6];
                for (int k = 0; k < 6; ++k) w[k] = work + (int64_t)k * nrows + ro;
                status = bicgstab_system<T, T, BLOCK>(n, rp, col, val, b, x, w, ps, red, tol, maxit, false, true,
                                                      iters, relres);
            }
        } else {
            // outer FP64 refinement
            const double *val = reinterpret_cast<const double *>(val_all) + nnz_off[s];
            const float *v32 = val32_all + nnz_off[s];
            double *xs = smem_vec ? reinterpret_cast<double *>(smem) : reinterpret_cast<double *>(work) + 6 * nrows + ro;
            double *r64 = reinterpret_cast<double *>(work) + ro;
            float *fw = reinterpret_cast<float *>(reinterpret_cast<double *>(work) + nrows);
            float *r32 = fw + ro, *d32 = fw + nrows + ro;
            float *fv[6];
            for (int k = 0; k < 6; ++k) fv[k] = fw + (int64_t)(2 + k) * nrows + ro;
            const double *bd = reinterpret_cast<const double *>(b);
            double *xd = reinterpret_cast<double *>(x);
            double bb = 0.0;
            for (int i = threadIdx.x; i < n; i += BLOCK) bb = fma(bd[i], bd[i], bb);
            bb = bsum<double, BLOCK>(bb, reinterpret_cast<double *>(red));
            status = SPX_MAX_ITER;
            if (bb == 0.0) {
                for (int i = threadIdx.x; i < n; i += BLOCK) xd[i] = 0.0;
                status = SPX_CONVERGED;
            }
            for (outer = 0; status != SPX_CONVERGED && outer <= 20; ++outer) {
                for (int i = threadIdx.x; i < n; i += BLOCK) xs[i] = xd[i];
                __syncthreads();
                double rr = 0.0;
                for (int i = threadIdx.x; i < n; i += BLOCK) {
                    const double ri = bd[i] - row_dot<double, double>(rp, col, val, xs, i);
                    r64[i] = ri;
                    rr = fma(ri, ri, rr);
                }
                rr = bsum<double, BLOCK>(rr, reinterpret_cast<double *>(red));
                relres = (T)sqrt(rr / bb);
                if (rr <= (double)tol * (double)tol * bb) {
                    status = SPX_CONVERGED;
                    break;
                }
                if (outer == 20 || iters >= maxit) break;
                const double rn = sqrt(rr);
                for (int i = threadIdx.x; i < n; i += BLOCK) r32[i] = (float)(r64[i] / rn);
                __syncthreads();
                float rel32 = 0.f;
                float *ps32 = smem_vec ? reinterpret_cast<float *>(smem)
                                       : reinterpret_cast<float *>(reinterpret_cast<double *>(work) + 7 * nrows) + ro;
                // at most kIrInnerCap inner iterations per refinement cycle
                const long long cyc_max = min(maxit, iters + (long long)kIrInnerCap);
                if (SOLVER == SPX_CG)
                    cg_system<float, float, BLOCK>(n, rp, col, v32, r32, d32, fv[0], fv[1], ps32, redf, 1e-4f,
                                                   cyc_max, true, false, iters, rel32);
                else if (SOLVER == SPX_CGS)
                    cgs_system<float, float, BLOCK>(n, rp, col, v32, r32, d32, fv, ps32, redf, 1e-4f, cyc_max, true,
                                                    false, iters, rel32, kIrCgsStall);
                else
                    bicgstab_system<float, float, BLOCK>(n, rp, col, v32, r32, d32, fv, ps32, redf, 1e-4f, cyc_max,
                                                         true, false, iters, rel32);
                for (int i = threadIdx.x; i < n; i += BLOCK) xd[i] = fma(rn, (double)d32[i], xd[i]);
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) {
            out.status[s] = status;
            out.iters[s] = iters;
            out.relres[s] = (double)relres;
            out.cycles[s] = outer;
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
    int64_t grid = (int64_t)per_sm * ctx->sm_count;
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
            k_cast_f32<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(nnz, B->val.as<double>(), B->val32.as<float>());
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMallocHost(&B->host_out, bout_bytes(nsys) + 64);
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
                        (uint64_t)max_iter, (uint64_t)block, (uint64_t)(uintptr_t)ctx->stream, 0, 0};
    std::memcpy(&key[4], &tol, 8);
    bool same = use_graph && B->gexec;
    for (int i = 0; i < 10 && same; ++i) same = B->gkey[i] == key[i];
    auto body = [&]() -> int {
        SPX_TRY(launch_batch(ctx, B, block, solver, precision, b, x, tol, max_iter));
        SPX_CUDA(cudaMemcpyAsync(B->host_out, B->out.p, out_bytes, cudaMemcpyDeviceToHost, ctx->stream));
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
        const char *h = static_cast<const char *>(B->host_out);
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
