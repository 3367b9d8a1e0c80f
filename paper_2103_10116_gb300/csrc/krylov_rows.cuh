// krylov_rows.cuh -- one system solved entirely on the device by a group of
// threads that owns its rows: CG, BiCGSTAB, CGS (Section 5's Krylov methods,
// the textbook recurrences in the order the general path runs them) and FP64
// iterative refinement around an FP32 inner solve.
//
// The group is either one thread block that owns all rows of the system (the
// persistent batched kernel, batch.cu) or the blocks of one thread-block
// cluster, block k owning a contiguous slice of rows (the single-launch solve
// of a mid-size system, cluster.cu).  A group provides
//   lo, hi       the rows of this block;
//   sum(v, red)  the sum of v over the group's threads, the same bits in every
//                thread of every block (fixed reduction order);
//   sum2(a, b)   two such sums at the cost of one group barrier;
//   sync()       a barrier after which every block sees the others' writes of
//                the vector a product gathers from;
//   gather(v, c) a read of entry c of such a vector.
// Every thread of the group keeps the same rows in every loop (row i belongs to
// thread (i - lo) mod BLOCK of its block), so only the gathered vectors are
// read by threads other than their writers.  Scalars (alpha, beta, omega) are
// formed by thread 0 of each block from group sums that are equal in every
// block, so all blocks take the same decisions.
#pragma once

#include <cooperative_groups.h>

#include "dev_common.cuh"
#include "spx_internal.cuh"

namespace spx {

constexpr int kGroupMaxRestarts = 3;

// One thread block owns rows [0, n).
template <int BLOCK> struct BlockRows {
    static constexpr int U = 1;  // rows per thread in flight in a product
    int lo, hi;
    __device__ explicit BlockRows(int n) : lo(0), hi(n) {}
    __device__ __forceinline__ void sync() { __syncthreads(); }
    template <class T> __device__ __forceinline__ T sum(T v, T *red) { return block_sum<T, BLOCK>(v, red); }
    template <class T> __device__ __forceinline__ void sum2(T &a, T &b, T *red)
    {
        a = block_sum<T, BLOCK>(a, red);
        b = block_sum<T, BLOCK>(b, red);
    }
    template <class T> __device__ __forceinline__ T gather(const T *v, int c) const { return v[c]; }
};

// The CL blocks of one cluster; block k owns rows [k R, (k+1) R) (R a
// multiple of 32).  A sum adds the block partials, published in each block's
// shared memory, in a fixed tree order over the ranks; a partial slot is
// rewritten only four sums later, by when every block has passed a later
// cluster barrier and so finished reading it.  Gathered vectors are written
// with plain stores and read through L2 (ld.global.cg) after a cluster
// barrier (release / acquire at cluster scope).
template <int CL, int BLOCK, int UROWS = 2> struct ClusterRows {
    static_assert(CL >= 2 && CL <= 32, "cluster size");
    static constexpr int U = UROWS;  // rows per thread in flight in a product
    int lo, hi;
    double *part;  // shared: [2][4] partial slots of this block
    double *bc;    // shared: [2] broadcast of the totals
    int slot = 0;
    __device__ __forceinline__ void sync() { cooperative_groups::this_cluster().sync(); }
    // warp 0 adds the CL partials of slot `which` (tree order, lanes past CL add
    // zero) and leaves the total in bc[which]
    template <class T> __device__ __forceinline__ void combine(int which)
    {
        if (threadIdx.x < 32) {
            T p = T(0);
            if (threadIdx.x < CL)
                p = (T)*cooperative_groups::this_cluster().map_shared_rank(part + which * 4 + slot,
                                                                           (unsigned)threadIdx.x);
            p = warp_sum(p);
            if (threadIdx.x == 0) bc[which] = (double)p;
        }
    }
    template <class T> __device__ __forceinline__ T sum(T v, T *red)
    {
        v = block_sum<T, BLOCK>(v, red);
        if (threadIdx.x == 0) part[slot] = (double)v;  // exact for float and double
        sync();
        combine<T>(0);
        __syncthreads();
        const T s = (T)bc[0];  // rewritten by the next sum only past its block barriers
        slot = (slot + 1) & 3;
        return s;
    }
    template <class T> __device__ __forceinline__ void sum2(T &a, T &b, T *red)
    {
        a = block_sum<T, BLOCK>(a, red);
        b = block_sum<T, BLOCK>(b, red);
        if (threadIdx.x == 0) {
            part[slot] = (double)a;
            part[4 + slot] = (double)b;
        }
        sync();
        combine<T>(0);
        combine<T>(1);
        __syncthreads();
        a = (T)bc[0];
        b = (T)bc[1];
        slot = (slot + 1) & 3;
    }
    template <class T> __device__ __forceinline__ T gather(const T *v, int c) const { return __ldcg(v + c); }
};

// (A x)_i for row i, x gathered through the group
template <class T, class V, class G>
__device__ __forceinline__ T row_dot(const G &g, const int *__restrict__ rp, const int *__restrict__ col,
                                     const V *__restrict__ val, const T *xs, int i)
{
    T s = T(0);
    const int a = rp[i], b = rp[i + 1];
    for (int k = a; k < b; ++k) s = fma((T)val[k], g.gather(xs, col[k]), s);
    return s;
}

// A product over the rows this thread owns: t = (A x)_i, then body(i, t), rows
// in ascending order.  G::U rows are reduced at once with their loads
// interleaved, so a thread has U gathers in flight instead of one; each row is
// still summed in index order, so the bits do not depend on U.
template <class T, class V, int BLOCK, class G, class F>
__device__ __forceinline__ void product_rows(const G &g, const int *__restrict__ rp, const int *__restrict__ col,
                                             const V *__restrict__ val, const T *xs, F body)
{
    constexpr int U = G::U;
    if constexpr (U == 1) {
        for (int i = g.lo + (int)threadIdx.x; i < g.hi; i += BLOCK) body(i, row_dot<T, V>(g, rp, col, val, xs, i));
    } else {
        for (int i0 = g.lo + (int)threadIdx.x; i0 < g.hi; i0 += U * BLOCK) {
            int a[U], e[U];
            T s[U];
            int len = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * BLOCK;
                a[u] = i < g.hi ? rp[i] : 0;
                e[u] = i < g.hi ? rp[i + 1] : 0;
                s[u] = T(0);
                len = max(len, e[u] - a[u]);
            }
            for (int k = 0; k < len; ++k) {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (a[u] + k < e[u]) s[u] = fma((T)val[a[u] + k], g.gather(xs, col[a[u] + k]), s[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (i0 + u * BLOCK < g.hi) body(i0 + u * BLOCK, s[u]);
        }
    }
}

// The scalars of an iteration (alpha, beta, omega) are computed once per block,
// by thread 0, and read from shared memory: a division is a sequence of FP64
// instructions, and every thread of the block computing it cost as much FP64
// issue as a fifth of a small system's iteration (ncu: the FP64 pipe 78% busy
// on one 4096-row system).  Slot k is written once per iteration and read right
// after the barrier that follows the write; the group sums between two writes
// of a slot end every read of it.
template <class T> __device__ __forceinline__ T share_scalar(T v, T *slot)
{
    if (threadIdx.x == 0) *slot = v;
    __syncthreads();
    return *slot;
}

#define SPX_OWN_ROWS(i) for (int i = g.lo + (int)threadIdx.x; i < g.hi; i += BLOCK)

// CG in precision T on values V (V = T, or float values in the FP32 inner
// solve).  x: initial guess (zero_x0: start from 0).  check_true: form the true
// residual at exit and restart from x if it misses tol.  ps: the vector the
// products gather from.
template <class T, class V, int BLOCK, class G>
__device__ int cg_rows(G &g, const int *__restrict__ rp, const int *__restrict__ col, const V *__restrict__ val,
                       const T *__restrict__ b, T *__restrict__ x, T *__restrict__ r, T *__restrict__ q, T *ps,
                       T *red, T tol, long long maxit, bool zero_x0, bool check_true, long long &iters, T &relres)
{
    __shared__ T sc[2];
    T bb = T(0);
    SPX_OWN_ROWS(i) bb = fma(b[i], b[i], bb);
    bb = g.sum(bb, red);
    if (bb == T(0)) {
        SPX_OWN_ROWS(i) x[i] = T(0);
        relres = T(0);
        return SPX_CONVERGED;
    }
    const T tol2 = tol * tol * bb;
    if (zero_x0) SPX_OWN_ROWS(i) x[i] = T(0);
    int status = SPX_MAX_ITER;
    for (int restart = 0;; ++restart) {
        // r = b - A x ; p = r ; rho = r.r
        SPX_OWN_ROWS(i) ps[i] = x[i];
        g.sync();
        T rho = T(0);
        product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T t) {
            const T ri = b[i] - t;
            r[i] = ri;
            rho = fma(ri, ri, rho);
        });
        rho = g.sum(rho, red);  // every gather of ps is done
        SPX_OWN_ROWS(i) ps[i] = r[i];
        g.sync();
        T last = rho;  // the last recurrence residual, squared
        status = rho <= tol2 ? SPX_CONVERGED : SPX_MAX_ITER;
        while (status == SPX_MAX_ITER && iters < maxit) {
            T pq = T(0);
            product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T qi) {
                q[i] = qi;
                pq = fma(ps[i], qi, pq);
            });
            pq = g.sum(pq, red);
            if (pq == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            const T alpha = share_scalar(threadIdx.x == 0 ? rho / pq : T(0), &sc[0]);
            T rr = T(0);
            SPX_OWN_ROWS(i)
            {
                x[i] = fma(alpha, ps[i], x[i]);
                const T ri = fma(-alpha, q[i], r[i]);
                r[i] = ri;
                rr = fma(ri, ri, rr);
            }
            rr = g.sum(rr, red);
            ++iters;
            last = rr;
            if (rr <= tol2) {
                status = SPX_CONVERGED;
                break;
            }
            const T beta = share_scalar(threadIdx.x == 0 ? rr / rho : T(0), &sc[1]);
            rho = rr;
            SPX_OWN_ROWS(i) ps[i] = fma(beta, ps[i], r[i]);
            g.sync();
        }
        if (threadIdx.x == 0) relres = sqrt(last / bb);
        if (!check_true || status != SPX_CONVERGED) break;
        // true residual
        g.sync();
        SPX_OWN_ROWS(i) ps[i] = x[i];
        g.sync();
        T rt = T(0);
        product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T t) {
            const T ri = b[i] - t;
            rt = fma(ri, ri, rt);
        });
        rt = g.sum(rt, red);
        relres = sqrt(rt / bb);
        if (rt <= tol2) break;
        if (restart == kGroupMaxRestarts) {
            status = SPX_STAGNATED;
            break;
        }
    }
    __syncthreads();
    return status;
}

// BiCGSTAB (r^ = r0), vectors r, rh, p, v, s, t in w[0..5]; the vector a
// product gathers from is staged in ps.
template <class T, class V, int BLOCK, class G>
__device__ int bicgstab_rows(G &g, const int *__restrict__ rp, const int *__restrict__ col,
                             const V *__restrict__ val, const T *__restrict__ b, T *__restrict__ x, T *const *w, T *ps,
                             T *red, T tol, long long maxit, bool zero_x0, bool check_true, long long &iters,
                             T &relres)
{
    __shared__ T sc[3];
    T *r = w[0], *rh = w[1], *p = w[2], *v = w[3], *s = w[4], *t = w[5];
    T bb = T(0);
    SPX_OWN_ROWS(i) bb = fma(b[i], b[i], bb);
    bb = g.sum(bb, red);
    if (bb == T(0)) {
        SPX_OWN_ROWS(i) x[i] = T(0);
        relres = T(0);
        return SPX_CONVERGED;
    }
    const T tol2 = tol * tol * bb;
    if (zero_x0) SPX_OWN_ROWS(i) x[i] = T(0);
    int status = SPX_MAX_ITER;
    for (int restart = 0;; ++restart) {
        SPX_OWN_ROWS(i) ps[i] = x[i];
        g.sync();
        T rr0 = T(0);
        product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T t) {
            const T ri = b[i] - t;
            r[i] = ri;
            rh[i] = ri;
            p[i] = T(0);
            v[i] = T(0);
            rr0 = fma(ri, ri, rr0);
        });
        rr0 = g.sum(rr0, red);
        T rho = T(1), alpha = T(1), omega = T(1), rho1 = rr0;
        T last = rr0;  // the last recurrence residual, squared
        status = rr0 <= tol2 ? SPX_CONVERGED : SPX_MAX_ITER;
        while (status == SPX_MAX_ITER && iters < maxit) {
            if (rho1 == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            const T beta = share_scalar(threadIdx.x == 0 ? (rho1 / rho) * (alpha / omega) : T(0), &sc[0]);
            SPX_OWN_ROWS(i)
            {
                const T pi = fma(beta, fma(-omega, v[i], p[i]), r[i]);
                p[i] = pi;
                ps[i] = pi;
            }
            g.sync();
            T rv = T(0);
            product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T vi) {
                v[i] = vi;
                rv = fma(rh[i], vi, rv);
            });
            rv = g.sum(rv, red);
            if (rv == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            alpha = share_scalar(threadIdx.x == 0 ? rho1 / rv : T(0), &sc[1]);
            T ss = T(0);
            SPX_OWN_ROWS(i)
            {
                const T si = fma(-alpha, v[i], r[i]);
                s[i] = si;
                ps[i] = si;
                ss = fma(si, si, ss);
            }
            ss = g.sum(ss, red);  // its group barrier also publishes ps
            ++iters;
            if (ss <= tol2) {
                SPX_OWN_ROWS(i)
                {
                    x[i] = fma(alpha, p[i], x[i]);
                    r[i] = s[i];
                }
                last = ss;
                status = SPX_CONVERGED;
                __syncthreads();
                break;
            }
            T ts = T(0), tt = T(0);
            product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T ti) {
                t[i] = ti;
                ts = fma(ti, s[i], ts);
                tt = fma(ti, ti, tt);
            });
            g.sum2(ts, tt, red);
            if (tt == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            omega = share_scalar(threadIdx.x == 0 ? ts / tt : T(0), &sc[2]);
            T rr = T(0), rhr = T(0);
            SPX_OWN_ROWS(i)
            {
                x[i] = fma(omega, s[i], fma(alpha, p[i], x[i]));
                const T ri = fma(-omega, t[i], s[i]);
                r[i] = ri;
                rr = fma(ri, ri, rr);
                rhr = fma(rh[i], ri, rhr);
            }
            g.sum2(rr, rhr, red);
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
        if (threadIdx.x == 0) relres = sqrt(last / bb);
        if (!check_true || status != SPX_CONVERGED) break;
        g.sync();
        SPX_OWN_ROWS(i) ps[i] = x[i];
        g.sync();
        T rt = T(0);
        product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T t) {
            const T ri = b[i] - t;
            rt = fma(ri, ri, rt);
        });
        rt = g.sum(rt, red);
        relres = sqrt(rt / bb);
        if (rt <= tol2) break;
        if (restart == kGroupMaxRestarts) {
            status = SPX_STAGNATED;
            break;
        }
    }
    __syncthreads();
    return status;
}

// CGS (Sonneveld; shadow residual r^ = r0).  The product operands (p, then
// u + q) are staged in turn through ps.  stall > 0 (inner cycle of
// refinement, x0 = 0): also stop once the recurrence residual has gone `stall`
// iterations without halving.
template <class T, class V, int BLOCK, class G>
__device__ int cgs_rows(G &g, const int *__restrict__ rp, const int *__restrict__ col, const V *__restrict__ val,
                        const T *__restrict__ b, T *__restrict__ x, T *const *w, T *ps, T *red, T tol,
                        long long maxit, bool zero_x0, bool check_true, long long &iters, T &relres, int stall = 0)
{
    T mark2 = T(1);  // the squared relative residual the stall test measures against
    long long mark_it = iters;
    __shared__ T sc[2];
    T *r = w[0], *rh = w[1], *p = w[2], *u = w[3], *q = w[4], *v = w[5];
    T bb = T(0);
    SPX_OWN_ROWS(i) bb = fma(b[i], b[i], bb);
    bb = g.sum(bb, red);
    if (bb == T(0)) {
        SPX_OWN_ROWS(i) x[i] = T(0);
        relres = T(0);
        return SPX_CONVERGED;
    }
    const T tol2 = tol * tol * bb;
    if (zero_x0) SPX_OWN_ROWS(i) x[i] = T(0);
    int status = SPX_MAX_ITER;
    for (int restart = 0;; ++restart) {
        SPX_OWN_ROWS(i) ps[i] = x[i];
        g.sync();
        T rr0 = T(0);
        product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T t) {
            const T ri = b[i] - t;
            r[i] = ri;
            rh[i] = ri;
            p[i] = ri;
            u[i] = ri;
            rr0 = fma(ri, ri, rr0);
        });
        rr0 = g.sum(rr0, red);  // (its barrier also ends every gather of ps)
        SPX_OWN_ROWS(i) ps[i] = p[i];
        g.sync();
        T rho = rr0;
        T last = rr0;  // the last recurrence residual, squared
        status = rr0 <= tol2 ? SPX_CONVERGED : SPX_MAX_ITER;
        while (status == SPX_MAX_ITER && iters < maxit) {
            if (rho == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            T rv = T(0);
            product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T vi) {  // v = A p
                v[i] = vi;
                rv = fma(rh[i], vi, rv);
            });
            rv = g.sum(rv, red);
            if (rv == T(0)) {
                status = SPX_BREAKDOWN;
                break;
            }
            const T alpha = share_scalar(threadIdx.x == 0 ? rho / rv : T(0), &sc[0]);
            SPX_OWN_ROWS(i)
            {
                const T qi = fma(-alpha, v[i], u[i]);
                q[i] = qi;
                const T wi = u[i] + qi;
                x[i] = fma(alpha, wi, x[i]);
                ps[i] = wi;
            }
            g.sync();
            T rr = T(0), rhr = T(0);
            product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T t) {  // r -= alpha A (u + q)
                const T ri = fma(-alpha, t, r[i]);
                r[i] = ri;
                rr = fma(ri, ri, rr);
                rhr = fma(rh[i], ri, rhr);
            });
            g.sum2(rr, rhr, red);
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
            const T beta = share_scalar(threadIdx.x == 0 ? rhr / rho : T(0), &sc[1]);
            SPX_OWN_ROWS(i)
            {
                const T ui = fma(beta, q[i], r[i]);
                u[i] = ui;
                const T pi = fma(beta, fma(beta, p[i], q[i]), ui);
                p[i] = pi;
                ps[i] = pi;
            }
            g.sync();
            rho = rhr;
        }
        if (threadIdx.x == 0) relres = sqrt(last / bb);
        if (!check_true || status != SPX_CONVERGED) break;
        g.sync();
        SPX_OWN_ROWS(i) ps[i] = x[i];
        g.sync();
        T rt = T(0);
        product_rows<T, V, BLOCK>(g, rp, col, val, ps, [&](int i, T t) {
            const T ri = b[i] - t;
            rt = fma(ri, ri, rt);
        });
        rt = g.sum(rt, red);
        relres = sqrt(rt / bb);
        if (rt <= tol2) break;
        if (restart == kGroupMaxRestarts) {
            status = SPX_STAGNATED;
            break;
        }
    }
    __syncthreads();
    return status;
}

// Mixed-precision CG with reliable updates (the residual replacement of
// Sleijpen and van der Vorst, 1996), the iteration spx_solve runs for MIXED CG:
// FP32 CG on the FP32 values, its iterate accumulated in an FP32 correction y.
// When the FP32 recurrence residual has fallen below delta = 0.1 of its largest
// value since the last update (compared in squares), or to tol ||b||, or the
// budget is spent, y is added to the FP64 x, the residual b - A x is formed in
// FP64 with the FP64 values and its rounding replaces the FP32 residual; the
// direction p is kept and beta is formed with the replaced residual, so the
// solve keeps CG's iteration count.  p is the vector the FP32 products gather
// from; the FP64 residual gathers x itself.  updates: the reliable updates.
constexpr float kRuDelta2 = 0.01f;  // delta^2, delta = 0.1

template <int BLOCK, class G>
__device__ int cg_reliable_rows(G &g, const int *__restrict__ rp, const int *__restrict__ col,
                                const double *__restrict__ val, const float *__restrict__ v32,
                                const double *__restrict__ b, double *__restrict__ x, double *__restrict__ r64,
                                float *__restrict__ r32, float *__restrict__ y, float *__restrict__ q, float *p,
                                double *red, float *redf, double tol, long long maxit, long long &iters,
                                double &relres, int &updates)
{
    __shared__ float sc[2];
    double bb = 0.0;
    SPX_OWN_ROWS(i) bb = fma(b[i], b[i], bb);
    bb = g.sum(bb, red);
    if (bb == 0.0) {
        SPX_OWN_ROWS(i) x[i] = 0.0;
        relres = 0.0;
        return SPX_CONVERGED;
    }
    const double tol2_64 = tol * tol * bb;
    const float tol2 = (float)tol2_64;
    // r64 = b - A x in FP64 (x gathered as written), returns ||r64||^2
    auto fp64_residual = [&]() -> double {
        g.sync();
        double rr = 0.0;
        product_rows<double, double, BLOCK>(g, rp, col, val, x, [&](int i, double t) {
            const double ri = b[i] - t;
            r64[i] = ri;
            rr = fma(ri, ri, rr);
        });
        return g.sum(rr, red);
    };
    double rr64 = fp64_residual();
    relres = sqrt(rr64 / bb);
    if (rr64 <= tol2_64) return SPX_CONVERGED;
    float rho = 0.f;
    SPX_OWN_ROWS(i)
    {
        const float ri = (float)r64[i];
        r32[i] = ri;
        p[i] = ri;
        y[i] = 0.f;
        rho = fmaf(ri, ri, rho);
    }
    rho = g.sum(rho, redf);  // its group barrier also publishes p
    float maxr2 = rho;
    int status = SPX_MAX_ITER;
    while (iters < maxit) {
        float pq = 0.f;
        product_rows<float, float, BLOCK>(g, rp, col, v32, p, [&](int i, float qi) {
            q[i] = qi;
            pq = fmaf(p[i], qi, pq);
        });
        pq = g.sum(pq, redf);
        if (pq == 0.f) {
            status = SPX_BREAKDOWN;
            break;
        }
        const float alpha = share_scalar(threadIdx.x == 0 ? rho / pq : 0.f, &sc[0]);
        float rr = 0.f;
        SPX_OWN_ROWS(i)
        {
            y[i] = fmaf(alpha, p[i], y[i]);
            const float ri = fmaf(-alpha, q[i], r32[i]);
            r32[i] = ri;
            rr = fmaf(ri, ri, rr);
        }
        rr = g.sum(rr, redf);
        ++iters;
        if (rr > maxr2) maxr2 = rr;
        if (rr <= tol2 || iters >= maxit || rr < kRuDelta2 * maxr2) {  // reliable update
            SPX_OWN_ROWS(i)
            {
                x[i] += (double)y[i];
                y[i] = 0.f;
            }
            rr64 = fp64_residual();
            ++updates;
            relres = sqrt(rr64 / bb);
            if (rr64 <= tol2_64) {
                status = SPX_CONVERGED;
                break;
            }
            if (iters >= maxit) break;
            float r2 = 0.f;
            SPX_OWN_ROWS(i)
            {
                const float ri = (float)r64[i];
                r32[i] = ri;
                r2 = fmaf(ri, ri, r2);
            }
            rr = g.sum(r2, redf);
            maxr2 = rr;
        }
        const float beta = share_scalar(threadIdx.x == 0 ? rr / rho : 0.f, &sc[1]);
        rho = rr;
        SPX_OWN_ROWS(i) p[i] = fmaf(beta, p[i], r32[i]);
        g.sync();
    }
    __syncthreads();
    return status;
}

// Result of one system: status, refinement cycles (mixed precision, else 0),
// Krylov iterations, last relative residual.
struct SysOut {
    int status;
    int cycles;
    long long iters;
    double relres;
};

// Solve one system (SOLVER = SPX_CG / SPX_BICGSTAB / SPX_CGS).  The workspace
// is a batch-wide array of 8 doubles per row (nrows rows in all, this system's
// rows starting at ro):
//   one precision: vectors k = 0..5 at work + k nrows + ro (T), the gathered
//                  vector at slot 6;
//   MIXED:         r64 at slot 0 (double); FP32 vectors from slot 1 on (r32, d32
//                  and six inner vectors: 8 float vectors in 4 double slots); the
//                  gathered FP64 x at slot 6, the gathered FP32 vector at slot 7.
// MIXED: CG runs with reliable updates (cg_reliable_rows; cycles = updates);
// BiCGSTAB and CGS run FP64 refinement (r = b - A64 x, x += ||r|| d) around an
// FP32 inner solve of A32 d = r / ||r|| to 1e-4 on float values, at most
// kIrInnerCap inner iterations per cycle and 20 cycles.  smem_vec: the gathered vector in shared
// memory, or null for the global slots.  Every thread returns the same record
// (relres is exact in thread 0).
template <class T, int BLOCK, int SOLVER, bool MIXED, class G>
__device__ SysOut solve_rows(G &g, const int *__restrict__ rp, const int *__restrict__ col,
                             const T *__restrict__ val_all, const float *__restrict__ v32, const T *__restrict__ b,
                             T *__restrict__ x, T *__restrict__ work, int64_t nrows, int64_t ro, void *smem_vec,
                             T *red, float *redf, T tol, long long maxit)
{
    long long iters = 0;
    T relres = T(0);
    int status;
    int outer = 0;
    if constexpr (!MIXED) {
        T *ps = smem_vec ? reinterpret_cast<T *>(smem_vec) : work + 6 * nrows + ro;
        T *w[6];
        for (int k = 0; k < 6; ++k) w[k] = work + (int64_t)k * nrows + ro;
        if constexpr (SOLVER == SPX_CG)
            status = cg_rows<T, T, BLOCK>(g, rp, col, val_all, b, x, w[0], w[1], ps, red, tol, maxit, false, true,
                                          iters, relres);
        else if constexpr (SOLVER == SPX_CGS)
            status = cgs_rows<T, T, BLOCK>(g, rp, col, val_all, b, x, w, ps, red, tol, maxit, false, true, iters,
                                           relres);
        else
            status = bicgstab_rows<T, T, BLOCK>(g, rp, col, val_all, b, x, w, ps, red, tol, maxit, false, true,
                                                iters, relres);
    } else {
        static_assert(sizeof(T) == 8, "refinement runs on FP64 systems");
        const double *val = reinterpret_cast<const double *>(val_all);
        double *wd = reinterpret_cast<double *>(work);
        double *xs = smem_vec ? reinterpret_cast<double *>(smem_vec) : wd + 6 * nrows + ro;
        double *r64 = wd + ro;
        float *fw = reinterpret_cast<float *>(wd + nrows);
        float *r32 = fw + ro, *d32 = fw + nrows + ro;
        float *fv[6];
        for (int k = 0; k < 6; ++k) fv[k] = fw + (int64_t)(2 + k) * nrows + ro;
        float *ps32 = smem_vec ? reinterpret_cast<float *>(smem_vec) : reinterpret_cast<float *>(wd + 7 * nrows) + ro;
        const double *bd = reinterpret_cast<const double *>(b);
        double *xd = reinterpret_cast<double *>(x);
        double *redd = reinterpret_cast<double *>(red);
        if constexpr (SOLVER == SPX_CG) {  // reliable updates instead of restarted refinement cycles
            double rel = 0.0;
            status = cg_reliable_rows<BLOCK>(g, rp, col, val, v32, bd, xd, r64, r32, d32, fv[0], ps32, redd, redf,
                                             (double)tol, maxit, iters, rel, outer);
            return SysOut{status, outer, iters, rel};
        }
        double bb = 0.0;
        SPX_OWN_ROWS(i) bb = fma(bd[i], bd[i], bb);
        bb = g.sum(bb, redd);
        status = SPX_MAX_ITER;
        if (bb == 0.0) {
            SPX_OWN_ROWS(i) xd[i] = 0.0;
            status = SPX_CONVERGED;
        }
        for (outer = 0; status != SPX_CONVERGED && outer <= 20; ++outer) {
            SPX_OWN_ROWS(i) xs[i] = xd[i];
            g.sync();
            double rr = 0.0;
            product_rows<double, double, BLOCK>(g, rp, col, val, xs, [&](int i, double t) {
                const double ri = bd[i] - t;
                r64[i] = ri;
                rr = fma(ri, ri, rr);
            });
            rr = g.sum(rr, redd);
            relres = (T)sqrt(rr / bb);
            if (rr <= (double)tol * (double)tol * bb) {
                status = SPX_CONVERGED;
                break;
            }
            if (outer == 20 || iters >= maxit) break;
            const double rn = sqrt(rr);
            SPX_OWN_ROWS(i) r32[i] = (float)(r64[i] / rn);
            __syncthreads();
            float rel32 = 0.f;
            // at most kIrInnerCap inner iterations per refinement cycle
            const long long cyc_max = min(maxit, iters + (long long)kIrInnerCap);
            if constexpr (SOLVER == SPX_CG)
                cg_rows<float, float, BLOCK>(g, rp, col, v32, r32, d32, fv[0], fv[1], ps32, redf, 1e-4f, cyc_max,
                                             true, false, iters, rel32);
            else if constexpr (SOLVER == SPX_CGS)
                cgs_rows<float, float, BLOCK>(g, rp, col, v32, r32, d32, fv, ps32, redf, 1e-4f, cyc_max, true, false,
                                              iters, rel32, kIrCgsStall);
            else
                bicgstab_rows<float, float, BLOCK>(g, rp, col, v32, r32, d32, fv, ps32, redf, 1e-4f, cyc_max, true,
                                                   false, iters, rel32);
            SPX_OWN_ROWS(i) xd[i] = fma(rn, (double)d32[i], xd[i]);
            __syncthreads();
        }
    }
    return SysOut{status, outer, iters, (double)relres};
}

#undef SPX_OWN_ROWS

}  // namespace spx
