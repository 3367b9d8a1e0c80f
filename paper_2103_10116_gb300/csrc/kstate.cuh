// kstate.cuh -- device-resident scalar state of a Krylov solve and the scalar
// updates that the last block of a fused kernel runs after its reduction.
//
// Keeping alpha, beta, omega, rho and the convergence flag on the device
// means an iteration needs no host round trip: every kernel of an iteration
// first reads `done` and returns at once when the solve has stopped, so the
// host may enqueue (or replay in a CUDA graph) several iterations ahead and
// look at the flag only every few iterations.
#pragma once

#include <math.h>

#include "dev_common.cuh"
#include "spx_internal.cuh"

namespace spx {

template <class T> struct KState {
    T rho;     // CG: r.r ; BiCGSTAB: r^.r of the current iteration (rho_i)
    T alpha, beta, omega;
    T bb;      // ||b||^2
    T tol2;    // (tol * ||b||)^2: squared-norm threshold
    T relres;  // last recurrence relative residual
    T rtol2;   // tol^2 (relative, set by the host)
    int done;     // nonzero: every kernel of the iteration returns at once
    int skip_t;   // BiCGSTAB: skip the t = A s half (set with s-convergence or done)
    int status;   // spx_solve_status once done
    int s_conv;   // BiCGSTAB: converged on s, x += alpha p still to apply
    long long iters;
    long long maxit;
    // stall rule of an inner CGS cycle (stall > 0): the cycle ends once the
    // recurrence residual has not fallen below half of `mark` for `stall`
    // iterations; mark starts at 1 (x0 = 0) and is lowered at each halving
    T mark;
    long long mark_it;
    int stall;
    // reliable updates (FP32 CG inside FP64 residual replacement): when
    // ru_delta2 > 0 the iteration also stops, for an update, once r.r has
    // fallen below ru_delta2 times its largest value since the last update
    // (maxr2); 0 in every other solve
    T ru_delta2;
    T maxr2;
};

enum : int {
    FIN_NONE = 0,
    FIN_CG_ALPHA = 1,   // dots[0] = p.q              -> alpha = rho / (p.q)
    FIN_CG_RHO = 2,     // dots[0] = r.r              -> convergence, beta, rho
    FIN_BI_RV = 3,      // dots[0] = r^.v             -> alpha
    FIN_BI_S = 4,       // dots[0] = s.s              -> early convergence on s
    FIN_BI_OMEGA = 5,   // dots[0] = t.s, dots[1] = t.t -> omega
    FIN_BI_R = 6,       // dots[0] = r.r, dots[1] = r^.r -> convergence, beta, rho
    FIN_INIT_CG = 7,    // dots[1] = r.r              -> initial rho (CG)
    FIN_INIT_BI = 8,    // dots[1] = r.r (r^ = r)     -> initial rho = r^.r = r.r, beta
    FIN_SET_BB = 9,     // dots[0] = b.b              -> ||b||^2 and the absolute threshold
    FIN_CGS_R = 10,     // dots[0] = r.r, dots[1] = r^.r -> convergence, beta = (r^.r)' / (r^.r), rho
    FIN_PCG_RHO0 = 11,  // dots[0] = r.z (z = M^-1 r)  -> initial rho of preconditioned CG
    FIN_PCG_R = 12,     // dots[0] = r.r, dots[1] = r.z -> convergence on r, beta = (r.z)' / (r.z), rho
    FIN_CG_RR = 13,     // dots[0] = r.r              -> convergence only (block-PCG: r.z comes next)
    FIN_PCG_RZ = 14,    // dots[0] = r.z (z = M^-1 r) -> beta = (r.z)' / (r.z), rho (block-PCG)
    FIN_RU_FIRST = 15,  // dots[0] = r.r of the first FP32 residual -> rho, maxr2; iterating again
    FIN_RU_NEXT = 16,   // dots[0] = r.r of a replaced FP32 residual -> beta with it, rho, maxr2
};

template <class T> __device__ __forceinline__ void kstop(KState<T> *s, int status)
{
    s->done = 1;
    s->skip_t = 1;
    s->status = status;
}

// Runs in one thread of the last block of a fused kernel, after dots[] are final.
template <class T> __device__ __forceinline__ void run_fin(int fin, void *state, const T *dots)
{
    if (fin == FIN_NONE || state == nullptr) return;
    KState<T> *s = static_cast<KState<T> *>(state);
    switch (fin) {
    case FIN_SET_BB: {
        s->bb = dots[0];
        s->tol2 = s->rtol2 * dots[0];
        break;
    }
    case FIN_INIT_CG:
    case FIN_INIT_BI: {  // (re)start from the current x; the iteration count carries on
        const T rr = dots[1];
        s->relres = s->bb > T(0) ? sqrt(rr / s->bb) : T(0);
        s->rho = rr;
        s->alpha = T(1);
        s->omega = T(1);
        s->beta = rr;  // BiCGSTAB: (rho_0 / 1) * (1 / 1) with p = v = 0 gives p = r
        s->s_conv = 0;
        s->done = 0;
        s->skip_t = 0;
        s->status = SPX_MAX_ITER;
        if (rr <= s->tol2) kstop(s, SPX_CONVERGED);
        else if (s->iters >= s->maxit) kstop(s, SPX_MAX_ITER);
        break;
    }
    case FIN_CG_ALPHA: {
        const T pq = dots[0];
        if (pq == T(0)) kstop(s, SPX_BREAKDOWN);
        else s->alpha = s->rho / pq;
        break;
    }
    case FIN_CG_RHO: {
        const T rr = dots[0];
        s->iters += 1;
        s->relres = sqrt(rr / s->bb);
        if (rr <= s->tol2) { kstop(s, SPX_CONVERGED); break; }
        if (s->iters >= s->maxit) { kstop(s, SPX_MAX_ITER); break; }
        if (s->ru_delta2 > T(0)) {  // due for a reliable update: the host replaces r, keeps p
            if (rr > s->maxr2) s->maxr2 = rr;
            if (rr < s->ru_delta2 * s->maxr2) { kstop(s, SPX_CONVERGED); break; }
        }
        s->beta = rr / s->rho;
        s->rho = rr;
        break;
    }
    case FIN_RU_FIRST:
    case FIN_RU_NEXT: {  // r holds the rounding of the FP64 residual; p = r (first) or r + beta p
        const T rr = dots[0];
        s->beta = fin == FIN_RU_NEXT ? rr / s->rho : T(0);
        s->rho = rr;
        s->maxr2 = rr;
        s->done = 0;
        s->skip_t = 0;
        s->status = SPX_MAX_ITER;
        if (s->iters >= s->maxit) kstop(s, SPX_MAX_ITER);
        break;
    }
    case FIN_BI_RV: {
        const T rv = dots[0];
        if (rv == T(0)) kstop(s, SPX_BREAKDOWN);
        else s->alpha = s->rho / rv;
        break;
    }
    case FIN_BI_S: {
        const T ss = dots[0];
        s->iters += 1;
        if (ss <= s->tol2) {
            s->s_conv = 1;
            s->skip_t = 1;
            s->relres = sqrt(ss / s->bb);
        }
        break;
    }
    case FIN_BI_OMEGA: {
        const T ts = dots[0], tt = dots[1];
        if (tt == T(0)) kstop(s, SPX_BREAKDOWN);
        else s->omega = ts / tt;
        break;
    }
    case FIN_BI_R: {
        if (s->s_conv) { kstop(s, SPX_CONVERGED); break; }
        const T rr = dots[0], rhr = dots[1];
        s->relres = sqrt(rr / s->bb);
        if (rr <= s->tol2) { kstop(s, SPX_CONVERGED); break; }
        if (s->omega == T(0)) { kstop(s, SPX_BREAKDOWN); break; }
        if (s->iters >= s->maxit) { kstop(s, SPX_MAX_ITER); break; }
        if (rhr == T(0)) { kstop(s, SPX_BREAKDOWN); break; }
        s->beta = (rhr / s->rho) * (s->alpha / s->omega);
        s->rho = rhr;
        break;
    }
    case FIN_PCG_RHO0: {
        if (s->done) break;
        if (dots[0] == T(0)) kstop(s, SPX_BREAKDOWN);
        else s->rho = dots[0];
        break;
    }
    case FIN_PCG_R: {
        const T rr = dots[0], rz = dots[1];
        s->iters += 1;
        s->relres = sqrt(rr / s->bb);
        if (rr <= s->tol2) { kstop(s, SPX_CONVERGED); break; }
        if (s->iters >= s->maxit) { kstop(s, SPX_MAX_ITER); break; }
        if (rz == T(0)) { kstop(s, SPX_BREAKDOWN); break; }
        s->beta = rz / s->rho;
        s->rho = rz;
        break;
    }
    case FIN_CG_RR: {
        const T rr = dots[0];
        s->iters += 1;
        s->relres = sqrt(rr / s->bb);
        if (rr <= s->tol2) { kstop(s, SPX_CONVERGED); break; }
        if (s->iters >= s->maxit) { kstop(s, SPX_MAX_ITER); break; }
        break;
    }
    case FIN_PCG_RZ: {
        const T rz = dots[0];
        if (rz == T(0)) { kstop(s, SPX_BREAKDOWN); break; }
        s->beta = rz / s->rho;
        s->rho = rz;
        break;
    }
    case FIN_CGS_R: {
        const T rr = dots[0], rhr = dots[1];
        s->iters += 1;
        s->relres = sqrt(rr / s->bb);
        if (rr <= s->tol2) { kstop(s, SPX_CONVERGED); break; }
        if (s->iters >= s->maxit) { kstop(s, SPX_MAX_ITER); break; }
        if (s->stall > 0) {
            if (s->relres < T(0.5) * s->mark) {
                s->mark = s->relres;
                s->mark_it = s->iters;
            } else if (s->iters - s->mark_it >= s->stall) {
                kstop(s, SPX_STAGNATED);
                break;
            }
        }
        if (rhr == T(0)) { kstop(s, SPX_BREAKDOWN); break; }
        s->beta = rhr / s->rho;
        s->rho = rhr;
        break;
    }
    default: break;
    }
}

// Grid-wide finish of up to two dot products: block partials, then the last
// block to arrive sums them in block order (deterministic), stores dots[0..1]
// (if dots != null) and runs the scalar update.  Every block must call it.
template <class T, int BLOCK>
__device__ __forceinline__ void grid_dots_finish(T d0, T d1, T *dots, int fin, void *fst, T *partials,
                                                 unsigned *ticket)
{
    __shared__ T red[BLOCK / 32];
    const T b0 = block_sum<T, BLOCK>(d0, red);
    const T b1 = block_sum<T, BLOCK>(d1, red);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = b0;
        partials[2 * blockIdx.x + 1] = b1;
    }
    if (!last_block(ticket, gridDim.x)) return;
    T s0 = T(0), s1 = T(0);
    for (unsigned b = threadIdx.x; b < gridDim.x; b += BLOCK) {
        s0 += ldcg(partials + 2 * b);
        s1 += ldcg(partials + 2 * b + 1);
    }
    s0 = block_sum<T, BLOCK>(s0, red);
    s1 = block_sum<T, BLOCK>(s1, red);
    if (threadIdx.x == 0) {
        if (dots) {
            dots[0] = s0;
            dots[1] = s1;
        }
        const T dd[2] = {s0, s1};
        run_fin<T>(fin, fst, dd);
    }
}

}  // namespace spx
