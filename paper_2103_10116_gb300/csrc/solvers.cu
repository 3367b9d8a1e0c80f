// solvers.cu -- Krylov solvers on the device: CG, BiCGSTAB, CGS, restarted GMRES(m),
// and FP64 iterative refinement around an FP32 inner solve.
//
// The methods are the ones Section 5 of arXiv 2103.10116 names (CG for SPD
// systems; BiCGSTAB, CGS and GMRES for general ones; GMRES orthogonalises each new
// direction against all previous ones).  The GPU form differs from a textbook
// loop only in scheduling:
//   * every scalar (alpha, beta, omega, rho, norms, Hessenberg column) stays
//     on the device, updated by the last block of the kernel that reduces it;
//   * an iteration is a fixed sequence of fused kernels (SpMV with a dot
//     epilogue, vector update with a dot, direction update), each returning
//     at once once the solve has stopped, so the host enqueues a chunk of
//     iterations as one CUDA graph and reads the stop flag once per chunk;
//   * GMRES orthogonalises with classical Gram-Schmidt, repeated once when the
//     first pass cancels nearly all of the vector (selective reorthogonalisation),
//     which reads the Krylov basis in long coalesced streams instead of one
//     dependent dot product per basis vector (modified Gram-Schmidt).
// Convergence policy: recurrence residual ||r||/||b|| <= tol, then the true
// residual b - A x is formed; if it misses tol the solve restarts from x (at
// most 3 times, then STAGNATED).
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "dev_common.cuh"
#include "kstate.cuh"
#include "spx_internal.cuh"

namespace spx {

constexpr int kVB = 256;        // block of the vector kernels
constexpr int kGmKmax = 32;     // largest GMRES restart length (basis held in registers per row)
constexpr int kMaxRestarts = 3;
// When a solve replays its iterations as CUDA graphs: systems of at least
// kGraphMinRows rows, from their second solve on the same matrix (the first
// launches directly).  Mixed CG to 1e-8 on a 27 000-row 7-point stencil took
// 4.48 ms launched directly and 2.37 ms replaying graphs (BiCGSTAB on 30 000
// rows of 20 random columns: 2.02 against 1.18 ms); but a request server that
// solves every matrix once lost throughput capturing a graph per request
// (sixteen slots capturing at once: the solve phases of its 25 000 - 100 000-row
// requests summed to 206 s against 187 s).
constexpr int64_t kGraphMinRows = 8192;
bool graphs_for(const spx_matrix *A) { return A->n >= kGraphMinRows && A->solves > 0; }

// ------------------------------------------------------------------ GMRES state
template <class T> struct GState {
    T bnorm;     // ||b||
    T tol;       // relative tolerance
    T beta;      // ||r|| at the start of the cycle
    T relres;    // residual estimate |g_{j+1}| / ||b||, or the true one after a restart
    int done;    // solve finished
    int skip;    // Arnoldi kernels return at once (done or cycle stopped)
    int cyc_stop;
    int est_conv;  // last cycle stopped because the estimate met tol
    int jdone;     // Arnoldi steps completed in the current cycle
    int status;
    int restarts;  // cycles that ended on the estimate but failed the true residual
    int m;
    int reorth;    // the current Arnoldi step needs the second Gram-Schmidt pass
    long long iters, maxit;
};

// small per-solve arrays of GMRES (device): H[(m+1) x m] row-major, cs, sn, g, y, h1, h2
template <class T> struct GSmall {
    T *H, *cs, *sn, *g, *y, *h1, *h2;
};

// ------------------------------------------------------------------ workspace
struct SolverWork {
    int dtype = -1, solver = -1, m = 0;
    int64_t n = 0, ld = 0;
    int nvec = 0;
    DBuf vecs, state, dots, red, ticket, small;
    int red_grid = 0;
    void *host = nullptr;  // pinned copy of the state
    // CUDA graph of one chunk of iterations
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey[8] = {0};
    // mixed precision
    SolverWork *inner = nullptr;
    DBuf ir;  // r (FP64), r32, d32
    // Jacobi preconditioning: M^{-1} = 1 / diag(A) in the work's precision;
    // block-Jacobi (bs > 0, pre also set): inverses of the bs x bs diagonal
    // blocks, row-major per block
    bool pre = false;
    int bs = 0;
    bool bj_adapt = false;  // adaptive storage: FP32 copies of the blocks that qualify
    DBuf dinv, bjinv, bjinv32;
};

void solver_work_release(spx_ctx *ctx, SolverWork *w)
{
    if (!w) return;
    if (w->gexec) cudaGraphExecDestroy(w->gexec);
    DBuf *bufs[] = {&w->vecs, &w->state, &w->dots, &w->red, &w->ticket, &w->small, &w->ir, &w->dinv, &w->bjinv,
                    &w->bjinv32};
    for (DBuf *b : bufs) dbuf_free(ctx, *b);
    if (w->host) cudaFreeHost(w->host);
    solver_work_release(ctx, w->inner);
    delete w;
}

void solver_work_free(spx_matrix *A)
{
    if (A->work) {
        cudaStreamSynchronize(A->ctx->stream);
        solver_work_release(A->ctx, A->work);
    }
    A->work = nullptr;
}

static int nvec_for(int solver, int m, bool pre)
{
    if (solver == SPX_CG) return 4;                   // r, p, q, scratch (z = M^-1 r in q's place, or never stored)
    if (solver == SPX_BICGSTAB) return pre ? 9 : 7;   // r, rh, p, v, s, t, scratch (+ M^-1 p, M^-1 s)
    if (solver == SPX_CGS) return pre ? 9 : 8;        // r, rh, p, u, q, v, w, scratch (+ M^-1 p)
    return m + (pre ? 3 : 2);                         // V[0..m], scratch (+ M^-1 v_j)
}

template <class T>
static int work_prepare(spx_ctx *ctx, SolverWork *&wk, int64_t n, int solver, int m, bool pre = false, int bs = 0,
                        bool adapt = false)
{
    const int dtype = sizeof(T) == 8 ? SPX_F64 : SPX_F32;
    adapt = adapt && sizeof(T) == 8;  // FP32 solves store FP32 inverses anyway
    if (wk && (wk->dtype != dtype || wk->n != n || wk->solver != solver || wk->m != m || wk->pre != pre ||
               wk->bs != bs || wk->bj_adapt != adapt)) {
        SolverWork *inner = wk->inner;
        wk->inner = nullptr;
        cudaStreamSynchronize(ctx->stream);
        solver_work_release(ctx, wk);
        wk = nullptr;
        if (inner) {
            wk = new SolverWork();
            wk->inner = inner;
        }
    }
    if (!wk) wk = new SolverWork();
    if (wk->vecs.p) return SPX_OK;
    wk->dtype = dtype;
    wk->n = n;
    wk->solver = solver;
    wk->m = m;
    wk->pre = pre;
    wk->bs = bs;
    wk->bj_adapt = adapt;
    wk->ld = (int64_t)round_up((size_t)(n > 0 ? n : 1), 64);
    wk->nvec = nvec_for(solver, m, pre);
    SPX_TRY(dbuf_alloc(ctx, wk->vecs, (size_t)wk->nvec * wk->ld * sizeof(T)));
    SPX_TRY(dbuf_alloc(ctx, wk->state, 512));
    SPX_TRY(dbuf_alloc(ctx, wk->dots, 64));
    wk->red_grid = ctx->sm_count * 4;
    SPX_TRY(dbuf_alloc(ctx, wk->red, (size_t)wk->red_grid * (kGmKmax + 2) * 8));
    SPX_TRY(dbuf_alloc(ctx, wk->ticket, 64));
    SPX_CUDA(cudaMemsetAsync(wk->ticket.p, 0, 64, ctx->stream));
    SPX_TRY(dbuf_alloc(ctx, wk->small, (size_t)((m + 1) * m + 4 * (m + 2) + 2 * (kGmKmax + 2) + 16) * 8));
    if (!wk->host) SPX_CUDA(cudaMallocHost(&wk->host, 512));
    return SPX_OK;
}

// ------------------------------------------------------------------ fused vector kernels
// Each returns at once when *skip is set (by an earlier kernel), reduces its
// dots deterministically and lets the last block update the scalar state.
// Grid-stride loops over a fixed grid take kU elements per thread per step,
// all their loads issued before the arithmetic (kU * operands loads in
// flight), then a scalar tail.
constexpr int kU = 4;

#define SPX_ROWS_LOOP(LOAD, STORE)                                                   \
    {                                                                                \
        const int64_t stride_ = (int64_t)gridDim.x * kVB;                            \
        int64_t i0_ = blockIdx.x * (int64_t)kVB + threadIdx.x;                       \
        for (; i0_ + (kU - 1) * stride_ < n; i0_ += kU * stride_) {                  \
            _Pragma("unroll") for (int u = 0; u < kU; ++u) {                         \
                const int64_t i = i0_ + u * stride_;                                 \
                LOAD                                                                 \
            }                                                                        \
            _Pragma("unroll") for (int u = 0; u < kU; ++u) {                         \
                const int64_t i = i0_ + u * stride_;                                 \
                (void)i;                                                             \
                STORE                                                                \
            }                                                                        \
        }                                                                            \
        for (; i0_ < n; i0_ += stride_) {                                            \
            constexpr int u = 0;                                                     \
            const int64_t i = i0_;                                                   \
            LOAD                                                                     \
            STORE                                                                    \
        }                                                                            \
    }

template <class T>
__global__ void __launch_bounds__(kVB)
    k_dot_fin(int64_t n, const T *__restrict__ a, const T *__restrict__ b, int fin, KState<T> *st,
              T *partials, unsigned *ticket)
{
    T d0 = T(0);
    T av[kU], bv[kU];
    SPX_ROWS_LOOP(av[u] = a[i]; bv[u] = b[i];, d0 = fma(av[u], bv[u], d0);)
    grid_dots_finish<T, kVB>(d0, T(0), (T *)nullptr, fin, st, partials, ticket);
}

// CG: x += alpha p; r -= alpha q; rho' = r.r.  PRE 1 (Jacobi): also r.z with
// z = dinv r, for beta; PRE 2 (block-Jacobi): r.r for the convergence test
// only, r.z follows from the block apply.  Convergence is tested on r.r.
template <class T, int PRE>
__global__ void __launch_bounds__(kVB)
    k_cg_xr(int64_t n, T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p, const T *__restrict__ q,
            const T *__restrict__ dinv, KState<T> *st, T *partials, unsigned *ticket)
{
    if (st->done) return;
    const T alpha = st->alpha;
    T d0 = T(0), d1 = T(0);
    T xv[kU], rv[kU], pv[kU], qv[kU], dv[kU];
    SPX_ROWS_LOOP(xv[u] = x[i]; rv[u] = r[i]; pv[u] = p[i]; qv[u] = q[i]; if (PRE == 1) dv[u] = dinv[i];,
                  x[i] = fma(alpha, pv[u], xv[u]); const T ri = fma(-alpha, qv[u], rv[u]); r[i] = ri;
                  d0 = fma(ri, ri, d0); if (PRE == 1) d1 = fma(ri, dv[u] * ri, d1);)
    grid_dots_finish<T, kVB>(d0, d1, (T *)nullptr, PRE == 1 ? FIN_PCG_R : PRE == 2 ? FIN_CG_RR : FIN_CG_RHO, st,
                             partials, ticket);
}

// CG: p = r + beta p  (PRE: p = dinv r + beta p)
template <class T, bool PRE>
__global__ void __launch_bounds__(kVB)
    k_cg_p(int64_t n, const T *__restrict__ r, T *__restrict__ p, const T *__restrict__ dinv, const KState<T> *st)
{
    if (st->done) return;
    const T beta = st->beta;
    T rv[kU], pv[kU], dv[kU];
    SPX_ROWS_LOOP(rv[u] = r[i]; pv[u] = p[i]; if (PRE) dv[u] = dinv[i];,
                  p[i] = fma(beta, pv[u], PRE ? dv[u] * rv[u] : rv[u]);)
}

// Preconditioned CG start: p = z = dinv r; rho = r.z
template <class T>
__global__ void __launch_bounds__(kVB)
    k_pcg_init(int64_t n, const T *__restrict__ r, T *__restrict__ p, const T *__restrict__ dinv, KState<T> *st,
               T *partials, unsigned *ticket)
{
    if (st->done) return;
    T d0 = T(0);
    T rv[kU], dv[kU];
    SPX_ROWS_LOOP(rv[u] = r[i]; dv[u] = dinv[i];, const T zi = dv[u] * rv[u]; p[i] = zi; d0 = fma(rv[u], zi, d0);)
    grid_dots_finish<T, kVB>(d0, T(0), (T *)nullptr, FIN_PCG_RHO0, st, partials, ticket);
}

// out = dinv in (M^-1 applied to a vector)
template <class T>
__global__ void __launch_bounds__(kVB)
    k_jscale(int64_t n, const T *__restrict__ in, const T *__restrict__ dinv, T *__restrict__ out, const KState<T> *st)
{
    if (st && st->done) return;
    T iv[kU], dv[kU];
    SPX_ROWS_LOOP(iv[u] = in[i]; dv[u] = dinv[i];, out[i] = dv[u] * iv[u];)
}

// BiCGSTAB: p = r + beta (p - omega v)  (PRE: also ph = dinv p)
template <class T, bool PRE>
__global__ void __launch_bounds__(kVB)
    k_bi_p(int64_t n, const T *__restrict__ r, T *__restrict__ p, const T *__restrict__ v, T *__restrict__ ph,
           const T *__restrict__ dinv, const KState<T> *st)
{
    if (st->done) return;
    const T beta = st->beta, omega = st->omega;
    T rv[kU], pv[kU], vv[kU], dv[kU];
    SPX_ROWS_LOOP(rv[u] = r[i]; pv[u] = p[i]; vv[u] = v[i]; if (PRE) dv[u] = dinv[i];,
                  const T pi = fma(beta, fma(-omega, vv[u], pv[u]), rv[u]); p[i] = pi; if (PRE) ph[i] = dv[u] * pi;)
}

// BiCGSTAB: s = r - alpha v; s.s  (PRE: also sh = dinv s)
template <class T, bool PRE>
__global__ void __launch_bounds__(kVB)
    k_bi_s(int64_t n, const T *__restrict__ r, const T *__restrict__ v, T *__restrict__ s, T *__restrict__ sh,
           const T *__restrict__ dinv, KState<T> *st, T *partials, unsigned *ticket)
{
    if (st->done) return;
    const T alpha = st->alpha;
    T d0 = T(0);
    T rv[kU], vv[kU], dv[kU];
    SPX_ROWS_LOOP(rv[u] = r[i]; vv[u] = v[i]; if (PRE) dv[u] = dinv[i];,
                  const T si = fma(-alpha, vv[u], rv[u]); s[i] = si; if (PRE) sh[i] = dv[u] * si;
                  d0 = fma(si, si, d0);)
    grid_dots_finish<T, kVB>(d0, T(0), (T *)nullptr, FIN_BI_S, st, partials, ticket);
}

// BiCGSTAB: x += alpha p + omega s; r = s - omega t  (or, converged on s:
// x += alpha p; r = s); dots r.r and r^.r.  Right preconditioning: the x
// update takes M^-1 p and M^-1 s (pp, ss point at those or at p, s).
template <class T>
__global__ void __launch_bounds__(kVB)
    k_bi_xr(int64_t n, T *__restrict__ x, T *__restrict__ r, const T *__restrict__ rh, const T *__restrict__ pp,
            const T *__restrict__ s, const T *__restrict__ ss, const T *__restrict__ t, KState<T> *st, T *partials,
            unsigned *ticket)
{
    if (st->done) return;
    const T alpha = st->alpha, omega = st->omega;
    const bool sconv = st->s_conv != 0;
    T d0 = T(0), d1 = T(0);
    T xv[kU], pv[kU], sv[kU], qv[kU], tv[kU], hv[kU];
    if (sconv) {
        SPX_ROWS_LOOP(xv[u] = x[i]; pv[u] = pp[i]; sv[u] = s[i]; hv[u] = rh[i];,
                      x[i] = fma(alpha, pv[u], xv[u]); const T ri = sv[u]; r[i] = ri; d0 = fma(ri, ri, d0);
                      d1 = fma(hv[u], ri, d1);)
    } else {
        SPX_ROWS_LOOP(xv[u] = x[i]; pv[u] = pp[i]; sv[u] = s[i]; qv[u] = ss[i]; tv[u] = t[i]; hv[u] = rh[i];,
                      x[i] = fma(omega, qv[u], fma(alpha, pv[u], xv[u])); const T ri = fma(-omega, tv[u], sv[u]);
                      r[i] = ri; d0 = fma(ri, ri, d0); d1 = fma(hv[u], ri, d1);)
    }
    grid_dots_finish<T, kVB>(d0, d1, (T *)nullptr, FIN_BI_R, st, partials, ticket);
}

// CGS: q = u - alpha v; w = u + q (PRE 1: w = dinv (u + q)); x += alpha w.
// PRE 2 (block-Jacobi): q and w = u + q only; the block apply forms
// M^-1 (u + q) and updates x.
template <class T, int PRE>
__global__ void __launch_bounds__(kVB)
    k_cgs_qw(int64_t n, T *__restrict__ x, const T *__restrict__ uu, const T *__restrict__ v, T *__restrict__ q,
             T *__restrict__ w, const T *__restrict__ dinv, const KState<T> *st)
{
    if (st->done) return;
    const T alpha = st->alpha;
    T xv[kU], uv[kU], vv[kU], dv[kU];
    SPX_ROWS_LOOP(if (PRE != 2) xv[u] = x[i]; uv[u] = uu[i]; vv[u] = v[i]; if (PRE == 1) dv[u] = dinv[i];,
                  const T qi = fma(-alpha, vv[u], uv[u]); q[i] = qi;
                  const T wi = PRE == 1 ? dv[u] * (uv[u] + qi) : uv[u] + qi; w[i] = wi;
                  if (PRE != 2) x[i] = fma(alpha, wi, xv[u]);)
}

// CGS: r -= alpha v (v = A w); dots r.r and r^.r
template <class T>
__global__ void __launch_bounds__(kVB)
    k_cgs_r(int64_t n, T *__restrict__ r, const T *__restrict__ rh, const T *__restrict__ v, KState<T> *st,
            T *partials, unsigned *ticket)
{
    if (st->done) return;
    const T alpha = st->alpha;
    T d0 = T(0), d1 = T(0);
    T rv[kU], hv[kU], vv[kU];
    SPX_ROWS_LOOP(rv[u] = r[i]; hv[u] = rh[i]; vv[u] = v[i];,
                  const T ri = fma(-alpha, vv[u], rv[u]); r[i] = ri; d0 = fma(ri, ri, d0); d1 = fma(hv[u], ri, d1);)
    grid_dots_finish<T, kVB>(d0, d1, (T *)nullptr, FIN_CGS_R, st, partials, ticket);
}

// CGS: u = r + beta q; p = u + beta (q + beta p)  (PRE: also ph = dinv p)
template <class T, bool PRE>
__global__ void __launch_bounds__(kVB)
    k_cgs_up(int64_t n, const T *__restrict__ r, const T *__restrict__ q, T *__restrict__ uu, T *__restrict__ p,
             T *__restrict__ ph, const T *__restrict__ dinv, const KState<T> *st)
{
    if (st->done) return;
    const T beta = st->beta;
    T rv[kU], qv[kU], pv[kU], dv[kU];
    SPX_ROWS_LOOP(rv[u] = r[i]; qv[u] = q[i]; pv[u] = p[i]; if (PRE) dv[u] = dinv[i];,
                  const T ui = fma(beta, qv[u], rv[u]); uu[i] = ui; const T pi = fma(beta, fma(beta, pv[u], qv[u]), ui);
                  p[i] = pi; if (PRE) ph[i] = dv[u] * pi;)
}

// the inverse diagonal, 1 / sum of the diagonal entries of row i in CSR order
// (1 where that sum is 0), from whichever storage the matrix holds: CSR
// arrays, or the ELL slots and then the COO entries of the row (HYB, COO)
template <class V, class T>
__global__ void k_jacobi_dinv(int64_t n, const int *__restrict__ rp, const int *__restrict__ col,
                              const V *__restrict__ val, int64_t ell_ld, int64_t ell_w, const int *__restrict__ ecol,
                              const V *__restrict__ evals, int64_t coo_nnz, const int *__restrict__ crow,
                              const int *__restrict__ ccol, const V *__restrict__ cval, T *__restrict__ dinv)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        if (rp)
            for (int k = rp[i]; k < rp[i + 1]; ++k)
                if (col[k] == i) d += (double)val[k];
        for (int64_t j = 0; j < ell_w; ++j)
            if (ecol[j * ell_ld + i] == i) d += (double)evals[j * ell_ld + i];
        if (coo_nnz > 0) {  // first entry of row i: rows are sorted
            int64_t lo = 0, hi = coo_nnz;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (crow[mid] < i) lo = mid + 1;
                else hi = mid;
            }
            for (int64_t k = lo; k < coo_nnz && crow[k] == i; ++k)
                if (ccol[k] == i) d += (double)cval[k];
        }
        dinv[i] = d != 0.0 ? (T)(1.0 / d) : T(1);
    }
}

// ------------------------------------------------------------------ block-Jacobi
// M = the block diagonal of A, blocks of bs consecutive rows and columns
// (bs a power of two up to 32, so a block never straddles a warp); the last
// block is padded with identity rows.  Section 2 lists block-Jacobi among the
// library's preconditioners.
constexpr int kBjWarps = 2;  // warps per block of the inversion kernel
// Adaptive storage (the adaptive-precision block-Jacobi Section 2 cites, with
// this rule read into it): a block's inverse is applied from an FP32 copy when
// its 1-norm condition number times the FP32 unit roundoff is at most this,
// so that the rounded inverse stays within 1% of the identity in the
// preconditioned block; else from the FP64 inverse.
constexpr double kBjFp32Bound = 1e-2;

__device__ __forceinline__ double bj_warp_max(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// One warp per diagonal block: gather the block's entries (the block's rows,
// columns inside the block; duplicates summed in storage order) into the
// augmented matrix [D | I] (bs x 2bs, FP64, shared memory), then Gauss-Jordan
// with partial pivoting: pick the largest |entry| at or below the diagonal of
// the pivot column (the first one on ties), swap, scale the pivot row by the
// reciprocal of the pivot, subtract multiples of it from the other rows.  A
// block with an exactly zero pivot is stored as the identity (Jacobi's rule
// for a zero diagonal).  Lanes own rows while gathering, columns while
// eliminating.
template <class V, class T>
__global__ void __launch_bounds__(32 * kBjWarps)
    k_bj_build(int64_t n, int bs, const int *__restrict__ rp, const int *__restrict__ col, const V *__restrict__ val,
               int64_t ell_ld, int64_t ell_w, const int *__restrict__ ecol, const V *__restrict__ evals,
               int64_t coo_nnz, const int *__restrict__ crow, const int *__restrict__ ccol,
               const V *__restrict__ cval, T *__restrict__ minv, float *__restrict__ minv32)
{
    extern __shared__ double bj_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int w2 = 2 * bs;
    double *aug = bj_smem + (size_t)wib * (size_t)(bs * w2 + bs);
    double *fcol = aug + bs * w2;  // the pivot column, read before the rows change
    const int64_t nb = (n + bs - 1) / bs;
    for (int64_t k = (int64_t)blockIdx.x * kBjWarps + wib; k < nb; k += (int64_t)gridDim.x * kBjWarps) {
        const int64_t c0 = k * bs;
        for (int e = lane; e < bs * w2; e += 32) aug[e] = 0.0;
        __syncwarp();
        if (lane < bs) {
            const int r = lane;
            const int64_t i = c0 + r;
            double *row = aug + r * w2;
            row[bs + r] = 1.0;
            if (i >= n) {
                row[r] = 1.0;
            } else {
                if (rp)
                    for (int e = rp[i]; e < rp[i + 1]; ++e) {
                        const int64_t c = col[e];
                        if (c >= c0 && c < c0 + bs) row[c - c0] += (double)val[e];
                    }
                for (int64_t j = 0; j < ell_w; ++j) {
                    const int64_t c = ecol[j * ell_ld + i];
                    if (c >= c0 && c < c0 + bs) row[c - c0] += (double)evals[j * ell_ld + i];
                }
                if (coo_nnz > 0) {  // the row's entries: rows are sorted
                    int64_t lo = 0, hi = coo_nnz;
                    while (lo < hi) {
                        const int64_t mid = (lo + hi) >> 1;
                        if (crow[mid] < i) lo = mid + 1;
                        else hi = mid;
                    }
                    for (int64_t e = lo; e < coo_nnz && crow[e] == i; ++e) {
                        const int64_t c = ccol[e];
                        if (c >= c0 && c < c0 + bs) row[c - c0] += (double)cval[e];
                    }
                }
            }
        }
        __syncwarp();
        // ||D||_1 (adaptive storage): column sums in row order, then the largest
        double dnorm = 0.0;
        if (minv32) {
            double cs = 0.0;
            if (lane < bs)
                for (int r = 0; r < bs; ++r) cs += fabs(aug[r * w2 + lane]);
            dnorm = bj_warp_max(cs);
        }
        bool singular = false;
        for (int p = 0; p < bs; ++p) {
            double best = -1.0;
            int piv = p;
            if (lane >= p && lane < bs) {
                best = fabs(aug[lane * w2 + p]);
                piv = lane;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, off);
                const int op = __shfl_down_sync(0xffffffffu, piv, off);
                if (ob > best || (ob == best && op < piv)) {
                    best = ob;
                    piv = op;
                }
            }
            best = __shfl_sync(0xffffffffu, best, 0);
            piv = __shfl_sync(0xffffffffu, piv, 0);
            if (best == 0.0) {  // warp-uniform
                singular = true;
                break;
            }
            if (piv != p) {
                for (int c = lane; c < w2; c += 32) {
                    const double t = aug[p * w2 + c];
                    aug[p * w2 + c] = aug[piv * w2 + c];
                    aug[piv * w2 + c] = t;
                }
                __syncwarp();
            }
            const double inv = 1.0 / aug[p * w2 + p];
            __syncwarp();
            for (int c = lane; c < w2; c += 32) aug[p * w2 + c] *= inv;
            if (lane < bs) fcol[lane] = aug[lane * w2 + p];
            __syncwarp();
            for (int c = lane; c < w2; c += 32) {
                const double pc = aug[p * w2 + c];
                for (int r = 0; r < bs; ++r) {
                    const double f = fcol[r];
                    if (r != p && f != 0.0) aug[r * w2 + c] -= f * pc;
                }
            }
            __syncwarp();
        }
        T *out = minv + (size_t)k * (size_t)(bs * bs);
        for (int e = lane; e < bs * bs; e += 32) {
            const int r = e / bs, c = e - r * bs;
            out[e] = singular ? (r == c ? T(1) : T(0)) : (T)aug[r * w2 + bs + c];
        }
        if (minv32) {
            // FP32 copy when kappa_1 * 2^-24 <= kBjFp32Bound and every nonzero
            // entry is inside FP32's normal range; else every row of the copy
            // starts with a NaN, which sends the apply to the FP64 inverse
            double cs = 0.0, amax = 0.0, amin = INFINITY;
            if (lane < bs)
                for (int r = 0; r < bs; ++r) {
                    const double v = fabs(singular ? (r == lane ? 1.0 : 0.0) : aug[r * w2 + bs + lane]);
                    cs += v;
                    amax = fmax(amax, v);
                    if (v != 0.0) amin = fmin(amin, v);
                }
            const double inorm = bj_warp_max(cs);
            amax = bj_warp_max(amax);
            amin = -bj_warp_max(-amin);
            const bool in_range = amax <= (double)FLT_MAX && (amin == INFINITY || amin >= (double)FLT_MIN);
            const bool fp64 = !singular && (dnorm * inorm * 0x1p-24 > kBjFp32Bound || !in_range);
            float *o32 = minv32 + (size_t)k * (size_t)(bs * bs);
            for (int e = lane; e < bs * bs; e += 32) {
                const int r = e / bs, c = e - r * bs;
                o32[e] = fp64 ? (c == 0 ? __int_as_float(0x7fc00000) : 0.0f)
                              : (singular ? (r == c ? 1.0f : 0.0f) : (float)aug[r * w2 + bs + c]);
            }
        }
        __syncwarp();
    }
}

// Small blocks (bs <= 8): one thread per diagonal block, so that each FP64
// warp instruction works on 32 blocks (GB300 issues two FP64 lanes per SM
// per clock; a warp per 8 x 8 block left most of every instruction idle).
// The block sits in shared memory interleaved across the threads (element
// e of thread t at e * kBjTpb + t: no bank conflicts) and is inverted in
// place by Gauss-Jordan with partial pivoting (the same pivot choice and
// zero-pivot rule as the warp kernel; the row swaps are undone on the
// columns at the end).
constexpr int kBjTpb = 64;

template <class V, class T, int BS>
__global__ void __launch_bounds__(kBjTpb)
    k_bj_build_t(int64_t n, const int *__restrict__ rp, const int *__restrict__ col, const V *__restrict__ val,
                 int64_t ell_ld, int64_t ell_w, const int *__restrict__ ecol, const V *__restrict__ evals,
                 int64_t coo_nnz, const int *__restrict__ crow, const int *__restrict__ ccol,
                 const V *__restrict__ cval, T *__restrict__ minv, float *__restrict__ minv32)
{
    __shared__ double sa[BS * BS * kBjTpb];
    const int t = threadIdx.x;
    const int64_t nb = (n + BS - 1) / BS;
#define BJA(r_, c_) sa[((r_) * BS + (c_)) * kBjTpb + t]
    for (int64_t k = (int64_t)blockIdx.x * kBjTpb + t; k - t < nb; k += (int64_t)gridDim.x * kBjTpb) {
        if (k >= nb) continue;
        const int64_t c0 = k * BS;
#pragma unroll
        for (int e = 0; e < BS * BS; ++e) sa[e * kBjTpb + t] = 0.0;
        for (int r = 0; r < BS; ++r) {
            const int64_t i = c0 + r;
            if (i >= n) {
                BJA(r, r) = 1.0;
                continue;
            }
            if (rp)
                for (int e = rp[i]; e < rp[i + 1]; ++e) {
                    const int64_t c = col[e];
                    if (c >= c0 && c < c0 + BS) BJA(r, c - c0) += (double)val[e];
                }
            for (int64_t j = 0; j < ell_w; ++j) {
                const int64_t c = ecol[j * ell_ld + i];
                if (c >= c0 && c < c0 + BS) BJA(r, c - c0) += (double)evals[j * ell_ld + i];
            }
            if (coo_nnz > 0) {
                int64_t lo = 0, hi = coo_nnz;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (crow[mid] < i) lo = mid + 1;
                    else hi = mid;
                }
                for (int64_t e = lo; e < coo_nnz && crow[e] == i; ++e) {
                    const int64_t c = ccol[e];
                    if (c >= c0 && c < c0 + BS) BJA(r, c - c0) += (double)cval[e];
                }
            }
        }
        double dnorm = 0.0;
        if (minv32)
            for (int c = 0; c < BS; ++c) {
                double cs = 0.0;
                for (int r = 0; r < BS; ++r) cs += fabs(BJA(r, c));
                dnorm = fmax(dnorm, cs);
            }
        int perm[BS];
        bool singular = false;
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            int piv = p;
            double best = fabs(BJA(p, p));
            for (int r = p + 1; r < BS; ++r) {
                const double a = fabs(BJA(r, p));
                if (a > best) {
                    best = a;
                    piv = r;
                }
            }
            perm[p] = piv;
            if (best == 0.0) {
                singular = true;
                break;
            }
            if (piv != p)
                for (int c = 0; c < BS; ++c) {
                    const double tmp = BJA(p, c);
                    BJA(p, c) = BJA(piv, c);
                    BJA(piv, c) = tmp;
                }
            const double inv = 1.0 / BJA(p, p);
            BJA(p, p) = 1.0;
            for (int c = 0; c < BS; ++c) BJA(p, c) *= inv;
            for (int r = 0; r < BS; ++r) {
                if (r == p) continue;
                const double f = BJA(r, p);
                if (f == 0.0) continue;
                BJA(r, p) = 0.0;
                for (int c = 0; c < BS; ++c) BJA(r, c) -= f * BJA(p, c);
            }
        }
        if (!singular)
#pragma unroll
            for (int p = BS - 1; p >= 0; --p)
                if (perm[p] != p)
                    for (int r = 0; r < BS; ++r) {
                        const double tmp = BJA(r, p);
                        BJA(r, p) = BJA(r, perm[p]);
                        BJA(r, perm[p]) = tmp;
                    }
        T *out = minv + (size_t)k * (BS * BS);
        for (int r = 0; r < BS; ++r)
            for (int c = 0; c < BS; ++c) out[r * BS + c] = singular ? (r == c ? T(1) : T(0)) : (T)BJA(r, c);
        if (minv32) {
            double inorm = 0.0, amax = 0.0, amin = INFINITY;
            for (int c = 0; c < BS; ++c) {
                double cs = 0.0;
                for (int r = 0; r < BS; ++r) {
                    const double v = fabs(singular ? (r == c ? 1.0 : 0.0) : BJA(r, c));
                    cs += v;
                    amax = fmax(amax, v);
                    if (v != 0.0) amin = fmin(amin, v);
                }
                inorm = fmax(inorm, cs);
            }
            const bool in_range = amax <= (double)FLT_MAX && (amin == INFINITY || amin >= (double)FLT_MIN);
            const bool fp64 = !singular && (dnorm * inorm * 0x1p-24 > kBjFp32Bound || !in_range);
            float *o32 = minv32 + (size_t)k * (BS * BS);
            for (int r = 0; r < BS; ++r)
                for (int c = 0; c < BS; ++c)
                    o32[r * BS + c] = fp64 ? (c == 0 ? __int_as_float(0x7fc00000) : 0.0f)
                                           : (singular ? (r == c ? 1.0f : 0.0f) : (float)BJA(r, c));
        }
    }
#undef BJA
}

// out = M^-1 in, one element per thread: the lanes of a warp hold 32
// consecutive elements, so a block's inputs are exchanged with shuffles
// inside a group of BS lanes and each lane forms its row of the block times
// them (column order).  Modes: BJ_PLAIN; BJ_DOT also reduces in.out (r.z
// with in = r) and runs `fin`; BJ_AXPY also does x += alpha out (CGS, alpha
// from the state); BJ_ADDX does x += M^-1 in and stores nothing (GMRES's
// cycle update).  Returns at once while *skip is set.
enum { BJ_PLAIN = 0, BJ_DOT = 1, BJ_AXPY = 2, BJ_ADDX = 3 };

template <class T, int BS> __device__ __forceinline__ void bj_load_row(const T *__restrict__ row, T (&m)[BS])
{
    if constexpr (sizeof(T) == 8 && BS >= 2) {
#pragma unroll
        for (int j = 0; j < BS; j += 2) {
            const double2 t = __ldg(reinterpret_cast<const double2 *>(row + j));
            m[j] = t.x;
            m[j + 1] = t.y;
        }
    } else if constexpr (sizeof(T) == 4 && BS >= 4) {
#pragma unroll
        for (int j = 0; j < BS; j += 4) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(row + j));
            m[j] = t.x;
            m[j + 1] = t.y;
            m[j + 2] = t.z;
            m[j + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < BS; ++j) m[j] = __ldg(row + j);
    }
}

// FP32 -> FP64 widening of a zero, normal, infinite or NaN number (IEEE 754
// binary32 to binary64: same sign, exponent rebiased by 1023 - 127 or kept
// all-ones, fraction shifted up by 29 bits), on the integer units: a
// float-to-double conversion instruction runs on GB300's FP64 pipe, which the
// block apply's FMAs already fill.  The adaptive storage rule keeps every
// nonzero FP32 entry normal, and the NaN marker of an FP64 block stays a NaN.
__device__ __forceinline__ double bj_widen(unsigned b)
{
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    const unsigned mag = b & 0x7fffffffu;
    const unsigned e = mag >> 23;
    const unsigned long long ex = e == 0xffu ? 0x7ffull : (unsigned long long)(e + (1023u - 127u));
    const unsigned long long body = (ex << 52) | ((unsigned long long)(mag & 0x7fffffu) << 29);
    return __longlong_as_double((long long)(sign | (mag ? body : 0ull)));
}

template <int BS> __device__ __forceinline__ void bj_load_row32(const float *__restrict__ row, double (&m)[BS])
{
    if constexpr (BS >= 4) {
#pragma unroll
        for (int j = 0; j < BS; j += 4) {
            const uint4 t = __ldg(reinterpret_cast<const uint4 *>(row + j));
            m[j] = bj_widen(t.x);
            m[j + 1] = bj_widen(t.y);
            m[j + 2] = bj_widen(t.z);
            m[j + 3] = bj_widen(t.w);
        }
    } else if constexpr (BS == 2) {
        const uint2 t = __ldg(reinterpret_cast<const uint2 *>(row));
        m[0] = bj_widen(t.x);
        m[1] = bj_widen(t.y);
    } else {
        m[0] = bj_widen(__ldg(reinterpret_cast<const unsigned *>(row)));
    }
}

// ADAPT (FP64 solves with adaptive storage): each row comes from the FP32
// copy unless that row starts with the NaN marker of an FP64 block; the
// arithmetic stays FP64.  Each thread takes U elements per step (warp-uniform
// bounds; all loads before the shuffles) so that U rows are in flight.
template <class T, int BS, int MODE, bool ADAPT>
__global__ void __launch_bounds__(kVB)
    k_bj_apply(int64_t n, const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ minv,
               const float *__restrict__ minv32, const int *skip, T *__restrict__ x, KState<T> *st, int fin,
               T *partials, unsigned *ticket)
{
    if (skip && *skip) return;
    constexpr int U = BS >= 16 ? 1 : BS == 8 ? 2 : 4;  // at most 16 row values in registers
    const int lane = threadIdx.x & 31;
    const int g0 = lane & ~(BS - 1);
    const T alpha = MODE == BJ_AXPY ? st->alpha : T(0);
    T d0 = T(0);
    const int64_t stride = (int64_t)gridDim.x * kVB;
    for (int64_t base = (int64_t)blockIdx.x * kVB + (threadIdx.x & ~31); base < n; base += U * stride) {
        T v[U], m[U][BS];
        bool act[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + u * stride + lane;
            act[u] = i < n;
            v[u] = act[u] ? in[i] : T(0);
        }
        // every row load of the step is issued before the first use; the FP64
        // rows of an adaptive matrix follow only where the marker asks for them
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + u * stride + lane;
            if (!act[u]) continue;
            if constexpr (ADAPT) bj_load_row32<BS>(minv32 + i * BS, m[u]);
            else if constexpr (BS == 1) m[u][0] = minv[i];
            else bj_load_row<T, BS>(minv + i * BS, m[u]);
        }
        if constexpr (ADAPT) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = base + u * stride + lane;
                if (act[u] && isnan(m[u][0])) bj_load_row<T, BS>(minv + i * BS, m[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + u * stride + lane;
            T s = T(0);
            if constexpr (BS == 1 && !ADAPT) {
                if (act[u]) s = m[u][0] * v[u];
            } else {
#pragma unroll
                for (int j = 0; j < BS; ++j) {
                    const T vj = __shfl_sync(0xffffffffu, v[u], g0 + j);
                    if (act[u]) s = fma(m[u][j], vj, s);
                }
            }
            if (act[u]) {
                if (MODE == BJ_DOT) d0 = fma(v[u], s, d0);
                if (MODE != BJ_ADDX) out[i] = s;
                if (MODE == BJ_AXPY) x[i] = fma(alpha, s, x[i]);
                if (MODE == BJ_ADDX) x[i] += s;
            }
        }
    }
    if constexpr (MODE == BJ_DOT) grid_dots_finish<T, kVB>(d0, T(0), (T *)nullptr, fin, st, partials, ticket);
}

// ------------------------------------------------------------------ GMRES kernels
// Basis V[k] = base + k*ld, k = 0..m.  The Arnoldi step j forms w = A v_j in
// V[j+1] (with ||w||^2 from the SpMV epilogue), then classical Gram-Schmidt
// with selective reorthogonalisation: h1 = V_j^T w; w -= V_j h1; and only if
// that pass cancelled nearly all of w (||w_new|| < ||w_old|| / 8) a second
// pass h2 = V_j^T w; w -= V_j h2.  h = h1 + h2; H(j+1, j) = ||w||;
// v_{j+1} = w / ||w||.  One pass leaves w_new orthogonal to V_j up to about
// eps ||w_old|| / ||w_new||, so the threshold bounds that loss at 8 eps per
// step.  (The classic criterion of Daniel, Gragg, Kaufman and Stewart, 1976,
// reorthogonalises below 1/sqrt 2: on diagonally dominant matrices such as the
// upwind convection-diffusion operator, A v_j is mostly v_j and one pass keeps
// 26-42% of the norm, so that criterion asks for the second pass at every step,
// doubling the FP64 work of the orthogonalisation for an orthogonality gain
// from about 4 eps to eps.)
constexpr double kGmReorthKeep2 = 1.0 / 64.0;  // (||w_new|| / ||w_old||)^2 below which the second pass runs

// Gram-Schmidt kernels.  Rows are processed in chunks of kGmRows (grid-stride
// over a fixed grid).  Dots: the chunk of w sits in shared memory; warp wp
// owns basis vectors k = wp, wp+8, wp+16, wp+24 and each lane takes four
// rows at a time, so up to 16 independent loads per lane are in flight.
// Block partials [k][block] are summed by the last block in block order
// (deterministic).  Updates: a thread owns rows, two basis vectors per step.
constexpr int kGmRows = 1024;

// acc[q] += sum over the chunk's rows of V[wp + 8q][r0 + i] * ws[i]
template <class T>
__device__ __forceinline__ void gm_chunk_dots(const T *__restrict__ V, int64_t ld, int64_t r0, int nr, const T *ws,
                                              int j, int lane, int wp, T acc[4])
{
    if constexpr (sizeof(T) == 8) {
        // FP64: one owned vector at a time (four loads in flight), so no FP64
        // instruction is issued for a vector the warp does not own
        for (int i0 = lane; i0 < nr; i0 += 128) {
            T wi[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) wi[u] = i0 + 32 * u < nr ? ws[i0 + 32 * u] : T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = wp + 8 * q;
                if (k > j) break;  // warp-uniform
                const T *vk = V + (int64_t)k * ld + r0;
                T v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = i0 + 32 * u < nr ? vk[i0 + 32 * u] : T(0);
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[q] = fma(v[u], wi[u], acc[q]);
            }
        }
        return;
    }
    // FP32: every owned vector's rows are loaded before any FMA (up to 16 loads in flight)
    const int nq = wp > j ? 0 : min(4, (j - wp) / 8 + 1);  // vectors this warp owns (warp-uniform)
    if (nq == 0) return;
    for (int i0 = lane; i0 < nr; i0 += 128) {
        T wi[4], v[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) wi[u] = i0 + 32 * u < nr ? ws[i0 + 32 * u] : T(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T *vk = V + (int64_t)(wp + 8 * q) * ld + r0;
#pragma unroll
            for (int u = 0; u < 4; ++u) v[q][u] = q < nq && i0 + 32 * u < nr ? vk[i0 + 32 * u] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < nq) {  // warp-uniform
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[q] = fma(v[q][u], wi[u], acc[q]);
            }
    }
}

// The last block of a dots pass: hout[k] = sum of the block partials of k.
template <class T>
__device__ __forceinline__ void gm_store_dots(const T acc[4], int j, int lane, int wp, T *partials, T *hout,
                                              unsigned *ticket, bool &last)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = wp + 8 * q;
        const T s = warp_sum(acc[q]);
        if (lane == 0 && k <= j) partials[(int64_t)k * gridDim.x + blockIdx.x] = s;
    }
    last = last_block(ticket, gridDim.x);
    if (!last) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = wp + 8 * q;
        if (k > j) continue;
        T s = T(0);
        for (unsigned b = lane; b < gridDim.x; b += 32) s += ldcg(partials + (int64_t)k * gridDim.x + b);
        s = warp_sum(s);
        if (lane == 0) hout[k] = s;
    }
}

// w_i -= sum_{k<=j} hs[k] V[k][i] for R rows i = i0 + stride * u (those with
// ok[u]); two basis vectors per step, so 2R loads are in flight together.
template <class T, int R>
__device__ __forceinline__ void gm_rows_update(const T *__restrict__ V, int64_t ld, int64_t i0, int64_t stride,
                                               const bool ok[R], int jn, const T *hs, T wr[R])
{
    int k = 0;
    for (; k + 2 <= jn; k += 2) {
        const T *v0 = V + (int64_t)k * ld + i0, *v1 = v0 + ld;
        T a[R], c[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            a[u] = ok[u] ? v0[stride * u] : T(0);
            c[u] = ok[u] ? v1[stride * u] : T(0);
        }
        const T h0 = hs[k], h1 = hs[k + 1];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            wr[u] = fma(-h0, a[u], wr[u]);
            wr[u] = fma(-h1, c[u], wr[u]);
        }
    }
    if (k < jn) {
        const T *v0 = V + (int64_t)k * ld + i0;
        T a[R];
#pragma unroll
        for (int u = 0; u < R; ++u) a[u] = ok[u] ? v0[stride * u] : T(0);
#pragma unroll
        for (int u = 0; u < R; ++u) wr[u] = fma(-hs[k], a[u], wr[u]);
    }
}

// A dots pass: h = V_j^T w.  The first pass always runs (h1); the second
// (h2, second = true) only when the first update asked for it.
template <class T>
__global__ void __launch_bounds__(kVB)
    k_gm_dots(int64_t n, int64_t ld, const T *__restrict__ V, int j, const GState<T> *gs, T *hout, T *partials,
              unsigned *ticket, bool second)
{
    if (gs->skip || (second && !gs->reorth)) return;
    const T *w = V + (int64_t)(j + 1) * ld;
    __shared__ T ws[kGmRows];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int64_t r0 = (int64_t)blockIdx.x * kGmRows; r0 < n; r0 += (int64_t)gridDim.x * kGmRows) {
        const int nr = (int)min((int64_t)kGmRows, n - r0);
        __syncthreads();
        for (int i = threadIdx.x; i < nr; i += kVB) ws[i] = w[r0 + i];
        __syncthreads();
        gm_chunk_dots<T>(V, ld, r0, nr, ws, j, lane, wp, acc);
    }
    bool last;
    gm_store_dots<T>(acc, j, lane, wp, partials, hout, ticket, last);
}

// Column j of the Hessenberg matrix from h1 + h2 and ||w|| = sqrt(ww): the
// earlier Givens rotations, a new rotation, the residual estimate and the
// stopping decision (one thread).
template <class T> __device__ void gm_finish_column(GState<T> *gs, GSmall<T> sm, int j, T ww)
{
    const int m = gs->m;
    T *H = sm.H;
    const T hn = sqrt(ww);
    for (int k = 0; k <= j; ++k) H[k * m + j] = ldcg(sm.h1 + k) + ldcg(sm.h2 + k);
    H[(j + 1) * m + j] = hn;
    for (int k = 0; k < j; ++k) {  // earlier rotations on column j
        const T a = H[k * m + j], c = H[(k + 1) * m + j];
        H[k * m + j] = sm.cs[k] * a + sm.sn[k] * c;
        H[(k + 1) * m + j] = -sm.sn[k] * a + sm.cs[k] * c;
    }
    const T a = H[j * m + j], c = H[(j + 1) * m + j];
    const T d = hypot(a, c);
    sm.cs[j] = d == T(0) ? T(1) : a / d;
    sm.sn[j] = d == T(0) ? T(0) : c / d;
    H[j * m + j] = d;
    H[(j + 1) * m + j] = T(0);
    const T gj = sm.g[j];
    sm.g[j + 1] = -sm.sn[j] * gj;
    sm.g[j] = sm.cs[j] * gj;
    gs->iters += 1;
    gs->jdone = j + 1;
    gs->relres = fabs(sm.g[j + 1]) / gs->bnorm;
    sm.h1[kGmKmax] = hn;  // the norm for the normalisation kernel
    const bool conv = gs->relres <= gs->tol;
    if (conv || hn == T(0) || gs->iters >= gs->maxit || j + 1 >= m) {
        gs->cyc_stop = 1;
        gs->est_conv = conv || hn == T(0);
        if (conv || hn == T(0) || gs->iters >= gs->maxit) gs->skip = 1;
    }
}

// First update: w -= V_j h1 with ||w||^2 of the result accumulated on the way.
// The last block compares it with ||A v_j||^2 (wa[1], from the SpMV): if the
// pass kept more than 1/8 of the norm, the column is finished with h2 = 0;
// otherwise the reorthogonalisation runs (second dots pass, second update).
// The common case thus costs one dots pass and one update over the basis:
// 2 (j+1) n FMAs per Arnoldi step.
template <class T>
__global__ void __launch_bounds__(kVB)
    k_gm_upd1(int64_t n, int64_t ld, T *__restrict__ V, int j, GState<T> *gs, GSmall<T> sm, const T *wa,
              T *partials, unsigned *ticket)
{
    if (gs->skip) return;
    T *w = V + (int64_t)(j + 1) * ld;
    __shared__ T hs[kGmKmax];
    __shared__ T red[kVB / 32];
    const int jn = j + 1;
    if (threadIdx.x < kGmKmax) hs[threadIdx.x] = threadIdx.x < jn ? ldcg(sm.h1 + threadIdx.x) : T(0);
    __syncthreads();
    constexpr int R = 4;
    T ww = T(0);
    const int64_t stride = (int64_t)gridDim.x * kVB;
    for (int64_t i = blockIdx.x * (int64_t)kVB + threadIdx.x; i < n; i += R * stride) {
        bool ok[R];
        T wr[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            ok[u] = i + u * stride < n;
            wr[u] = ok[u] ? w[i + u * stride] : T(0);
        }
        gm_rows_update<T, R>(V, ld, i, stride, ok, jn, hs, wr);
#pragma unroll
        for (int u = 0; u < R; ++u) {
            if (ok[u]) w[i + u * stride] = wr[u];
            ww = fma(wr[u], wr[u], ww);  // zero for rows past the end
        }
    }
    const T bsum = block_sum<T, kVB>(ww, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = bsum;
    if (!last_block(ticket, gridDim.x)) return;
    T s = T(0);
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kVB) s += ldcg(partials + b);
    s = block_sum<T, kVB>(s, red);
    const bool again = s < T(kGmReorthKeep2) * ldcg(wa + 1);
    if (!again && threadIdx.x < jn) sm.h2[threadIdx.x] = T(0);
    __syncthreads();
    if (threadIdx.x != 0) return;
    gs->reorth = again ? 1 : 0;
    if (!again) gm_finish_column<T>(gs, sm, j, s);
}

// Second update (only when asked for): w -= V_j h2, ||w||^2; the last block
// finishes the column.
template <class T>
__global__ void __launch_bounds__(kVB)
    k_gm_upd2(int64_t n, int64_t ld, T *__restrict__ V, int j, GState<T> *gs, GSmall<T> sm, T *partials,
              unsigned *ticket)
{
    if (gs->skip || !gs->reorth) return;
    T *w = V + (int64_t)(j + 1) * ld;
    __shared__ T hs[kGmKmax];
    __shared__ T red[kVB / 32];
    const int jn = j + 1;
    if (threadIdx.x < kGmKmax) hs[threadIdx.x] = threadIdx.x < jn ? ldcg(sm.h2 + threadIdx.x) : T(0);
    __syncthreads();
    T ww = T(0);
    const int64_t stride = (int64_t)gridDim.x * kVB;
    for (int64_t i = blockIdx.x * (int64_t)kVB + threadIdx.x; i < n; i += 2 * stride) {
        const bool ok[2] = {true, i + stride < n};
        T wr[2] = {w[i], ok[1] ? w[i + stride] : T(0)};
        gm_rows_update<T, 2>(V, ld, i, stride, ok, jn, hs, wr);
        w[i] = wr[0];
        if (ok[1]) w[i + stride] = wr[1];
        ww = fma(wr[0], wr[0], ww);
        ww = fma(wr[1], wr[1], ww);
    }
    const T bsum = block_sum<T, kVB>(ww, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = bsum;
    if (!last_block(ticket, gridDim.x)) return;
    T s = T(0);
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kVB) s += ldcg(partials + b);
    s = block_sum<T, kVB>(s, red);
    if (threadIdx.x == 0) gm_finish_column<T>(gs, sm, j, s);
}

// v_{j+1} = w / ||w||  (Jacobi, right: also z = dinv v_{j+1}, the next SpMV's input)
template <class T>
__global__ void __launch_bounds__(kVB) k_gm_scale(int64_t n, int64_t ld, T *__restrict__ V, int j, const GState<T> *gs,
                                                  GSmall<T> sm, const T *__restrict__ dinv, T *__restrict__ z)
{
    // v_{j+1} is needed only while the cycle goes on
    if (gs->skip || gs->cyc_stop || gs->jdone != j + 1) return;
    const T inv = T(1) / ldcg(sm.h1 + kGmKmax);
    T *w = V + (int64_t)(j + 1) * ld;
    if (dinv) {
        for (int64_t i = blockIdx.x * (int64_t)kVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVB) {
            const T vi = w[i] * inv;
            w[i] = vi;
            z[i] = dinv[i] * vi;
        }
    } else {
        for (int64_t i = blockIdx.x * (int64_t)kVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVB) w[i] *= inv;
    }
}

// End of a cycle: y = H^{-1} g by back substitution (one thread; m <= 32)
template <class T> __global__ void k_gm_solve(GState<T> *gs, GSmall<T> sm)
{
    if (gs->done || threadIdx.x != 0 || blockIdx.x != 0) return;
    const int jn = gs->jdone, m = gs->m;
    for (int i = jn - 1; i >= 0; --i) {
        T s = sm.g[i];
        for (int k = i + 1; k < jn; ++k) s -= sm.H[i * m + k] * sm.y[k];
        sm.y[i] = s / sm.H[i * m + i];
    }
}

// x += sum_k y_k v_k  (Jacobi, right: x += dinv sum_k y_k v_k; uout != null
// (block-Jacobi): u = sum_k y_k v_k goes to uout and x is left to the block
// apply, which adds M^-1 u)
template <class T>
__global__ void __launch_bounds__(kVB)
    k_gm_update(int64_t n, int64_t ld, const T *__restrict__ V, T *__restrict__ x, const GState<T> *gs, GSmall<T> sm,
                const T *__restrict__ dinv, T *__restrict__ uout)
{
    if (gs->done) return;
    const int jn = gs->jdone;
    if (jn == 0) {
        if (uout)
            for (int64_t i = blockIdx.x * (int64_t)kVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVB)
                uout[i] = T(0);
        return;
    }
    __shared__ T ys[kGmKmax];
    if (threadIdx.x < kGmKmax) ys[threadIdx.x] = threadIdx.x < jn ? ldcg(sm.y + threadIdx.x) : T(0);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)kVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVB) {
        if (dinv || uout) {
            T ui = T(0);
#pragma unroll
            for (int k = 0; k < kGmKmax; ++k)
                if (k < jn) ui = fma(ys[k], V[(int64_t)k * ld + i], ui);
            if (uout) uout[i] = ui;
            else x[i] = fma(dinv[i], ui, x[i]);
        } else {
            T xi = x[i];
#pragma unroll
            for (int k = 0; k < kGmKmax; ++k)
                if (k < jn) xi = fma(ys[k], V[(int64_t)k * ld + i], xi);
            x[i] = xi;
        }
    }
}

// Start of a cycle: V[0] holds r = b - A x and dots[1] = r.r (SpMV epilogue).
// Decide convergence on the TRUE residual, else v_0 = r / ||r||, g = ||r|| e_1.
template <class T>
__global__ void __launch_bounds__(kVB) k_gm_start(int64_t n, T *__restrict__ v0, const T *dots, GState<T> *gs, GSmall<T> sm,
                                                  const T *__restrict__ dinv, T *__restrict__ z)
{
    if (gs->done) return;
    const T rr = ldcg(dots + 1);
    const T beta = sqrt(rr);
    const T rel = beta / gs->bnorm;
    const bool conv = rel <= gs->tol;
    const bool stag = !conv && gs->est_conv && gs->restarts >= kMaxRestarts;
    const bool maxed = gs->iters >= gs->maxit;
    if (conv || stag || maxed || beta == T(0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            gs->relres = rel;
            gs->done = 1;
            gs->skip = 1;
            gs->status = conv || beta == T(0) ? SPX_CONVERGED : (stag ? SPX_STAGNATED : SPX_MAX_ITER);
        }
        return;
    }
    const T inv = T(1) / beta;
    for (int64_t i = blockIdx.x * (int64_t)kVB + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVB) {
        const T vi = v0[i] * inv;
        v0[i] = vi;
        if (dinv) z[i] = dinv[i] * vi;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (gs->est_conv) gs->restarts += 1;
        gs->beta = beta;
        gs->relres = rel;
        gs->cyc_stop = 0;
        gs->est_conv = 0;
        gs->jdone = 0;
        gs->skip = 0;
        sm.g[0] = beta;
        for (int k = 1; k <= gs->m; ++k) sm.g[k] = T(0);
    }
}

// Splits a solver code of the ABI into the method, the Jacobi flag, the
// block-Jacobi block size (0: none) and block-Jacobi's adaptive storage.
int parse_solver_code(int code, int *solver, bool *jacobi, int *bs, bool *adaptive)
{
    const int base = code & 0xff;
    const int flags = code & ~0xff;
    *jacobi = false;
    *bs = 0;
    *adaptive = false;
    if (base < SPX_CG || base > SPX_CGS) return fail(SPX_ERR_INVALID, "unknown solver");
    if (flags == SPX_PRECOND_JACOBI) {
        *jacobi = true;
    } else if ((flags & 0xffff) == SPX_PRECOND_BLOCK_JACOBI ||
               (flags & 0xffff) == (SPX_PRECOND_BLOCK_JACOBI | SPX_PRECOND_BLOCK_ADAPTIVE)) {
        *adaptive = (flags & SPX_PRECOND_BLOCK_ADAPTIVE) != 0;
        const int b = (int)((unsigned)code >> SPX_PRECOND_BLOCK_SHIFT);
        if (b != 1 && b != 2 && b != 4 && b != 8 && b != 16 && b != 32)
            return fail(SPX_ERR_INVALID, "block-Jacobi block size must be 1, 2, 4, 8, 16 or 32");
        *jacobi = true;
        *bs = b;
    } else if (flags != 0) {
        return fail(SPX_ERR_INVALID, "unknown preconditioner flags in the solver code");
    }
    *solver = base;
    return SPX_OK;
}

// ------------------------------------------------------------------ host drivers
namespace {

template <class T> T *vec(SolverWork *w, int k) { return w->vecs.as<T>() + (int64_t)k * w->ld; }

// Grid of the fused vector kernels: a fixed number of blocks per SM, each
// thread striding over kU elements per step.  Three blocks of 256 per SM
// measured best on the 128^3 solves (CG 31.7 ms against 32.1 at four and 34.2
// at eight; BiCGSTAB 42.2 against 43.7 and 46.2): more blocks lengthen the
// last block's reduction of the partials, fewer leave bandwidth unused.
int vgrid(spx_ctx *ctx, int64_t n, int cap_per_sm = 3)
{
    int64_t g = ceil_div(n, kVB);
    const int64_t cap = (int64_t)ctx->grid_sms * cap_per_sm;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

template <class T> Epi<T> epi_plain(T *y) { Epi<T> e; e.y = y; return e; }

struct Timer {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double ms() const
    {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

// Runs `body` either directly on ctx->stream or, for reuse, as a captured CUDA
// graph keyed by `key` (captured on the private capture stream, launched on
// ctx->stream).  Keys include the context: a graph holds the context's error
// word, so a matrix solved from another context captures its own graph.  The first call of a key runs eagerly so that every lazily
// allocated scratch exists before capture.
template <class F> int run_chunk(spx_ctx *ctx, SolverWork *w, const uint64_t key_in[8], bool use_graph, F &&body)
{
    // the grids a capture records depend on the context's grid share: part of the key
    // (bits 52 and up of the context slot; context addresses stay below 2^48)
    uint64_t key[8];
    std::memcpy(key, key_in, sizeof(key));
    key[7] ^= (uint64_t)ctx->grid_sms << 52;
    bool same = w->gexec != nullptr;
    for (int i = 0; i < 8 && same; ++i) same = w->gkey[i] == key[i];
    if (same) {
        SPX_CUDA(cudaGraphLaunch(w->gexec, ctx->stream));
        return SPX_OK;
    }
    SPX_TRY(body());  // eager run (also the warm-up that allocates scratch)
    if (!use_graph) return SPX_OK;
    if (w->gexec) {
        cudaGraphExecDestroy(w->gexec);
        w->gexec = nullptr;
    }
    // capture the next chunk on the private stream, ordered after ctx->stream
    cudaEvent_t ev;
    SPX_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    SPX_CUDA(cudaEventRecord(ev, ctx->stream));
    SPX_CUDA(cudaStreamWaitEvent(ctx->capture_stream, ev, 0));
    cudaEventDestroy(ev);
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->capture_stream;
    cudaError_t e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeRelaxed);
    int st = SPX_OK;
    if (e == cudaSuccess) st = body();
    cudaGraph_t g = nullptr;
    cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ctx->capture_stream, &g) : e;
    ctx->stream = user;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    if (st != SPX_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    w->gexec = ex;
    std::memcpy(w->gkey, key, sizeof(w->gkey));
    return SPX_OK;
}

template <class T> struct KrylovRun {
    spx_ctx *ctx;
    spx_matrix *A;
    SolverWork *w;
    const T *b;
    T *x;
    bool use32;
    int solver;
};

// out = M^-1 in for block-Jacobi (see k_bj_apply for the modes)
template <class T, int BS, bool ADAPT>
int bj_apply_bs(spx_ctx *ctx, SolverWork *w, int64_t n, const T *in, T *out, int mode, const int *skip, T *x,
                int fin)
{
    const int g = vgrid(ctx, n);
    const T *minv = w->bjinv.as<T>();
    const float *m32 = ADAPT ? w->bjinv32.as<float>() : nullptr;
    KState<T> *st = w->state.as<KState<T>>();
    T *part = w->red.as<T>();
    unsigned *tk = w->ticket.as<unsigned>();
    cudaStream_t sm = ctx->stream;
    switch (mode) {
    case BJ_PLAIN:
        k_bj_apply<T, BS, BJ_PLAIN, ADAPT><<<g, kVB, 0, sm>>>(n, in, out, minv, m32, skip, x, st, fin, part, tk);
        break;
    case BJ_DOT:
        k_bj_apply<T, BS, BJ_DOT, ADAPT><<<g, kVB, 0, sm>>>(n, in, out, minv, m32, skip, x, st, fin, part, tk);
        break;
    case BJ_AXPY:
        k_bj_apply<T, BS, BJ_AXPY, ADAPT><<<g, kVB, 0, sm>>>(n, in, out, minv, m32, skip, x, st, fin, part, tk);
        break;
    default:
        k_bj_apply<T, BS, BJ_ADDX, ADAPT><<<g, kVB, 0, sm>>>(n, in, out, minv, m32, skip, x, st, fin, part, tk);
        break;
    }
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

template <class T, int BS>
int bj_apply_sel(spx_ctx *ctx, SolverWork *w, int64_t n, const T *in, T *out, int mode, const int *skip, T *x,
                 int fin)
{
    if constexpr (sizeof(T) == 8)
        if (w->bj_adapt) return bj_apply_bs<T, BS, true>(ctx, w, n, in, out, mode, skip, x, fin);
    return bj_apply_bs<T, BS, false>(ctx, w, n, in, out, mode, skip, x, fin);
}

template <class T>
int bj_apply(spx_ctx *ctx, SolverWork *w, int64_t n, const T *in, T *out, int mode, const int *skip, T *x = nullptr,
             int fin = FIN_NONE)
{
    switch (w->bs) {
    case 1: return bj_apply_sel<T, 1>(ctx, w, n, in, out, mode, skip, x, fin);
    case 2: return bj_apply_sel<T, 2>(ctx, w, n, in, out, mode, skip, x, fin);
    case 4: return bj_apply_sel<T, 4>(ctx, w, n, in, out, mode, skip, x, fin);
    case 8: return bj_apply_sel<T, 8>(ctx, w, n, in, out, mode, skip, x, fin);
    case 16: return bj_apply_sel<T, 16>(ctx, w, n, in, out, mode, skip, x, fin);
    case 32: return bj_apply_sel<T, 32>(ctx, w, n, in, out, mode, skip, x, fin);
    default: return fail(SPX_ERR_INVALID, "block-Jacobi block size must be 1, 2, 4, 8, 16 or 32");
    }
}

// One CG iteration: q = A p (+ p.q -> alpha); x, r update (+ r.r -> beta); p update.
// Jacobi: beta from r.z and p = z + beta p with z = dinv r (preconditioned CG).
// Block-Jacobi: x, r update with r.r (convergence); z = M^-1 r with r.z (beta)
// into q's place, q being spent; p = z + beta p.
template <class T> int cg_iter(KrylovRun<T> &R)
{
    SolverWork *w = R.w;
    KState<T> *st = w->state.as<KState<T>>();
    T *r = vec<T>(w, 0), *p = vec<T>(w, 1), *q = vec<T>(w, 2);
    const T *dinv = w->pre && !w->bs ? w->dinv.as<T>() : nullptr;
    const int64_t n = R.A->n;
    Epi<T> e = epi_plain(q);
    e.w = p;
    e.dots = w->dots.as<T>();
    e.fin = FIN_CG_ALPHA;
    e.fin_state = st;
    e.skip = &st->done;
    SPX_TRY(spmv_launch<T>(R.ctx, R.A, p, e, R.use32));
    const int g = vgrid(R.ctx, n);
    T *part = w->red.as<T>();
    unsigned *tk = w->ticket.as<unsigned>();
    if (w->bs) {
        k_cg_xr<T, 2><<<g, kVB, 0, R.ctx->stream>>>(n, R.x, r, p, q, nullptr, st, part, tk);
        SPX_TRY(bj_apply<T>(R.ctx, w, n, r, q, BJ_DOT, &st->done, nullptr, FIN_PCG_RZ));
        k_cg_p<T, false><<<g, kVB, 0, R.ctx->stream>>>(n, q, p, nullptr, st);
    } else if (dinv) {
        k_cg_xr<T, 1><<<g, kVB, 0, R.ctx->stream>>>(n, R.x, r, p, q, dinv, st, part, tk);
        k_cg_p<T, true><<<g, kVB, 0, R.ctx->stream>>>(n, r, p, dinv, st);
    } else {
        k_cg_xr<T, 0><<<g, kVB, 0, R.ctx->stream>>>(n, R.x, r, p, q, dinv, st, part, tk);
        k_cg_p<T, false><<<g, kVB, 0, R.ctx->stream>>>(n, r, p, dinv, st);
    }
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

// One BiCGSTAB iteration.  Jacobi / block-Jacobi (right): the SpMVs take
// ph = M^-1 p and sh = M^-1 s, and x is updated with them.
template <class T> int bi_iter(KrylovRun<T> &R)
{
    SolverWork *w = R.w;
    KState<T> *st = w->state.as<KState<T>>();
    T *r = vec<T>(w, 0), *rh = vec<T>(w, 1), *p = vec<T>(w, 2), *v = vec<T>(w, 3), *s = vec<T>(w, 4),
      *t = vec<T>(w, 5);
    const T *dinv = w->pre && !w->bs ? w->dinv.as<T>() : nullptr;
    T *ph = w->pre ? vec<T>(w, 6) : p, *sh = w->pre ? vec<T>(w, 7) : s;
    const int64_t n = R.A->n;
    const int g = vgrid(R.ctx, n);
    T *part = w->red.as<T>();
    unsigned *tk = w->ticket.as<unsigned>();
    if (dinv) k_bi_p<T, true><<<g, kVB, 0, R.ctx->stream>>>(n, r, p, v, ph, dinv, st);
    else k_bi_p<T, false><<<g, kVB, 0, R.ctx->stream>>>(n, r, p, v, ph, dinv, st);
    if (w->bs) SPX_TRY(bj_apply<T>(R.ctx, w, n, p, ph, BJ_PLAIN, &st->done));
    Epi<T> e = epi_plain(v);
    e.w = rh;
    e.dots = w->dots.as<T>();
    e.fin = FIN_BI_RV;
    e.fin_state = st;
    e.skip = &st->done;
    SPX_TRY(spmv_launch<T>(R.ctx, R.A, ph, e, R.use32));
    if (dinv) k_bi_s<T, true><<<g, kVB, 0, R.ctx->stream>>>(n, r, v, s, sh, dinv, st, part, tk);
    else k_bi_s<T, false><<<g, kVB, 0, R.ctx->stream>>>(n, r, v, s, sh, dinv, st, part, tk);
    if (w->bs) SPX_TRY(bj_apply<T>(R.ctx, w, n, s, sh, BJ_PLAIN, &st->skip_t));
    Epi<T> e2 = epi_plain(t);
    e2.w = s;
    e2.want_yy = true;
    e2.dots = w->dots.as<T>();
    e2.fin = FIN_BI_OMEGA;
    e2.fin_state = st;
    e2.skip = &st->skip_t;
    SPX_TRY(spmv_launch<T>(R.ctx, R.A, sh, e2, R.use32));
    k_bi_xr<T><<<g, kVB, 0, R.ctx->stream>>>(n, R.x, r, rh, ph, s, sh, t, st, part, tk);
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

// One CGS iteration: v = A p (+ r^.v -> alpha); q, w = u + q, x; v = A w;
// r update (+ r.r, r^.r -> convergence, beta); u, p updates.  Jacobi
// (right): the first SpMV takes ph = dinv p, and w = dinv (u + q).
// Block-Jacobi: w = u + q, then M^-1 w (in ph's place, ph being spent) with
// x += alpha M^-1 w, the second SpMV's input; after the p update ph = M^-1 p.
template <class T> int cgs_iter(KrylovRun<T> &R)
{
    SolverWork *w = R.w;
    KState<T> *st = w->state.as<KState<T>>();
    T *r = vec<T>(w, 0), *rh = vec<T>(w, 1), *p = vec<T>(w, 2), *u = vec<T>(w, 3), *q = vec<T>(w, 4),
      *v = vec<T>(w, 5), *ww = vec<T>(w, 6);
    const T *dinv = w->pre && !w->bs ? w->dinv.as<T>() : nullptr;
    T *ph = w->pre ? vec<T>(w, 7) : p;
    const int64_t n = R.A->n;
    const int g = vgrid(R.ctx, n);
    T *part = w->red.as<T>();
    unsigned *tk = w->ticket.as<unsigned>();
    Epi<T> e = epi_plain(v);
    e.w = rh;
    e.dots = w->dots.as<T>();
    e.fin = FIN_BI_RV;  // alpha = rho / (r^.v), breakdown on 0
    e.fin_state = st;
    e.skip = &st->done;
    SPX_TRY(spmv_launch<T>(R.ctx, R.A, ph, e, R.use32));
    if (w->bs) {
        k_cgs_qw<T, 2><<<g, kVB, 0, R.ctx->stream>>>(n, R.x, u, v, q, ww, nullptr, st);
        SPX_TRY(bj_apply<T>(R.ctx, w, n, ww, ph, BJ_AXPY, &st->done, R.x));
    } else if (dinv) {
        k_cgs_qw<T, 1><<<g, kVB, 0, R.ctx->stream>>>(n, R.x, u, v, q, ww, dinv, st);
    } else {
        k_cgs_qw<T, 0><<<g, kVB, 0, R.ctx->stream>>>(n, R.x, u, v, q, ww, dinv, st);
    }
    Epi<T> e2 = epi_plain(v);
    e2.skip = &st->done;
    SPX_TRY(spmv_launch<T>(R.ctx, R.A, w->bs ? ph : ww, e2, R.use32));
    k_cgs_r<T><<<g, kVB, 0, R.ctx->stream>>>(n, r, rh, v, st, part, tk);
    if (dinv) k_cgs_up<T, true><<<g, kVB, 0, R.ctx->stream>>>(n, r, q, u, p, ph, dinv, st);
    else k_cgs_up<T, false><<<g, kVB, 0, R.ctx->stream>>>(n, r, q, u, p, ph, dinv, st);
    if (w->bs) SPX_TRY(bj_apply<T>(R.ctx, w, n, p, ph, BJ_PLAIN, &st->done));
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

// r = b - A x with r.r; (re)initialise the recurrences.
template <class T> int krylov_init(KrylovRun<T> &R)
{
    SolverWork *w = R.w;
    KState<T> *st = w->state.as<KState<T>>();
    const int64_t n = R.A->n;
    T *r = vec<T>(w, 0);
    Epi<T> e;
    e.alpha = T(-1);
    e.beta = T(1);
    e.z = R.b;
    e.y = r;
    e.want_yy = true;
    e.dots = w->dots.as<T>();
    e.fin = R.solver == SPX_BICGSTAB ? FIN_INIT_BI : FIN_INIT_CG;  // CGS: rho = r^.r = r.r like CG
    e.fin_state = st;
    SPX_TRY(spmv_launch<T>(R.ctx, R.A, R.x, e, R.use32));
    const size_t bytes = (size_t)n * sizeof(T);
    if (R.solver == SPX_CG) {
        SPX_CUDA(cudaMemcpyAsync(vec<T>(w, 1), r, bytes, cudaMemcpyDeviceToDevice, R.ctx->stream));
    } else if (R.solver == SPX_CGS) {
        for (int k = 1; k <= 3; ++k)  // r^ = p = u = r
            SPX_CUDA(cudaMemcpyAsync(vec<T>(w, k), r, bytes, cudaMemcpyDeviceToDevice, R.ctx->stream));
    } else {
        SPX_CUDA(cudaMemcpyAsync(vec<T>(w, 1), r, bytes, cudaMemcpyDeviceToDevice, R.ctx->stream));  // r^
        SPX_CUDA(cudaMemsetAsync(vec<T>(w, 2), 0, bytes, R.ctx->stream));                        // p
        SPX_CUDA(cudaMemsetAsync(vec<T>(w, 3), 0, bytes, R.ctx->stream));                        // v
    }
    if (w->bs) {
        KState<T> *st = w->state.as<KState<T>>();
        if (R.solver == SPX_CG)  // p = z = M^-1 r, rho = r.z
            SPX_TRY(bj_apply<T>(R.ctx, w, n, r, vec<T>(w, 1), BJ_DOT, &st->done, nullptr, FIN_PCG_RHO0));
        else if (R.solver == SPX_CGS)  // ph = M^-1 p
            SPX_TRY(bj_apply<T>(R.ctx, w, n, vec<T>(w, 2), vec<T>(w, 7), BJ_PLAIN, &st->done));
    } else if (w->pre) {
        KState<T> *st = w->state.as<KState<T>>();
        const int g = vgrid(R.ctx, n);
        const T *dinv = w->dinv.as<T>();
        if (R.solver == SPX_CG)  // p = z = dinv r, rho = r.z
            k_pcg_init<T><<<g, kVB, 0, R.ctx->stream>>>(n, r, vec<T>(w, 1), dinv, st, w->red.as<T>(),
                                                       w->ticket.as<unsigned>());
        else if (R.solver == SPX_CGS)  // ph = dinv p
            k_jscale<T><<<g, kVB, 0, R.ctx->stream>>>(n, vec<T>(w, 2), dinv, vec<T>(w, 7), st);
        SPX_CUDA(cudaGetLastError());
    }
    return SPX_OK;
}

// M^{-1} = 1 / diag(A) for a Jacobi-preconditioned solve, in the work's precision
template <class T> int ensure_dinv(spx_ctx *ctx, spx_matrix *A, SolverWork *w)
{
    if (!w->pre || w->bs || w->dinv.p) return SPX_OK;
    const int64_t n = A->n;
    SPX_TRY(dbuf_alloc(ctx, w->dinv, (size_t)(n > 0 ? n : 1) * sizeof(T)));
    const int g = (int)std::min<int64_t>(ceil_div(n > 0 ? n : 1, 256), (int64_t)ctx->grid_sms * 16);
    const bool csr = A->format == SPX_CSR;
    const int64_t ew = (A->format == SPX_ELL || A->format == SPX_HYB) ? A->ell_w : 0;
    const int64_t cn = (A->format == SPX_COO || A->format == SPX_HYB) ? A->coo_nnz : 0;
    if (A->dtype == SPX_F64)
        k_jacobi_dinv<double, T><<<g, 256, 0, ctx->stream>>>(
            n, csr ? A->rp.as<int>() : nullptr, A->col.as<int>(), A->val.as<double>(), A->ell_ld, ew,
            A->ell_col.as<int>(), A->ell_val.as<double>(), cn, A->coo_row.as<int>(), A->coo_col.as<int>(),
            A->coo_val.as<double>(), w->dinv.as<T>());
    else
        k_jacobi_dinv<float, T><<<g, 256, 0, ctx->stream>>>(
            n, csr ? A->rp.as<int>() : nullptr, A->col.as<int>(), A->val.as<float>(), A->ell_ld, ew,
            A->ell_col.as<int>(), A->ell_val.as<float>(), cn, A->coo_row.as<int>(), A->coo_col.as<int>(),
            A->coo_val.as<float>(), w->dinv.as<T>());
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

template <class V, class T>
int bj_build_small(spx_ctx *ctx, spx_matrix *A, SolverWork *w, float *m32)
{
    const int64_t n = A->n, nb = ceil_div(n > 0 ? n : 1, (int64_t)w->bs);
    const int g = (int)std::min<int64_t>(ceil_div(nb, kBjTpb), (int64_t)ctx->grid_sms * 16);
    const bool csr = A->format == SPX_CSR;
    const int64_t ew = (A->format == SPX_ELL || A->format == SPX_HYB) ? A->ell_w : 0;
    const int64_t cn = (A->format == SPX_COO || A->format == SPX_HYB) ? A->coo_nnz : 0;
    const V *val = A->val.as<V>(), *ev = A->ell_val.as<V>(), *cv = A->coo_val.as<V>();
#define SPX_BJ_SMALL(B_)                                                                                            \
    k_bj_build_t<V, T, B_><<<g, kBjTpb, 0, ctx->stream>>>(n, csr ? A->rp.as<int>() : nullptr, A->col.as<int>(), val, \
                                                         A->ell_ld, ew, A->ell_col.as<int>(), ev, cn,               \
                                                         A->coo_row.as<int>(), A->coo_col.as<int>(), cv,             \
                                                         w->bjinv.as<T>(), m32)
    switch (w->bs) {
    case 1: SPX_BJ_SMALL(1); break;
    case 2: SPX_BJ_SMALL(2); break;
    case 4: SPX_BJ_SMALL(4); break;
    default: SPX_BJ_SMALL(8); break;
    }
#undef SPX_BJ_SMALL
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

// block-Jacobi inverses (FP64 elimination, stored in the work's precision)
template <class T> int ensure_bjinv(spx_ctx *ctx, spx_matrix *A, SolverWork *w)
{
    if (!w->bs || w->bjinv.p) return SPX_OK;
    const int64_t n = A->n, bs = w->bs;
    const int64_t nb = ceil_div(n > 0 ? n : 1, bs);
    SPX_TRY(dbuf_alloc(ctx, w->bjinv, (size_t)(nb * bs * bs) * sizeof(T)));
    if (w->bj_adapt) SPX_TRY(dbuf_alloc(ctx, w->bjinv32, (size_t)(nb * bs * bs) * sizeof(float)));
    float *m32 = w->bj_adapt ? w->bjinv32.as<float>() : nullptr;
    if (bs <= 8) return A->dtype == SPX_F64 ? bj_build_small<double, T>(ctx, A, w, m32) : bj_build_small<float, T>(ctx, A, w, m32);
    const int g = (int)std::min<int64_t>(ceil_div(nb, kBjWarps), (int64_t)ctx->grid_sms * 32);
    const int smem = kBjWarps * (int)(bs * 2 * bs + bs) * 8;
    const bool csr = A->format == SPX_CSR;
    const int64_t ew = (A->format == SPX_ELL || A->format == SPX_HYB) ? A->ell_w : 0;
    const int64_t cn = (A->format == SPX_COO || A->format == SPX_HYB) ? A->coo_nnz : 0;
    if (A->dtype == SPX_F64)
        k_bj_build<double, T><<<g, 32 * kBjWarps, smem, ctx->stream>>>(
            n, (int)bs, csr ? A->rp.as<int>() : nullptr, A->col.as<int>(), A->val.as<double>(), A->ell_ld, ew,
            A->ell_col.as<int>(), A->ell_val.as<double>(), cn, A->coo_row.as<int>(), A->coo_col.as<int>(),
            A->coo_val.as<double>(), w->bjinv.as<T>(), m32);
    else
        k_bj_build<float, T><<<g, 32 * kBjWarps, smem, ctx->stream>>>(
            n, (int)bs, csr ? A->rp.as<int>() : nullptr, A->col.as<int>(), A->val.as<float>(), A->ell_ld, ew,
            A->ell_col.as<int>(), A->ell_val.as<float>(), cn, A->coo_row.as<int>(), A->coo_col.as<int>(),
            A->coo_val.as<float>(), w->bjinv.as<T>(), m32);
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

template <class T> int ensure_prec(spx_ctx *ctx, spx_matrix *A, SolverWork *w)
{
    return w->bs ? ensure_bjinv<T>(ctx, A, w) : ensure_dinv<T>(ctx, A, w);
}

// true residual ||b - A x||^2 -> dots[1] (scratch vector)
template <class T> int true_residual(KrylovRun<T> &R, T *scratch)
{
    Epi<T> e;
    e.alpha = T(-1);
    e.beta = T(1);
    e.z = R.b;
    e.y = scratch;
    e.want_yy = true;
    SolverWork *wk = R.w;
    e.dots = wk->dots.as<T>();
    return spmv_launch<T>(R.ctx, R.A, R.x, e, R.use32);
}

template <class T> int read_state(spx_ctx *ctx, SolverWork *w, size_t bytes)
{
    SPX_CUDA(cudaMemcpyAsync(w->host, w->state.p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    return SPX_OK;
}

template <class T> int read_dots(spx_ctx *ctx, SolverWork *w, T out[2])
{
    SPX_CUDA(cudaMemcpyAsync(out, w->dots.p, 2 * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    return SPX_OK;
}

int check_dev_err(spx_ctx *ctx)
{
    unsigned h = 0;
    SPX_CUDA(cudaMemcpyAsync(&h, ctx->dev_err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    if (h) {
        cudaMemsetAsync(ctx->dev_err, 0, sizeof(unsigned), ctx->stream);
        return fail(SPX_ERR_TIMEOUT, "a bounded device-side wait gave up (error word " + std::to_string(h) + ")");
    }
    return SPX_OK;
}

// CG / BiCGSTAB / CGS.  inner: FP32 inner solve of refinement (no
// true-residual check, no restarts; x starts at 0; CGS also ends on the stall
// rule).  fixed > 0: run exactly that many iterations (tol ignored).
template <class T>
int run_short(spx_ctx *ctx, spx_matrix *A, SolverWork *w, int solver, const T *b, T *x, double tol,
              int64_t maxit, bool use32, bool inner, int64_t fixed, spx_solve_info *info)
{
    KrylovRun<T> R{ctx, A, w, b, x, use32, solver};
    KState<T> hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.rtol2 = fixed > 0 ? T(0) : (T)(tol * tol);
    hs.maxit = fixed > 0 ? fixed : maxit;
    hs.status = SPX_MAX_ITER;
    hs.mark = T(1);
    hs.stall = inner && solver == SPX_CGS ? kIrCgsStall : 0;
    KState<T> *st = w->state.as<KState<T>>();
    SPX_CUDA(cudaMemcpyAsync(st, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream));
    const int64_t n = A->n;
    k_dot_fin<T><<<vgrid(ctx, n), kVB, 0, ctx->stream>>>(n, b, b, FIN_SET_BB, st, w->red.as<T>(),
                                                         w->ticket.as<unsigned>());
    SPX_CUDA(cudaGetLastError());
    if (inner) SPX_CUDA(cudaMemsetAsync(x, 0, (size_t)n * sizeof(T), ctx->stream));
    KState<T> *h = static_cast<KState<T> *>(w->host);
    int restarts = 0;
    const int chunk = fixed > 0 ? 64 : (n < 200000 ? 32 : 16);
    const bool graphs = graphs_for(A);
    for (;;) {
        SPX_TRY(krylov_init(R));
        SPX_TRY(read_state<T>(ctx, w, sizeof(KState<T>)));
        if (h->bb == T(0)) {  // b = 0: x = 0
            SPX_CUDA(cudaMemsetAsync(x, 0, (size_t)n * sizeof(T), ctx->stream));
            SPX_CUDA(cudaStreamSynchronize(ctx->stream));
            info->status = SPX_CONVERGED;
            info->iterations = 0;
            info->relres_recurrence = info->relres_true = 0.0;
            return SPX_OK;
        }
        int64_t launched = 0;
        while (!h->done) {
            const uint64_t key[8] = {(uint64_t)solver, (uint64_t)(uintptr_t)x, (uint64_t)(uintptr_t)b,
                                     (uint64_t)use32, (uint64_t)chunk, (uint64_t)sizeof(T) | ((uint64_t)w->pre << 8) | ((uint64_t)w->bs << 16) |
                                     ((uint64_t)w->bj_adapt << 24),
                                     (uint64_t)(uintptr_t)A, (uint64_t)(uintptr_t)ctx << 1};
            SPX_TRY(run_chunk(ctx, w, key, graphs, [&]() -> int {
                for (int c = 0; c < chunk; ++c)
                    SPX_TRY(solver == SPX_CG ? cg_iter(R) : solver == SPX_CGS ? cgs_iter(R) : bi_iter(R));
                return SPX_OK;
            }));
            launched += chunk;
            SPX_TRY(read_state<T>(ctx, w, sizeof(KState<T>)));
            if (launched > hs.maxit + 4 * chunk) return fail(SPX_ERR_CUDA, "solver did not stop");
        }
        SPX_TRY(check_dev_err(ctx));
        info->status = h->status;
        info->iterations = h->iters;
        info->relres_recurrence = (double)h->relres;
        if (inner) break;
        T d[2];
        SPX_TRY(true_residual(R, vec<T>(w, w->nvec - 1)));
        SPX_TRY(read_dots<T>(ctx, w, d));
        info->relres_true = std::sqrt((double)d[1] / (double)h->bb);
        if (fixed > 0 || h->status != SPX_CONVERGED || info->relres_true <= tol) break;
        if (restarts == kMaxRestarts) {
            info->status = SPX_STAGNATED;
            break;
        }
        ++restarts;
    }
    info->restarts = restarts;
    return SPX_OK;
}

template <class T>
int run_gmres(spx_ctx *ctx, spx_matrix *A, SolverWork *w, const T *b, T *x, double tol, int64_t maxit, int m,
              bool use32, bool inner, int64_t fixed, spx_solve_info *info)
{
    const int64_t n = A->n, ld = w->ld;
    T *V = w->vecs.as<T>();
    const T *dinv = w->pre && !w->bs ? w->dinv.as<T>() : nullptr;
    T *Z = w->pre ? V + (int64_t)(m + 2) * ld : nullptr;  // M^{-1} v_j (right preconditioning)
    const bool bj = w->bs > 0;
    GState<T> *gs = w->state.as<GState<T>>();
    GSmall<T> sm;
    T *base = w->small.as<T>();
    sm.H = base;
    sm.cs = sm.H + (m + 1) * m;
    sm.sn = sm.cs + m + 1;
    sm.g = sm.sn + m + 1;
    sm.y = sm.g + m + 2;
    sm.h1 = sm.y + m + 1;
    sm.h2 = sm.h1 + kGmKmax + 2;
    T *dots = w->dots.as<T>();
    T *part = w->red.as<T>();
    unsigned *tk = w->ticket.as<unsigned>();
    // ||b||
    T bb = 0;
    {
        SPX_TRY(dot_launch<T>(ctx, n, b, b, dots));
        T d[2];
        SPX_CUDA(cudaMemcpyAsync(d, dots, sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
        SPX_CUDA(cudaStreamSynchronize(ctx->stream));
        bb = d[0];
    }
    if (inner) SPX_CUDA(cudaMemsetAsync(x, 0, (size_t)n * sizeof(T), ctx->stream));
    if (bb == T(0)) {
        SPX_CUDA(cudaMemsetAsync(x, 0, (size_t)n * sizeof(T), ctx->stream));
        SPX_CUDA(cudaStreamSynchronize(ctx->stream));
        info->status = SPX_CONVERGED;
        return SPX_OK;
    }
    GState<T> hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.bnorm = std::sqrt(bb);
    hs.tol = fixed > 0 ? T(0) : (T)tol;
    hs.m = m;
    hs.maxit = fixed > 0 ? fixed : maxit;
    hs.status = SPX_MAX_ITER;
    SPX_CUDA(cudaMemcpyAsync(gs, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream));
    const int g = vgrid(ctx, n, 2);
    int gd = (int)ceil_div(n, kGmRows);  // dots passes: persistent grid, at most 4 blocks per SM
    if (gd > 4 * ctx->grid_sms) gd = 4 * ctx->grid_sms;
    if (gd < 1) gd = 1;
    const int gu = vgrid(ctx, n, 8);
    auto cycle = [&]() -> int {
        // restart: V[0] = b - A x, r.r
        Epi<T> e;
        e.alpha = T(-1);
        e.beta = T(1);
        e.z = b;
        e.y = V;
        e.want_yy = true;
        e.dots = dots;
        e.skip = &gs->done;
        SPX_TRY(spmv_launch<T>(ctx, A, x, e, use32));
        k_gm_start<T><<<g, kVB, 0, ctx->stream>>>(n, V, dots, gs, sm, dinv, Z);
        if (bj) SPX_TRY(bj_apply<T>(ctx, w, n, V, Z, BJ_PLAIN, &gs->skip));
        for (int j = 0; j < m; ++j) {
            Epi<T> ea = epi_plain(V + (int64_t)(j + 1) * ld);
            ea.skip = &gs->skip;
            ea.want_yy = true;  // ||A v_j||^2 -> dots[1], for the reorthogonalisation test
            ea.dots = dots;
            SPX_TRY(spmv_launch<T>(ctx, A, Z ? Z : V + (int64_t)j * ld, ea, use32));  // A v_j or A M^-1 v_j
            k_gm_dots<T><<<gd, kVB, 0, ctx->stream>>>(n, ld, V, j, gs, sm.h1, part, tk, false);
            k_gm_upd1<T><<<gu, kVB, 0, ctx->stream>>>(n, ld, V, j, gs, sm, dots, part, tk);
            k_gm_dots<T><<<gd, kVB, 0, ctx->stream>>>(n, ld, V, j, gs, sm.h2, part, tk, true);
            k_gm_upd2<T><<<gu, kVB, 0, ctx->stream>>>(n, ld, V, j, gs, sm, part, tk);
            k_gm_scale<T><<<g, kVB, 0, ctx->stream>>>(n, ld, V, j, gs, sm, dinv, Z);
            // (when this step ended the cycle, the apply's Z is never read: the next
            // cycle's start recomputes it)
            if (bj) SPX_TRY(bj_apply<T>(ctx, w, n, V + (int64_t)(j + 1) * ld, Z, BJ_PLAIN, &gs->skip));
        }
        k_gm_solve<T><<<1, 32, 0, ctx->stream>>>(gs, sm);
        k_gm_update<T><<<g, kVB, 0, ctx->stream>>>(n, ld, V, x, gs, sm, dinv, bj ? Z : nullptr);
        if (bj) SPX_TRY(bj_apply<T>(ctx, w, n, Z, (T *)nullptr, BJ_ADDX, &gs->done, x));
        SPX_CUDA(cudaGetLastError());
        return SPX_OK;
    };
    GState<T> *h = static_cast<GState<T> *>(w->host);
    int64_t cycles = 0;
    for (;;) {
        const uint64_t key[8] = {(uint64_t)SPX_GMRES, (uint64_t)(uintptr_t)x, (uint64_t)(uintptr_t)b,
                                 (uint64_t)use32, (uint64_t)m, (uint64_t)sizeof(T) | ((uint64_t)w->pre << 8) | ((uint64_t)w->bs << 16) |
                                     ((uint64_t)w->bj_adapt << 24),
                                 (uint64_t)(uintptr_t)A, ((uint64_t)(uintptr_t)ctx << 1) | 1u};
        SPX_TRY(run_chunk(ctx, w, key, graphs_for(A), cycle));
        SPX_TRY(read_state<T>(ctx, w, sizeof(GState<T>)));
        ++cycles;
        if (h->done) break;
        if (inner && h->cyc_stop && (h->est_conv || h->iters >= h->maxit)) break;
        if (cycles > hs.maxit + 8) return fail(SPX_ERR_CUDA, "GMRES did not stop");
    }
    SPX_TRY(check_dev_err(ctx));
    info->status = h->done ? h->status : (h->est_conv ? SPX_CONVERGED : SPX_MAX_ITER);
    info->iterations = h->iters;
    info->restarts = h->restarts;
    info->relres_recurrence = (double)h->relres;
    if (!inner) {
        KrylovRun<T> R{ctx, A, w, b, x, use32, SPX_GMRES};
        T d[2];
        SPX_TRY(true_residual(R, V + (int64_t)(m + 1) * ld));
        SPX_TRY(read_dots<T>(ctx, w, d));
        info->relres_true = std::sqrt((double)d[1]) / (double)hs.bnorm;
    }
    return SPX_OK;
}

// ------------------------------------------------------------------ mixed precision
template <class S, class D> __global__ void k_cast_scale(int64_t n, const S *__restrict__ a, S scale, D *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = static_cast<D>(a[i] * scale);
}

__global__ void k_ir_update(int64_t n, double *__restrict__ x, const float *__restrict__ d, double s)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = fma(s, (double)d[i], x[i]);
}

// r32 = fl32(r64) with r32.r32 reduced (FP32, fixed order) into the state by `fin`
// (FIN_RU_FIRST / FIN_RU_NEXT)
__global__ void __launch_bounds__(kVB)
    k_ru_replace(int64_t n, const double *__restrict__ r64, float *__restrict__ r32, int fin, KState<float> *st,
                 float *partials, unsigned *ticket)
{
    float d0 = 0.f;
    double rv[kU];
    SPX_ROWS_LOOP(rv[u] = r64[i];, const float ri = (float)rv[u]; r32[i] = ri; d0 = fmaf(ri, ri, d0);)
    grid_dots_finish<float, kVB>(d0, 0.f, (float *)nullptr, fin, st, partials, ticket);
}

// Mixed-precision CG with reliable updates (the residual replacement of
// Sleijpen and van der Vorst, 1996): the FP32 CG iteration (the kernels of
// the FP32 solve, on the FP32 value copy) runs with its iterate accumulated
// in an FP32 correction d; when its recurrence residual has fallen below
// delta = 0.1 of its largest value since the last update (or below tol ||b||,
// or the budget is spent) the iteration stops, d is added to the FP64 x, the
// residual b - A x is formed in FP64 with the FP64 values, and its rounding
// replaces the FP32 residual; the direction p is kept and beta is formed with
// the replaced residual, so the solve keeps CG's iteration count (a
// refinement cycle that restarts the inner solve starts its Krylov space
// again: 618 FP32 iterations against 428 for FP64 CG on the 7-point Poisson
// matrix 128^3).  restarts reports the updates.
constexpr double kRuDelta = 0.1;

int run_cg_reliable(spx_ctx *ctx, spx_matrix *A, const double *b, double *x, double tol, int64_t maxit,
                    spx_solve_info *info)
{
    const int64_t n = A->n;
    SolverWork *&w = A->work;
    SPX_TRY(work_prepare<double>(ctx, w, n, SPX_CG, 0));  // FP64: the residual
    SPX_TRY(work_prepare<float>(ctx, w->inner, n, SPX_CG, 0));
    if (!w->ir.p) SPX_TRY(dbuf_alloc(ctx, w->ir, (size_t)n * 8 + 2 * (size_t)round_up(n, 64) * 4 + 256));
    SolverWork *wi = w->inner;
    double *r = w->ir.as<double>();
    float *d32 = reinterpret_cast<float *>(w->ir.as<char>() + round_up((size_t)n * 8, 256));
    float *r32 = vec<float>(wi, 0), *p32 = vec<float>(wi, 1);
    KState<float> *st = wi->state.as<KState<float>>();
    KState<float> *h = static_cast<KState<float> *>(wi->host);
    const int g = vgrid(ctx, n);
    double bb = 0;
    {
        double d[2];
        SPX_TRY(dot_launch<double>(ctx, n, b, b, w->dots.as<double>()));
        SPX_CUDA(cudaMemcpyAsync(d, w->dots.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
        SPX_CUDA(cudaStreamSynchronize(ctx->stream));
        bb = d[0];
    }
    if (bb == 0.0) {
        SPX_CUDA(cudaMemsetAsync(x, 0, (size_t)n * 8, ctx->stream));
        SPX_CUDA(cudaStreamSynchronize(ctx->stream));
        info->status = SPX_CONVERGED;
        return SPX_OK;
    }
    // r = b - A x in FP64 (with ||r||^2); true if it meets tol
    auto fp64_residual = [&](double &rel) -> int {
        Epi<double> e;
        e.alpha = -1.0;
        e.beta = 1.0;
        e.z = b;
        e.y = r;
        e.want_yy = true;
        e.dots = w->dots.as<double>();
        SPX_TRY(spmv_launch<double>(ctx, A, x, e, false));
        double d[2];
        SPX_TRY(read_dots<double>(ctx, w, d));
        rel = std::sqrt(d[1] / bb);
        return SPX_OK;
    };
    KState<float> hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.bb = (float)bb;
    hs.rtol2 = (float)(tol * tol);
    hs.tol2 = (float)(tol * tol * bb);
    hs.maxit = maxit;
    hs.status = SPX_MAX_ITER;
    hs.ru_delta2 = (float)(kRuDelta * kRuDelta);
    SPX_CUDA(cudaMemcpyAsync(st, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream));
    SPX_CUDA(cudaMemsetAsync(d32, 0, (size_t)n * 4, ctx->stream));
    double rel = 0.0;
    SPX_TRY(fp64_residual(rel));
    int status = rel <= tol ? SPX_CONVERGED : SPX_MAX_ITER;
    int updates = 0;
    if (status != SPX_CONVERGED) {
        k_ru_replace<<<g, kVB, 0, ctx->stream>>>(n, r, r32, FIN_RU_FIRST, st, wi->red.as<float>(),
                                                 wi->ticket.as<unsigned>());
        SPX_CUDA(cudaMemcpyAsync(p32, r32, (size_t)n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    KrylovRun<float> R{ctx, A, wi, nullptr, d32, true, SPX_CG};
    const int chunk = n < 200000 ? 32 : 16;
    const bool graphs = graphs_for(A);
    int64_t launched = 0;
    while (status != SPX_CONVERGED) {
        SPX_TRY(read_state<float>(ctx, wi, sizeof(KState<float>)));
        while (!h->done) {
            const uint64_t key[8] = {(uint64_t)SPX_CG,   (uint64_t)(uintptr_t)d32, 0, 1, (uint64_t)chunk, 4 | (1u << 30),
                                     (uint64_t)(uintptr_t)A, (uint64_t)(uintptr_t)ctx << 1};
            SPX_TRY(run_chunk(ctx, wi, key, graphs, [&]() -> int {
                for (int c = 0; c < chunk; ++c) SPX_TRY(cg_iter(R));
                return SPX_OK;
            }));
            launched += chunk;
            SPX_TRY(read_state<float>(ctx, wi, sizeof(KState<float>)));
            if (launched > maxit + 4 * chunk) return fail(SPX_ERR_CUDA, "solver did not stop");
        }
        // reliable update: x += d in FP64, the residual again in FP64
        k_ir_update<<<g, kVB, 0, ctx->stream>>>(n, x, d32, 1.0);
        SPX_CUDA(cudaGetLastError());
        SPX_CUDA(cudaMemsetAsync(d32, 0, (size_t)n * 4, ctx->stream));
        SPX_TRY(fp64_residual(rel));
        ++updates;
        if (rel <= tol) {
            status = SPX_CONVERGED;
            break;
        }
        if (h->status != SPX_CONVERGED) {  // the budget is spent, or the iteration broke down
            status = h->status;
            break;
        }
        // the rounding of the FP64 residual replaces r; beta with it; p = r + beta p
        k_ru_replace<<<g, kVB, 0, ctx->stream>>>(n, r, r32, FIN_RU_NEXT, st, wi->red.as<float>(),
                                                 wi->ticket.as<unsigned>());
        k_cg_p<float, false><<<g, kVB, 0, ctx->stream>>>(n, r32, p32, nullptr, st);
        SPX_CUDA(cudaGetLastError());
    }
    SPX_TRY(check_dev_err(ctx));
    SPX_TRY(read_state<float>(ctx, wi, sizeof(KState<float>)));
    info->status = status;
    info->iterations = h->iters;
    info->inner_iterations = h->iters;
    info->restarts = updates;
    info->relres_recurrence = rel;
    info->relres_true = rel;
    return SPX_OK;
}

int run_ir(spx_ctx *ctx, spx_matrix *A, const double *b, double *x, int solver, double tol, int64_t maxit,
           int m, bool pre, int bs, bool adapt, spx_solve_info *info)
{
    if (solver == SPX_CG && !pre && bs == 0) return run_cg_reliable(ctx, A, b, x, tol, maxit, info);
    const int64_t n = A->n;
    SolverWork *&w = A->work;
    SPX_TRY(work_prepare<double>(ctx, w, n, SPX_CG, 0));  // outer: r and scratch only
    SPX_TRY(work_prepare<float>(ctx, w->inner, n, solver, solver == SPX_GMRES ? m : 0, pre, bs, adapt));
    SPX_TRY(ensure_prec<float>(ctx, A, w->inner));
    if (!w->ir.p) SPX_TRY(dbuf_alloc(ctx, w->ir, (size_t)n * 8 + 2 * (size_t)round_up(n, 64) * 4 + 256));
    double *r = w->ir.as<double>();
    float *r32 = reinterpret_cast<float *>(w->ir.as<char>() + round_up((size_t)n * 8, 256));
    float *d32 = r32 + round_up((size_t)n, 64);
    double bb = 0;
    {
        double d[2];
        SPX_TRY(dot_launch<double>(ctx, n, b, b, w->dots.as<double>()));
        SPX_CUDA(cudaMemcpyAsync(d, w->dots.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
        SPX_CUDA(cudaStreamSynchronize(ctx->stream));
        bb = d[0];
    }
    if (bb == 0.0) {
        SPX_CUDA(cudaMemsetAsync(x, 0, (size_t)n * 8, ctx->stream));
        SPX_CUDA(cudaStreamSynchronize(ctx->stream));
        info->status = SPX_CONVERGED;
        return SPX_OK;
    }
    const double inner_tol = 1e-4;
    const int max_outer = 20;
    int64_t inner_total = 0;
    int outer = 0;
    double rel = 0.0;
    int status = SPX_MAX_ITER;
    const int g = vgrid(ctx, n);
    for (;; ++outer) {
        // r = b - A64 x (FP64), ||r||
        Epi<double> e;
        e.alpha = -1.0;
        e.beta = 1.0;
        e.z = b;
        e.y = r;
        e.want_yy = true;
        e.dots = w->dots.as<double>();
        SPX_TRY(spmv_launch<double>(ctx, A, x, e, false));
        double d[2];
        SPX_TRY(read_dots<double>(ctx, w, d));
        const double rn = std::sqrt(d[1]);
        rel = rn / std::sqrt(bb);
        if (rel <= tol) {
            status = SPX_CONVERGED;
            break;
        }
        if (outer >= max_outer || inner_total >= maxit) break;
        k_cast_scale<double, float><<<g, kVB, 0, ctx->stream>>>(n, r, 1.0 / rn, r32);
        SPX_CUDA(cudaGetLastError());
        spx_solve_info ii;
        std::memset(&ii, 0, sizeof(ii));
        const int64_t cyc_max = std::min<int64_t>(maxit - inner_total, kIrInnerCap);
        if (solver == SPX_GMRES)
            SPX_TRY(run_gmres<float>(ctx, A, w->inner, r32, d32, inner_tol, cyc_max, m, true, true, 0, &ii));
        else
            SPX_TRY(run_short<float>(ctx, A, w->inner, solver, r32, d32, inner_tol, cyc_max, true, true, 0, &ii));
        inner_total += ii.iterations;
        k_ir_update<<<g, kVB, 0, ctx->stream>>>(n, x, d32, rn);
        SPX_CUDA(cudaGetLastError());
    }
    info->status = status;
    info->iterations = inner_total;
    info->inner_iterations = inner_total;
    info->restarts = outer;
    info->relres_recurrence = rel;
    info->relres_true = rel;
    return SPX_OK;
}

template <class T>
int solve_typed(spx_ctx *ctx, spx_matrix *A, const T *b, T *x, int solver, double tol, int64_t maxit, int m,
                bool use32, int64_t fixed, bool pre, int bs, bool adapt, spx_solve_info *info)
{
    SPX_TRY(work_prepare<T>(ctx, A->work, A->n, solver, solver == SPX_GMRES ? m : 0, pre, bs, adapt));
    SPX_TRY(ensure_prec<T>(ctx, A, A->work));
    if (solver == SPX_GMRES) return run_gmres<T>(ctx, A, A->work, b, x, tol, maxit, m, use32, false, fixed, info);
    return run_short<T>(ctx, A, A->work, solver, b, x, tol, maxit, use32, false, fixed, info);
}

// ------------------------------------------------------------------ single-launch route for small systems
// Small systems are solved by one launch that runs every iteration, where the
// general path pays three launches and a device-wide reduction per iteration
// (the 2D Laplacian on a 64 x 64 grid, n = 4096: 23 us per CG iteration
// there).  CG in FP64 or FP32 on up to kSmallSolveRows rows runs on one
// cluster of 16 (or 8) SMs (cluster.cu); BiCGSTAB, CGS and FP32-inner
// refinement on up to kSmallBatchRows rows run in the persistent batched
// kernel as a batch of one (one SM, whose two FP64 lanes bound it, so larger
// systems take the general path).  CSR matrices whose SpMV kernel is left to
// the library, no preconditioner, run to a tolerance.  The batch (the matrix's
// own copy of the CSR arrays, from its creating context) is built on first use
// and kept with the matrix.
constexpr int64_t kSmallSolveRows = 32768;   // CG on a cluster
constexpr int64_t kSmallBatchRows = 4096;    // the other solvers on one SM

int small_solve(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, int solver, double tol, int64_t maxit,
                int precision, spx_solve_info *info)
{
    const bool mixed = precision == SPX_PREC_MIXED;
    if (mixed ? A->dtype != SPX_F64 : (precision == SPX_PREC_F64 ? SPX_F64 : SPX_F32) != A->dtype)
        return SPX_ERR_UNSUPPORTED;  // the general path reports the mismatch
    if (solver == SPX_CG && !mixed && A->n <= cluster_cg_max_rows()) {  // one cluster of SMs: see cluster.cu
        const int st = cluster_cg_solve(ctx, A, b, x, tol, maxit, info);
        if (st != SPX_ERR_UNSUPPORTED) return st;
    }
    if (A->n > kSmallBatchRows || A->n > batch_max_rows(ctx)) return SPX_ERR_UNSUPPORTED;
    if (!A->batch1 || (mixed && !A->batch1_shadow)) {
        if (A->batch1) spx_batch_destroy(A->batch1);
        A->batch1 = nullptr;
        const int64_t ro[2] = {0, A->n}, no[2] = {0, A->nnz};
        SPX_TRY(spx_batch_create(A->ctx, &A->batch1, A->dtype, 1, ro, no, A->rp.as<int32_t>(), A->col.as<int32_t>(),
                                 A->val.p, mixed ? SPX_MIXED_SHADOW : 0u));
        A->batch1_shadow = mixed;
        SPX_CUDA(cudaStreamSynchronize(A->ctx->stream));  // ready for any context's stream
    }
    const int block = A->n <= 2048 ? 256 : A->n <= 8192 ? 512 : 1024;
    spx_solve_info one;
    SPX_TRY(batch_solve_direct(ctx, A->batch1, b, x, solver, tol, maxit, precision, block, &one));
    *info = one;
    return SPX_OK;
}

int solve_entry(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, int solver, double tol, int64_t maxit,
                int restart, int precision, int64_t fixed, spx_solve_info *info)
{
    if (!ctx || !A || !info || (A->n > 0 && (!b || !x)))
        return fail(SPX_ERR_INVALID, "spx_solve: NULL argument");
    std::memset(info, 0, sizeof(*info));
    if (A->n != A->ncols) return fail(SPX_ERR_INVALID, "spx_solve: the matrix must be square");
    bool pre = false, adapt = false;
    int bs = 0;
    const bool one_cluster = (solver & SPX_SOLVE_ONE_CLUSTER) != 0;
    SPX_TRY(parse_solver_code(solver & ~SPX_SOLVE_ONE_CLUSTER, &solver, &pre, &bs, &adapt));
    if (!(tol >= 0.0) || maxit < 0) return fail(SPX_ERR_INVALID, "spx_solve: bad tol or max_iter");
    if (solver == SPX_GMRES && (restart < 1 || restart > kGmKmax - 1))
        return fail(SPX_ERR_UNSUPPORTED, "GMRES restart length must be in [1, 31]");
    if (A->n == 0) {
        info->status = SPX_CONVERGED;
        return SPX_OK;
    }
    Timer tm;
    int st;
    if (one_cluster) {
        if (fixed != 0 || pre || bs != 0 || solver == SPX_GMRES)
            return fail(SPX_ERR_UNSUPPORTED, "the one-cluster solve runs CG, BiCGSTAB or CGS to a tolerance, "
                                             "without preconditioner");
        st = cluster_solve(ctx, A, b, x, solver, tol, maxit, precision, info);
        info->time_ms = tm.ms();
        return st;
    }
    if (fixed == 0 && !pre && bs == 0 && solver != SPX_GMRES && A->format == SPX_CSR && A->n <= kSmallSolveRows &&
        A->rp.p && A->kernel == SPX_KERNEL_AUTO) {  // a pinned SpMV kernel keeps the general path
        st = small_solve(ctx, A, b, x, solver, tol, maxit, precision, info);
        if (st != SPX_ERR_UNSUPPORTED) {
            info->time_ms = tm.ms();
            return st;
        }
    }
    if (precision == SPX_PREC_MIXED) {
        if (A->dtype != SPX_F64 || !(A->val32.p || A->ell_val32.p || A->coo_val32.p))
            return fail(SPX_ERR_UNSUPPORTED, "mixed precision needs an FP64 matrix created with SPX_MIXED_SHADOW");
        if (fixed > 0) return fail(SPX_ERR_UNSUPPORTED, "fixed-iteration mode runs in one precision");
        st = run_ir(ctx, A, static_cast<const double *>(b), static_cast<double *>(x), solver, tol, maxit, restart, pre,
                    bs, adapt, info);
    } else if (precision == SPX_PREC_F64 || precision == SPX_PREC_F32) {
        const int want = precision == SPX_PREC_F64 ? SPX_F64 : SPX_F32;
        if (A->dtype != want) return fail(SPX_ERR_UNSUPPORTED, "precision must match the matrix dtype (or use MIXED)");
        st = A->dtype == SPX_F64
                 ? solve_typed<double>(ctx, A, static_cast<const double *>(b), static_cast<double *>(x), solver, tol,
                                       maxit, restart, false, fixed, pre, bs, adapt, info)
                 : solve_typed<float>(ctx, A, static_cast<const float *>(b), static_cast<float *>(x), solver, tol,
                                      maxit, restart, false, fixed, pre, bs, adapt, info);
    } else {
        return fail(SPX_ERR_INVALID, "spx_solve: unknown precision");
    }
    info->time_ms = tm.ms();
    return st;
}

}  // namespace
}  // namespace spx

using namespace spx;

namespace {
struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
        else prev = -1;
    }
    ~DevGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
}  // namespace

extern "C" int spx_solve(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, int solver, double tol,
                         int64_t max_iter, int restart, int precision, spx_solve_info *info)
{
    if (!ctx) return fail(SPX_ERR_INVALID, "spx_solve: ctx is NULL");
    DevGuard g(ctx->device);
    const int st = solve_entry(ctx, A, b, x, solver, tol, max_iter, restart, precision, 0, info);
    if (A) ++A->solves;
    return st;
}

extern "C" int spx_solve_fixed(spx_ctx *ctx, spx_matrix *A, const void *b, void *x, int solver, int64_t iterations,
                               int restart, int precision, spx_solve_info *info)
{
    if (!ctx) return fail(SPX_ERR_INVALID, "spx_solve_fixed: ctx is NULL");
    if (iterations < 1) return fail(SPX_ERR_INVALID, "spx_solve_fixed: iterations must be >= 1");
    DevGuard g(ctx->device);
    const int st = solve_entry(ctx, A, b, x, solver, 0.0, iterations, restart, precision, iterations, info);
    if (A) ++A->solves;
    return st;
}
