/*
 * spx_oracle.c -- plain, sequential CPU oracle for the sparse hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library product links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no source, header, table or helper with the
 * CUDA path.
 *
 * What it computes (all in IEEE double unless a function says otherwise):
 *   - sparse matrix-vector product y = A x for a CSR matrix, summed in index
 *     order (Section 5 defines SpMV and the CSR / COO layouts);
 *   - the storage conversions CSR -> COO, ELL, HYB as plain byte copies;
 *   - textbook CG, BiCGSTAB, CGS and restarted GMRES(m) with modified
 *     Gram-Schmidt and Givens rotations (the Krylov methods Section 5 names, in
 *     the form of the textbooks it cites), each also with Jacobi or
 *     block-Jacobi preconditioning (preconditioned CG; right preconditioning
 *     for the others; block inverses by Gauss-Jordan with partial pivoting,
 *     optionally stored in FP32 for well-conditioned blocks);
 *   - iterative refinement with an FP32 inner Krylov solve and FP64 outer
 *     residual and update, and CG with FP32 iterations and FP64 residual
 *     replacement ("reliable updates": the Krylov space is kept).
 *
 * Build flags must keep IEEE semantics: -O2 -ffp-contract=off, no fast-math,
 * so that x86-64 and aarch64 hosts produce identical bits.  A second build with
 * -DORC_OPENMP -fopenmp (same arithmetic) times the plain SpMV on all host cores
 * for the CPU baseline.
 *
 * Pins (the tests in tests/test_oracle_*.py) tie every function here to facts
 * that do not come from this file: exact dense products on integer data,
 * closed-form Laplacian eigenpairs, finite termination of CG / GMRES, one-step
 * convergence on scaled identities, and hand-worked examples.  Iterative
 * refinement is pinned cycle by cycle on scaled identities c*I (c a power of
 * two), where FP32 rounding bounds fix each cycle's error: 2^-24 after one,
 * 2^-47 after two.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* A planted mistake for the mutation tests: tests rebuild this file with
 * -DORC_MUTANT=<k> and check that the pins catch it.  0 = correct oracle. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

enum { ORC_CONVERGED = 0, ORC_MAX_ITER = 1, ORC_BREAKDOWN = 2, ORC_STAGNATED = 3 };
enum { ORC_OK = 0, ORC_INVALID = 1 };

typedef struct {
    int32_t status;
    int32_t restarts;
    int64_t iterations;
    double relres_recurrence;
    double relres_true;
} orc_info;

/* ------------------------------------------------------------------------- */
/* CSR validation (a CSR matrix: row_ptr[0] = 0, non-decreasing,             */
/* row_ptr[n] = nnz, 0 <= col < ncols).  Duplicates, unsorted columns and    */
/* explicit zeros are legal.                                                 */
/* ------------------------------------------------------------------------- */
int orc_csr_check(int64_t n, int64_t ncols, int64_t nnz, const int32_t *rp, const int32_t *col)
{
    if (n < 0 || ncols < 0 || nnz < 0) return ORC_INVALID;
    if (rp[0] != 0 || (int64_t)rp[n] != nnz) return ORC_INVALID;
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return ORC_INVALID;
    for (int64_t k = 0; k < nnz; ++k)
        if (col[k] < 0 || (int64_t)col[k] >= ncols) return ORC_INVALID;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* SpMV, Section 5: y_i = sum_{k = rp[i]}^{rp[i+1]-1} val[k] * x[col[k]].     */
/* Each product is formed in double and the row sum is accumulated in index  */
/* order with Neumaier's compensated summation, so the reference itself is   */
/* accurate to about one rounding of the exact sum.                          */
/* ------------------------------------------------------------------------- */
void orc_spmv_csr(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                  const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0, c = 0.0;
        int64_t lo = rp[i], hi = rp[i + 1];
#if ORC_MUTANT == 2
        hi = hi > lo ? hi - 1 : hi; /* planted: drop the last term of each row */
#endif
        for (int64_t k = lo; k < hi; ++k) {
#if ORC_MUTANT == 1
            double p = val[k] * x[i + 0 * col[k]] ; /* planted: wrong operand index */
#else
            double p = val[k] * x[col[k]];
#endif
            double t = s + p;
            if (fabs(s) >= fabs(p)) c += (s - t) + p;
            else                    c += (p - t) + s;
            s = t;
        }
        y[i] = s + c;
    }
}

/* (|A| |x|)_i, the scale of the rounding error of row i of any summation order. */
void orc_spmv_csr_absbound(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                           const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
#if ORC_MUTANT == 13
            s += fabs(val[k]) * fabs(x[i + 0 * col[k]]); /* planted: wrong operand index */
#else
            s += fabs(val[k]) * fabs(x[col[k]]);
#endif
        }
#if ORC_MUTANT == 12
        s *= 2.0; /* planted: an inflated bound */
#endif
        y[i] = s;
    }
}

/* Plain index-order SpMV without compensation, the literal definition.  Used
 * only by the CPU-baseline timing and the fixed-iteration solver loops.  In the
 * build with -DORC_OPENMP (the all-cores CPU baseline) rows are shared among
 * threads; each row is still summed alone, in index order, so the result is
 * the same bits. */
static void spmv_plain(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                       const double *x, double *y)
{
#ifdef ORC_OPENMP
#pragma omp parallel for schedule(static, 1024)
#endif
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += val[k] * x[col[k]];
        y[i] = s;
    }
}

void orc_spmv_csr_plain(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                        const double *x, double *y)
{
    spmv_plain(n, rp, col, val, x, y);
}

/* ------------------------------------------------------------------------- */
/* Storage conversions (Section 5 defines COO as CSR with explicit row       */
/* indices; ELL and HYB are storage orders of the same entries).  All are    */
/* byte copies: value bytes are copied unchanged (vbytes = 8 or 4).          */
/* ------------------------------------------------------------------------- */

/* COO row indices: row[k] = i for k in [rp[i], rp[i+1]); col/val unchanged. */
void orc_csr_to_coo_rows(int64_t n, const int32_t *rp, int32_t *row)
{
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) row[k] = (int32_t)i;
}

/* Maximum row length = ELL width. */
int64_t orc_max_row_len(int64_t n, const int32_t *rp)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t l = (int64_t)rp[i + 1] - rp[i];
        if (l > m) m = l;
    }
    return m;
}

/* ELL of width k, column-major with leading dimension ld >= n: slot (i, j)
 * sits at j*ld + i.  The first min(len_i, k) entries of row i fill slots
 * j = 0.. in CSR order; the remaining slots (and rows n..ld-1) are padding
 * with col = -1 and value bytes all zero (+0.0). */
void orc_csr_to_ell(int64_t n, int64_t ld, int64_t k, const int32_t *rp, const int32_t *col,
                    const void *val, int vbytes, int32_t *ell_col, void *ell_val)
{
    const unsigned char *v = (const unsigned char *)val;
    unsigned char *ev = (unsigned char *)ell_val;
    for (int64_t j = 0; j < k; ++j)
        for (int64_t i = 0; i < ld; ++i) {
            int64_t slot = j * ld + i;
            int64_t len = i < n ? (int64_t)rp[i + 1] - rp[i] : 0;
            if (j < len) {
                ell_col[slot] = col[rp[i] + j];
                memcpy(ev + slot * vbytes, v + ((int64_t)rp[i] + j) * vbytes, (size_t)vbytes);
            } else {
                ell_col[slot] = -1;
                memset(ev + slot * vbytes, 0, (size_t)vbytes);
            }
        }
}

/* Number of entries that spill out of an ELL part of width k. */
int64_t orc_hyb_coo_count(int64_t n, const int32_t *rp, int64_t k)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t l = (int64_t)rp[i + 1] - rp[i];
        if (l > k) c += l - k;
    }
    return c;
}

/* HYB: ELL part of width k as above, plus a COO part that holds, in CSR
 * order, entries k.. of every row longer than k. */
void orc_csr_to_hyb(int64_t n, int64_t ld, int64_t k, const int32_t *rp, const int32_t *col,
                    const void *val, int vbytes, int32_t *ell_col, void *ell_val,
                    int32_t *coo_row, int32_t *coo_col, void *coo_val)
{
    const unsigned char *v = (const unsigned char *)val;
    unsigned char *cv = (unsigned char *)coo_val;
    orc_csr_to_ell(n, ld, k, rp, col, val, vbytes, ell_col, ell_val);
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = (int64_t)rp[i] + k; e < rp[i + 1]; ++e) {
            coo_row[c] = (int32_t)i;
            coo_col[c] = col[e];
            memcpy(cv + c * vbytes, v + e * vbytes, (size_t)vbytes);
            ++c;
        }
}

/* Footprint-optimal HYB width: bytes(k) = (V+4) k n + (V+8) sum_i max(0, len_i - k).
 * Raising k by one changes bytes by (V+4) n - (V+8) #{i : len_i > k}; take the
 * smallest k at which that change is no longer negative. */
int64_t orc_hyb_auto_width(int64_t n, const int32_t *rp, int vbytes)
{
    int64_t kmax = orc_max_row_len(n, rp);
    for (int64_t k = 0; k <= kmax; ++k) {
        int64_t longer = 0;
        for (int64_t i = 0; i < n; ++i)
            if ((int64_t)rp[i + 1] - rp[i] > k) ++longer;
        if ((int64_t)(vbytes + 8) * longer <= (int64_t)(vbytes + 4) * n) return k;
    }
    return kmax;
}

/* ------------------------------------------------------------------------- */
/* Vector helpers (double).                                                  */
/* ------------------------------------------------------------------------- */
static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}
static double nrm2(int64_t n, const double *a) { return sqrt(dot(n, a, a)); }

static double true_relres(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                          const double *b, const double *x, double bnorm, double *work)
{
    orc_spmv_csr(n, rp, col, val, x, work);
    for (int64_t i = 0; i < n; ++i) work[i] = b[i] - work[i];
    return nrm2(n, work) / bnorm;
}

/* Convergence and exit policy shared by every solver below (the paper leaves
 * it open): the recurrence residual is tested each iteration; at exit the true
 * residual ||b - A x|| / ||b|| is formed; if it is above tol the method
 * restarts from the current x, at most ORC_MAX_RESTARTS times, after which the
 * status is STAGNATED.  b = 0 gives x = 0 in zero iterations. */
#define ORC_MAX_RESTARTS 3

/* ------------------------------------------------------------------------- */
/* A preconditioner M^{-1} given as the inverses of the diagonal blocks of A: */
/* block k covers rows and columns [k bs, (k+1) bs) (the last one clipped to */
/* n); minv holds each block's bs x bs inverse row-major.  bs = 1 is Jacobi, */
/* minv[i] = 1 / a_ii.  out = M^{-1} in, each row summed in column order.    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int bs;
    const double *minv;
} orc_prec;

static void prec_apply(const orc_prec *M, int64_t n, const double *in, double *out)
{
    if (M->bs == 1) {
        for (int64_t i = 0; i < n; ++i) out[i] = M->minv[i] * in[i];
        return;
    }
    const int64_t bs = M->bs;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t k = i / bs, r = i % bs, c0 = k * bs;
        const double *row = M->minv + (size_t)(k * bs + r) * (size_t)bs;
        double s = 0.0;
#if ORC_MUTANT == 8
        for (int64_t j = 0; j < bs && c0 + j < n; ++j) /* planted: the block's transpose */
            s += M->minv[(size_t)(k * bs + j) * (size_t)bs + (size_t)r] * in[c0 + j];
        (void)row;
#else
        for (int64_t j = 0; j < bs && c0 + j < n; ++j) s += row[j] * in[c0 + j];
#endif
        out[i] = s;
    }
}

/* ------------------------------------------------------------------------- */
/* CG (Hestenes-Stiefel) for symmetric positive definite A.                  */
/*   r = b - A x, p = r, rho = r.r                                           */
/*   loop: q = A p; alpha = rho / (p.q); x += alpha p; r -= alpha q;         */
/*         rho' = r.r; stop if sqrt(rho')/||b|| <= tol;                      */
/*         beta = rho'/rho; p = r + beta p; rho = rho'                        */
/* hist (optional) receives the recurrence relative residual after every     */
/* iteration, hist[0] being the initial one.                                 */
/* ------------------------------------------------------------------------- */
static int cg_run(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                  const double *b, double *x, double tol, int64_t maxit, orc_info *info, double *hist,
                  const orc_prec *M)
{
    memset(info, 0, sizeof(*info));
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        memset(x, 0, (size_t)n * sizeof(double));
        info->status = ORC_CONVERGED;
        return 0;
    }
    double *r = malloc((size_t)n * sizeof(double)), *p = malloc((size_t)n * sizeof(double));
    double *q = malloc((size_t)n * sizeof(double));
    double *z = M ? malloc((size_t)n * sizeof(double)) : NULL; /* z = M^{-1} r */
    int64_t it = 0;
    int status = ORC_MAX_ITER;
    double rel = 0.0, reltrue = 0.0;
    for (int restart = 0;; ++restart) {
        orc_spmv_csr(n, rp, col, val, x, q);
        for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
        if (M) {
            prec_apply(M, n, r, z);
            for (int64_t i = 0; i < n; ++i) p[i] = z[i];
        }
        double rr = dot(n, r, r);
        double rho = M ? dot(n, r, z) : rr;
        rel = sqrt(rr) / bnorm;
        if (hist && it == 0) hist[0] = rel;
        status = ORC_MAX_ITER;
        if (rel <= tol) status = ORC_CONVERGED;
        while (status == ORC_MAX_ITER && it < maxit) {
            orc_spmv_csr(n, rp, col, val, p, q);
            double pq = dot(n, p, q);
            if (pq == 0.0) { status = ORC_BREAKDOWN; break; }
            double alpha = rho / pq;
            for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
            double rr1 = dot(n, r, r);
            ++it;
            rel = sqrt(rr1) / bnorm;
            if (hist) hist[it] = rel;
            if (rel <= tol) { status = ORC_CONVERGED; break; }
            if (M) prec_apply(M, n, r, z);
            double rho1 = M ? dot(n, r, z) : rr1;
#if ORC_MUTANT == 3
            double beta = -rho1 / rho; /* planted: wrong sign */
#else
            double beta = rho1 / rho;
#endif
            const double *zr = M ? z : r;
            for (int64_t i = 0; i < n; ++i) p[i] = zr[i] + beta * p[i];
            rho = rho1;
        }
        reltrue = true_relres(n, rp, col, val, b, x, bnorm, q);
        info->restarts = restart;
        if (status != ORC_CONVERGED || reltrue <= tol) break;
        if (restart == ORC_MAX_RESTARTS) { status = ORC_STAGNATED; break; }
    }
    info->status = status;
    info->iterations = it;
    info->relres_recurrence = rel;
    info->relres_true = reltrue;
    free(r); free(p); free(q); free(z);
    return 0;
}

int orc_cg(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
           const double *b, double *x, double tol, int64_t maxit, orc_info *info, double *hist)
{
    return cg_run(n, rp, col, val, b, x, tol, maxit, info, hist, NULL);
}



/* ------------------------------------------------------------------------- */
/* BiCGSTAB (van der Vorst) for general A, shadow residual r^ = r0.          */
/*   rho = alpha = omega = 1, v = p = 0                                      */
/*   loop: rho' = r^.r; beta = (rho'/rho)(alpha/omega);                      */
/*         p = r + beta (p - omega v); v = A p; alpha = rho' / (r^.v);       */
/*         s = r - alpha v; if ||s||/||b|| <= tol: x += alpha p, stop;       */
/*         t = A s; omega = (t.s)/(t.t); x += alpha p + omega s;             */
/*         r = s - omega t; stop if ||r||/||b|| <= tol; rho = rho'            */
/* Breakdown when rho' = 0, r^.v = 0 or t.t = 0.                             */
/* ------------------------------------------------------------------------- */
static int bicgstab_run(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                        const double *b, double *x, double tol, int64_t maxit, orc_info *info,
                        double *hist, const orc_prec *M)
{
    memset(info, 0, sizeof(*info));
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        memset(x, 0, (size_t)n * sizeof(double));
        return 0;
    }
    size_t bytes = (size_t)n * sizeof(double);
    double *r = malloc(bytes), *rh = malloc(bytes), *p = malloc(bytes), *v = malloc(bytes);
    double *s = malloc(bytes), *t = malloc(bytes);
    double *ph = M ? malloc(bytes) : NULL, *sh = M ? malloc(bytes) : NULL; /* M^{-1} p, M^{-1} s */
    if (!M) { ph = p; sh = s; }
    int64_t it = 0;
    int status = ORC_MAX_ITER;
    double rel = 0.0, reltrue = 0.0;
    for (int restart = 0;; ++restart) {
        orc_spmv_csr(n, rp, col, val, x, t);
        for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - t[i]; rh[i] = r[i]; p[i] = 0.0; v[i] = 0.0; }
        double rho = 1.0, alpha = 1.0, omega = 1.0;
        rel = nrm2(n, r) / bnorm;
        if (hist && it == 0) hist[0] = rel;
        status = rel <= tol ? ORC_CONVERGED : ORC_MAX_ITER;
        while (status == ORC_MAX_ITER && it < maxit) {
            double rho1 = dot(n, rh, r);
            if (rho1 == 0.0) { status = ORC_BREAKDOWN; break; }
            double beta = (rho1 / rho) * (alpha / omega);
            for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            if (M) prec_apply(M, n, p, ph);
            orc_spmv_csr(n, rp, col, val, ph, v);
            double rv = dot(n, rh, v);
            if (rv == 0.0) { status = ORC_BREAKDOWN; break; }
            alpha = rho1 / rv;
            for (int64_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
            ++it;
            double snorm = nrm2(n, s);
            if (snorm / bnorm <= tol) {
                for (int64_t i = 0; i < n; ++i) x[i] += alpha * ph[i];
                for (int64_t i = 0; i < n; ++i) r[i] = s[i];
                rel = snorm / bnorm;
                if (hist) hist[it] = rel;
                status = ORC_CONVERGED;
                break;
            }
            if (M) prec_apply(M, n, s, sh);
            orc_spmv_csr(n, rp, col, val, sh, t);
            double tt = dot(n, t, t);
            if (tt == 0.0) { status = ORC_BREAKDOWN; break; }
            omega = dot(n, t, s) / tt;
#if ORC_MUTANT == 4
            for (int64_t i = 0; i < n; ++i) x[i] += alpha * ph[i] - omega * sh[i]; /* planted */
#elif ORC_MUTANT == 7
            for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i] + omega * sh[i]; /* planted: p for M^{-1} p */
#else
            for (int64_t i = 0; i < n; ++i) x[i] += alpha * ph[i] + omega * sh[i];
#endif
            for (int64_t i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
            rel = nrm2(n, r) / bnorm;
            if (hist) hist[it] = rel;
            if (rel <= tol) { status = ORC_CONVERGED; break; }
            if (omega == 0.0) { status = ORC_BREAKDOWN; break; }
            rho = rho1;
        }
        reltrue = true_relres(n, rp, col, val, b, x, bnorm, t);
        info->restarts = restart;
        if (status != ORC_CONVERGED || reltrue <= tol) break;
        if (restart == ORC_MAX_RESTARTS) { status = ORC_STAGNATED; break; }
    }
    info->status = status;
    info->iterations = it;
    info->relres_recurrence = rel;
    info->relres_true = reltrue;
    if (M) { free(ph); free(sh); }
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return 0;
}

int orc_bicgstab(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                 const double *b, double *x, double tol, int64_t maxit, orc_info *info,
                 double *hist)
{
    return bicgstab_run(n, rp, col, val, b, x, tol, maxit, info, hist, NULL);
}



/* ------------------------------------------------------------------------- */
/* CGS, Sonneveld's conjugate gradient squared method (the fourth Krylov     */
/* solver Section 5 lists), in the textbook form (Saad, Iterative Methods,   */
/* section 7.4.1): shadow residual r^ = r0, p = u = r0; each iteration       */
/*   alpha = (r, r^) / (A p, r^);  q = u - alpha A p;                         */
/*   x += alpha (u + q);  r -= alpha A (u + q);                               */
/*   beta = (r_new, r^) / (r, r^);  u = r + beta q;  p = u + beta (q + beta p). */
/* Two SpMVs per iteration.  Breakdown when (A p, r^) or (r, r^) is exactly 0. */
/* ------------------------------------------------------------------------- */
static int cgs_run(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                   const double *b, double *x, double tol, int64_t maxit, orc_info *info, double *hist,
                   const orc_prec *M)
{
    memset(info, 0, sizeof(*info));
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        memset(x, 0, (size_t)n * sizeof(double));
        return 0;
    }
    size_t bytes = (size_t)n * sizeof(double);
    double *r = malloc(bytes), *rh = malloc(bytes), *p = malloc(bytes), *u = malloc(bytes);
    double *q = malloc(bytes), *v = malloc(bytes), *w = malloc(bytes);
    double *ph = M ? malloc(bytes) : p;  /* M^{-1} p, and M^{-1} (u + q) on its way into w */
    int64_t it = 0;
    int status = ORC_MAX_ITER;
    double rel = 0.0, reltrue = 0.0;
    for (int restart = 0;; ++restart) {
        orc_spmv_csr(n, rp, col, val, x, v);
        for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - v[i]; rh[i] = r[i]; p[i] = r[i]; u[i] = r[i]; }
        double rho = dot(n, rh, r);
        rel = nrm2(n, r) / bnorm;
        if (hist && it == 0) hist[0] = rel;
        status = rel <= tol ? ORC_CONVERGED : ORC_MAX_ITER;
        while (status == ORC_MAX_ITER && it < maxit) {
            if (rho == 0.0) { status = ORC_BREAKDOWN; break; }
            if (M) prec_apply(M, n, p, ph);
            orc_spmv_csr(n, rp, col, val, ph, v);                      /* v = A M^{-1} p */
            double vr = dot(n, rh, v);
            if (vr == 0.0) { status = ORC_BREAKDOWN; break; }
            double alpha = rho / vr;
            for (int64_t i = 0; i < n; ++i) q[i] = u[i] - alpha * v[i];
            for (int64_t i = 0; i < n; ++i) w[i] = u[i] + q[i];      /* u + q */
            if (M) {                                                    /* M^{-1} (u + q) */
                prec_apply(M, n, w, ph);
                for (int64_t i = 0; i < n; ++i) w[i] = ph[i];
            }
            for (int64_t i = 0; i < n; ++i) x[i] += alpha * w[i];
            orc_spmv_csr(n, rp, col, val, w, v);                       /* A (u + q) */
#if ORC_MUTANT == 6
            for (int64_t i = 0; i < n; ++i) r[i] += alpha * v[i];     /* planted: wrong sign */
#else
            for (int64_t i = 0; i < n; ++i) r[i] -= alpha * v[i];
#endif
            ++it;
            rel = nrm2(n, r) / bnorm;
            if (hist) hist[it] = rel;
            if (rel <= tol) { status = ORC_CONVERGED; break; }
            double rho1 = dot(n, rh, r);
            double beta = rho1 / rho;
            for (int64_t i = 0; i < n; ++i) u[i] = r[i] + beta * q[i];
            for (int64_t i = 0; i < n; ++i) p[i] = u[i] + beta * (q[i] + beta * p[i]);
            rho = rho1;
        }
        reltrue = true_relres(n, rp, col, val, b, x, bnorm, v);
        info->restarts = restart;
        if (status != ORC_CONVERGED || reltrue <= tol) break;
        if (restart == ORC_MAX_RESTARTS) { status = ORC_STAGNATED; break; }
    }
    info->status = status;
    info->iterations = it;
    info->relres_recurrence = rel;
    info->relres_true = reltrue;
    if (M) free(ph);
    free(r); free(rh); free(p); free(u); free(q); free(v); free(w);
    return 0;
}

int orc_cgs(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
            const double *b, double *x, double tol, int64_t maxit, orc_info *info, double *hist)
{
    return cgs_run(n, rp, col, val, b, x, tol, maxit, info, hist, NULL);
}



/* ------------------------------------------------------------------------- */
/* Restarted GMRES(m) (Saad & Schultz): Arnoldi with modified Gram-Schmidt,  */
/* Givens rotations applied to the Hessenberg column as it is formed, the    */
/* residual estimate |g_{j+1}|, and at the end of each cycle x += V_j y_j    */
/* where H_j y_j = g_j is solved by back substitution.  One iteration = one  */
/* Arnoldi step (one SpMV).                                                  */
/* ------------------------------------------------------------------------- */
static int gmres_run(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                     const double *b, double *x, int m, double tol, int64_t maxit, orc_info *info,
                     double *hist, const orc_prec *M)
{
    memset(info, 0, sizeof(*info));
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        memset(x, 0, (size_t)n * sizeof(double));
        return 0;
    }
    size_t bytes = (size_t)n * sizeof(double);
    double *V = malloc(bytes * (size_t)(m + 1));
    double *w = malloc(bytes);
    double *z = M ? malloc(bytes) : NULL; /* M^{-1} v_j, and the cycle's update */
    double *H = calloc((size_t)(m + 1) * m, sizeof(double)); /* H[i*m + j] */
    double *cs = malloc(sizeof(double) * m), *sn = malloc(sizeof(double) * m);
    double *g = malloc(sizeof(double) * (m + 1)), *yv = malloc(sizeof(double) * m);
    int64_t it = 0;
    int status = ORC_MAX_ITER;
    double rel = 0.0, reltrue = 0.0;
    int cycles = 0;
    for (;;) {
        /* r = b - A x */
        orc_spmv_csr(n, rp, col, val, x, w);
        for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
        double beta = nrm2(n, w);
        rel = beta / bnorm;
        if (hist && it == 0) hist[0] = rel;
        if (rel <= tol) {
            reltrue = rel;
            status = ORC_CONVERGED;
            break;
        }
        if (it >= maxit) { reltrue = rel; status = ORC_MAX_ITER; break; }
        for (int64_t i = 0; i < n; ++i) V[i] = w[i] / beta;
        memset(g, 0, sizeof(double) * (m + 1));
        g[0] = beta;
        int j = 0, done = 0;
        for (; j < m && it < maxit; ++j) {
            double *vj = V + (size_t)j * n;
            if (M) {
                prec_apply(M, n, vj, z);
                orc_spmv_csr(n, rp, col, val, z, w);   /* w = A M^{-1} v_j */
            } else {
                orc_spmv_csr(n, rp, col, val, vj, w);
            }
            for (int i = 0; i <= j; ++i) {
                double *vi = V + (size_t)i * n;
                double h = dot(n, w, vi);
                H[i * m + j] = h;
                for (int64_t k = 0; k < n; ++k) w[k] -= h * vi[k];
            }
            double hn = nrm2(n, w);
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0) {
                double *vn = V + (size_t)(j + 1) * n;
                for (int64_t k = 0; k < n; ++k) vn[k] = w[k] / hn;
            }
            /* previous rotations on column j */
            for (int i = 0; i < j; ++i) {
                double a = H[i * m + j], c = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            /* new rotation zeroing H[j+1][j] */
            double a = H[j * m + j], c = H[(j + 1) * m + j];
            double d = hypot(a, c);
            cs[j] = d == 0.0 ? 1.0 : a / d;
            sn[j] = d == 0.0 ? 0.0 : c / d;
            H[j * m + j] = d;
            H[(j + 1) * m + j] = 0.0;
#if ORC_MUTANT == 5
            g[j + 1] = sn[j] * g[j]; /* planted: wrong sign (harmless to |g|), and */
            g[j] = -cs[j] * g[j];    /* wrong sign on the kept component */
#else
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
#endif
            ++it;
            rel = fabs(g[j + 1]) / bnorm;
            if (hist) hist[it] = rel;
            if (rel <= tol || hn == 0.0) { done = 1; ++j; break; }
        }
        /* back substitution H[0..j-1][0..j-1] y = g[0..j-1] */
        for (int i = j - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < j; ++k) s -= H[i * m + k] * yv[k];
            yv[i] = s / H[i * m + i];
        }
        if (M) {  /* x += M^{-1} V y */
            memset(z, 0, bytes);
            for (int i = 0; i < j; ++i) {
                double *vi = V + (size_t)i * n;
                for (int64_t k = 0; k < n; ++k) z[k] += yv[i] * vi[k];
            }
            prec_apply(M, n, z, w);
            for (int64_t k = 0; k < n; ++k) x[k] += w[k];
        } else {
            for (int i = 0; i < j; ++i) {
                double *vi = V + (size_t)i * n;
                for (int64_t k = 0; k < n; ++k) x[k] += yv[i] * vi[k];
            }
        }
        ++cycles;
        if (done) {
            reltrue = true_relres(n, rp, col, val, b, x, bnorm, w);
            if (reltrue <= tol) { status = ORC_CONVERGED; break; }
            /* the estimate said converged but the true residual did not:
             * continue with a fresh cycle, which counts as a restart. */
            if (info->restarts == ORC_MAX_RESTARTS) { status = ORC_STAGNATED; break; }
            info->restarts++;
        } else if (it >= maxit) {
            reltrue = true_relres(n, rp, col, val, b, x, bnorm, w);
            status = reltrue <= tol ? ORC_CONVERGED : ORC_MAX_ITER;
            break;
        }
    }
    info->status = status;
    info->iterations = it;
    info->relres_recurrence = rel;
    info->relres_true = reltrue;
    (void)cycles;
    free(V); free(w); free(H); free(cs); free(sn); free(g); free(yv);
    free(z);
    return 0;
}

int orc_gmres(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
              const double *b, double *x, int m, double tol, int64_t maxit, orc_info *info,
              double *hist)
{
    return gmres_run(n, rp, col, val, b, x, m, tol, maxit, info, hist, NULL);
}

/* ------------------------------------------------------------------------- */
/* Jacobi preconditioning, M = diag(A) (a zero diagonal entry is taken as 1; */
/* duplicate diagonal entries are summed in index order).  CG: the textbook  */
/* preconditioned CG, z = M^{-1} r, convergence on ||r||.  BiCGSTAB, CGS and */
/* GMRES: right preconditioning, the method runs on A M^{-1} and x gathers  */
/* M^{-1} times its search directions, so r stays the true residual.        */
/* ------------------------------------------------------------------------- */
static double *jacobi_dinv(int64_t n, const int32_t *rp, const int32_t *col, const double *val)
{
    double *d = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] == i) s += val[k];
        d[i] = s != 0.0 ? 1.0 / s : 1.0;
    }
    return d;
}

int orc_cg_jacobi(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                  const double *b, double *x, double tol, int64_t maxit, orc_info *info, double *hist)
{
    double *d = jacobi_dinv(n, rp, col, val);
    orc_prec M = {1, d};
    int st = cg_run(n, rp, col, val, b, x, tol, maxit, info, hist, &M);
    free(d);
    return st;
}

int orc_bicgstab_jacobi(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                        const double *b, double *x, double tol, int64_t maxit, orc_info *info, double *hist)
{
    double *d = jacobi_dinv(n, rp, col, val);
    orc_prec M = {1, d};
    int st = bicgstab_run(n, rp, col, val, b, x, tol, maxit, info, hist, &M);
    free(d);
    return st;
}

int orc_cgs_jacobi(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                   const double *b, double *x, double tol, int64_t maxit, orc_info *info, double *hist)
{
    double *d = jacobi_dinv(n, rp, col, val);
    orc_prec M = {1, d};
    int st = cgs_run(n, rp, col, val, b, x, tol, maxit, info, hist, &M);
    free(d);
    return st;
}

int orc_gmres_jacobi(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                     const double *b, double *x, int m, double tol, int64_t maxit, orc_info *info,
                     double *hist)
{
    double *d = jacobi_dinv(n, rp, col, val);
    orc_prec M = {1, d};
    int st = gmres_run(n, rp, col, val, b, x, m, tol, maxit, info, hist, &M);
    free(d);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Block-Jacobi preconditioning, M = the block diagonal of A with blocks of  */
/* bs consecutive rows and columns (Section 2 lists block-Jacobi, in its    */
/* adaptive-precision form, among the library's preconditioners; here the   */
/* inverses are kept at the solve's precision).  Block k's dense matrix D_k  */
/* gathers the entries of rows [k bs, (k+1) bs) whose columns fall in the    */
/* same range (duplicates summed in index order); rows past n are identity  */
/* rows.  D_k^{-1} by Gauss-Jordan elimination on [D_k | I] with partial     */
/* pivoting (the largest |entry| of the pivot column at or below the        */
/* diagonal, the first one on ties): swap, scale the pivot row by the       */
/* reciprocal of the pivot, subtract multiples of it from every other row.  */
/* A block with an exactly zero pivot is taken as the identity, as Jacobi   */
/* takes a zero diagonal as 1.  bs = 1 gives exactly Jacobi's 1 / a_ii.     */
/* ------------------------------------------------------------------------- */
/* Adaptive storage (flags != NULL): each block's inverse is kept in FP32    */
/* when its 1-norm condition number kappa = ||D_k||_1 ||D_k^{-1}||_1 times   */
/* the FP32 unit roundoff 2^-24 is at most 1e-2, so that the rounded        */
/* inverse differs from the exact one by at most 1% of the identity in the  */
/* preconditioned block, and every nonzero entry lies in FP32's normal      */
/* range; otherwise in FP64.  The FP32 entries are returned as the doubles  */
/* they round to; flags[k] = 1 marks an FP64 block.                         */
#define ORC_BJ_FP32_BOUND 1e-2

static int block_jacobi_inv_impl(int64_t n, const int32_t *rp, const int32_t *col, const double *val, int bs,
                                 double *minv, unsigned char *flags)
{
    if (bs < 1) return -1;
    const int64_t nb = (n + bs - 1) / bs;
    double *aug = malloc(sizeof(double) * (size_t)bs * (size_t)(2 * bs));
    for (int64_t k = 0; k < nb; ++k) {
        const int64_t c0 = k * bs;
        const int w = 2 * bs;
        memset(aug, 0, sizeof(double) * (size_t)bs * (size_t)w);
        for (int r = 0; r < bs; ++r) {
            const int64_t i = c0 + r;
            aug[r * w + bs + r] = 1.0;
            if (i >= n) { aug[r * w + r] = 1.0; continue; }
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
                if (col[e] >= c0 && col[e] < c0 + bs) aug[r * w + (col[e] - c0)] += val[e];
        }
        double dnorm = 0.0; /* ||D_k||_1, the largest column sum of |entries| */
        for (int c = 0; c < bs; ++c) {
            double cs = 0.0;
            for (int r = 0; r < bs; ++r) cs += fabs(aug[r * w + c]);
            if (cs > dnorm) dnorm = cs;
        }
        int singular = 0;
        for (int p = 0; p < bs && !singular; ++p) {
            int piv = p;
            for (int r = p + 1; r < bs; ++r)
                if (fabs(aug[r * w + p]) > fabs(aug[piv * w + p])) piv = r;
            if (aug[piv * w + p] == 0.0) { singular = 1; break; }
            if (piv != p)
                for (int c = 0; c < w; ++c) {
                    double t = aug[p * w + c];
                    aug[p * w + c] = aug[piv * w + c];
                    aug[piv * w + c] = t;
                }
            const double inv = 1.0 / aug[p * w + p];
            for (int c = 0; c < w; ++c) aug[p * w + c] *= inv;
            for (int r = 0; r < bs; ++r) {
                if (r == p) continue;
                const double f = aug[r * w + p];
                if (f == 0.0) continue;
                for (int c = 0; c < w; ++c) aug[r * w + c] -= f * aug[p * w + c];
            }
        }
        double *out = minv + (size_t)k * (size_t)bs * (size_t)bs;
        for (int r = 0; r < bs; ++r)
            for (int c = 0; c < bs; ++c)
                out[r * bs + c] = singular ? (r == c ? 1.0 : 0.0) : aug[r * w + bs + c];
        if (flags) {
            double inorm = 0.0;
            for (int c = 0; c < bs; ++c) {
                double cs = 0.0;
                for (int r = 0; r < bs; ++r) cs += fabs(out[r * bs + c]);
                if (cs > inorm) inorm = cs;
            }
            /* FP32 also needs every nonzero entry inside FP32's normal range */
            double amax = 0.0, amin = INFINITY;
            for (int e = 0; e < bs * bs; ++e) {
                const double v = fabs(out[e]);
                if (v > amax) amax = v;
                if (v != 0.0 && v < amin) amin = v;
            }
            const int in_range = amax <= (double)FLT_MAX && (amin == INFINITY || amin >= (double)FLT_MIN);
            const int fp64 = !singular && (dnorm * inorm * ldexp(1.0, -24) > ORC_BJ_FP32_BOUND || !in_range);
            flags[k] = (unsigned char)fp64;
            if (!fp64)
                for (int e = 0; e < bs * bs; ++e) out[e] = (double)(float)out[e];
        }
    }
    free(aug);
    return 0;
}

int orc_block_jacobi_inv(int64_t n, const int32_t *rp, const int32_t *col, const double *val, int bs,
                         double *minv)
{
    return block_jacobi_inv_impl(n, rp, col, val, bs, minv, NULL);
}

int orc_block_jacobi_inv_adaptive(int64_t n, const int32_t *rp, const int32_t *col, const double *val, int bs,
                                  double *minv, unsigned char *flags)
{
    return block_jacobi_inv_impl(n, rp, col, val, bs, minv, flags);
}

static double *block_jacobi(int64_t n, const int32_t *rp, const int32_t *col, const double *val, int bs,
                            int adaptive)
{
    const int64_t nb = (n + bs - 1) / bs;
    double *m = malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1) * (size_t)bs * (size_t)bs);
    unsigned char *f = adaptive ? malloc((size_t)(nb > 0 ? nb : 1)) : NULL;
    block_jacobi_inv_impl(n, rp, col, val, bs, m, f);
    free(f);
    return m;
}

int orc_cg_bjacobi(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                   const double *b, double *x, double tol, int64_t maxit, orc_info *info, double *hist, int bs,
                   int adaptive)
{
    double *m = block_jacobi(n, rp, col, val, bs, adaptive);
    orc_prec M = {bs, m};
    int st = cg_run(n, rp, col, val, b, x, tol, maxit, info, hist, &M);
    free(m);
    return st;
}

int orc_bicgstab_bjacobi(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                         const double *b, double *x, double tol, int64_t maxit, orc_info *info, double *hist,
                         int bs, int adaptive)
{
    double *m = block_jacobi(n, rp, col, val, bs, adaptive);
    orc_prec M = {bs, m};
    int st = bicgstab_run(n, rp, col, val, b, x, tol, maxit, info, hist, &M);
    free(m);
    return st;
}

int orc_cgs_bjacobi(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                    const double *b, double *x, double tol, int64_t maxit, orc_info *info, double *hist, int bs,
                   int adaptive)
{
    double *m = block_jacobi(n, rp, col, val, bs, adaptive);
    orc_prec M = {bs, m};
    int st = cgs_run(n, rp, col, val, b, x, tol, maxit, info, hist, &M);
    free(m);
    return st;
}

int orc_gmres_bjacobi(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                      const double *b, double *x, int m, double tol, int64_t maxit, orc_info *info,
                      double *hist, int bs, int adaptive)
{
    double *mi = block_jacobi(n, rp, col, val, bs, adaptive);
    orc_prec M = {bs, mi};
    int st = gmres_run(n, rp, col, val, b, x, m, tol, maxit, info, hist, &M);
    free(mi);
    return st;
}


/* ------------------------------------------------------------------------- */
/* FP32 Krylov for the inner solve of iterative refinement: the same CG and  */
/* BiCGSTAB recurrences in float, with float accumulation.  No restarts and  */
/* no true-residual check: the outer FP64 loop owns convergence.             */
/* ------------------------------------------------------------------------- */
static void spmv_f32(int64_t n, const int32_t *rp, const int32_t *col, const float *val,
                     const float *x, float *y)
{
    for (int64_t i = 0; i < n; ++i) {
        float s = 0.0f;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += val[k] * x[col[k]];
        y[i] = s;
    }
}
static float dot_f32(int64_t n, const float *a, const float *b)
{
    float s = 0.0f;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static int64_t cg_f32(int64_t n, const int32_t *rp, const int32_t *col, const float *val,
                      const float *b, float *x, float tol, int64_t maxit)
{
    size_t bytes = (size_t)n * sizeof(float);
    float *r = malloc(bytes), *p = malloc(bytes), *q = malloc(bytes);
    float bn = sqrtf(dot_f32(n, b, b));
    int64_t it = 0;
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0f; r[i] = b[i]; p[i] = b[i]; }
    float rho = dot_f32(n, r, r);
    while (it < maxit && bn > 0.0f && sqrtf(rho) / bn > tol) {
        spmv_f32(n, rp, col, val, p, q);
        float pq = dot_f32(n, p, q);
        if (pq == 0.0f) break;
        float alpha = rho / pq;
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        float rho1 = dot_f32(n, r, r);
        ++it;
        if (sqrtf(rho1) / bn <= tol) break;
        float beta = rho1 / rho;
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rho = rho1;
    }
    free(r); free(p); free(q);
    return it;
}

static int64_t bicgstab_f32(int64_t n, const int32_t *rp, const int32_t *col, const float *val,
                            const float *b, float *x, float tol, int64_t maxit)
{
    size_t bytes = (size_t)n * sizeof(float);
    float *r = malloc(bytes), *rh = malloc(bytes), *p = malloc(bytes), *v = malloc(bytes);
    float *s = malloc(bytes), *t = malloc(bytes);
    float bn = sqrtf(dot_f32(n, b, b));
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0f; r[i] = b[i]; rh[i] = b[i]; p[i] = 0.0f; v[i] = 0.0f; }
    float rho = 1.0f, alpha = 1.0f, omega = 1.0f;
    int64_t it = 0;
    while (it < maxit && bn > 0.0f) {
        float rho1 = dot_f32(n, rh, r);
        if (rho1 == 0.0f) break;
        float beta = (rho1 / rho) * (alpha / omega);
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        spmv_f32(n, rp, col, val, p, v);
        float rv = dot_f32(n, rh, v);
        if (rv == 0.0f) break;
        alpha = rho1 / rv;
        for (int64_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
        ++it;
        if (sqrtf(dot_f32(n, s, s)) / bn <= tol) {
            for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
            break;
        }
        spmv_f32(n, rp, col, val, s, t);
        float tt = dot_f32(n, t, t);
        if (tt == 0.0f) break;
        omega = dot_f32(n, t, s) / tt;
        for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i] + omega * s[i];
        for (int64_t i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
        if (sqrtf(dot_f32(n, r, r)) / bn <= tol || omega == 0.0f) break;
        rho = rho1;
    }
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return it;
}

/* FP32 CGS as the inner solver of refinement.  Besides inner_tol and the    */
/* cycle cap it stops once the recurrence relative residual has gone        */
/* CGS_IR_STALL iterations without falling below half of the level it last  */
/* halved to (1 at x0 = 0).  CGS squares its residual polynomial            */
/* (Sonneveld, SIAM J. Sci. Stat. Comput. 10, 1989), so from a right-hand   */
/* side that mixes smooth and rough components an FP32 cycle can blow the   */
/* residual up and never recover; the FP64 outer residual then restarts it. */
#define CGS_IR_STALL 20
static int64_t cgs_f32(int64_t n, const int32_t *rp, const int32_t *col, const float *val,
                       const float *b, float *x, float tol, int64_t maxit)
{
    size_t bytes = (size_t)n * sizeof(float);
    float *r = malloc(bytes), *rh = malloc(bytes), *p = malloc(bytes), *u = malloc(bytes);
    float *q = malloc(bytes), *v = malloc(bytes), *w = malloc(bytes);
    float bn = sqrtf(dot_f32(n, b, b));
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0f; r[i] = b[i]; rh[i] = b[i]; p[i] = b[i]; u[i] = b[i]; }
    float rho = dot_f32(n, rh, r);
    int64_t it = 0, mark_it = 0;
    float mark = 1.0f;  /* relative residual of x0 = 0 */
    while (it < maxit && bn > 0.0f && rho != 0.0f) {
        spmv_f32(n, rp, col, val, p, v);
        float vr = dot_f32(n, rh, v);
        if (vr == 0.0f) break;
        float alpha = rho / vr;
        for (int64_t i = 0; i < n; ++i) { q[i] = u[i] - alpha * v[i]; w[i] = u[i] + q[i]; x[i] += alpha * w[i]; }
        spmv_f32(n, rp, col, val, w, v);
        for (int64_t i = 0; i < n; ++i) r[i] -= alpha * v[i];
        ++it;
        float rel = sqrtf(dot_f32(n, r, r)) / bn;
        if (rel <= tol) break;
        if (rel < 0.5f * mark) { mark = rel; mark_it = it; }
        else if (it - mark_it >= CGS_IR_STALL) break;
        float rho1 = dot_f32(n, rh, r);
        float beta = rho1 / rho;
        for (int64_t i = 0; i < n; ++i) { u[i] = r[i] + beta * q[i]; p[i] = u[i] + beta * (q[i] + beta * p[i]); }
        rho = rho1;
    }
    free(r); free(rh); free(p); free(u); free(q); free(v); free(w);
    return it;
}

/* ------------------------------------------------------------------------- */
/* Mixed-precision iterative refinement.                                     */
/*   x = x0; loop: r = b - A64 x (double); stop if ||r||/||b|| <= tol;       */
/*   d32 solves A32 d = fl32(r / ||r||) to inner_tol by CG (solver 0),       */
/*   BiCGSTAB (solver 1) or CGS (solver 3) in float; x += ||r|| * fl64(d).   */
/* A32 is the FP32 rounding of A64's values on the same index arrays.        */
/* iterations counts inner Krylov iterations; restarts counts outer cycles.  */
/* ------------------------------------------------------------------------- */
int orc_ir(int64_t n, const int32_t *rp, const int32_t *col, const double *val, int solver,
           const double *b, double *x, double tol, double inner_tol, int max_outer,
           int64_t maxit_inner, orc_info *info)
{
    memset(info, 0, sizeof(*info));
    int64_t nnz = rp[n];
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        memset(x, 0, (size_t)n * sizeof(double));
        return 0;
    }
    float *v32 = malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    for (int64_t k = 0; k < nnz; ++k) v32[k] = (float)val[k];
    double *r = malloc(sizeof(double) * (size_t)n);
    float *r32 = malloc(sizeof(float) * (size_t)n), *d32 = malloc(sizeof(float) * (size_t)n);
    int status = ORC_MAX_ITER;
    int64_t inner = 0;
    double rel = 0.0;
    int outer = 0;
    for (;; ++outer) {
#if ORC_MUTANT == 11
        {  /* planted: residual with the FP32 values */
            double *v = malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
            for (int64_t k = 0; k < nnz; ++k) v[k] = (double)v32[k];
            orc_spmv_csr(n, rp, col, v, x, r);
            free(v);
        }
#else
        orc_spmv_csr(n, rp, col, val, x, r);
#endif
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double rn = nrm2(n, r);
        rel = rn / bnorm;
        if (rel <= tol) { status = ORC_CONVERGED; break; }
        if (outer >= max_outer) { status = ORC_MAX_ITER; break; }
        for (int64_t i = 0; i < n; ++i) r32[i] = (float)(r[i] / rn);
        inner += solver == 0   ? cg_f32(n, rp, col, v32, r32, d32, (float)inner_tol, maxit_inner)
                 : solver == 3 ? cgs_f32(n, rp, col, v32, r32, d32, (float)inner_tol, maxit_inner)
                               : bicgstab_f32(n, rp, col, v32, r32, d32, (float)inner_tol, maxit_inner);
#if ORC_MUTANT == 9
        for (int64_t i = 0; i < n; ++i) x[i] += (double)d32[i];  /* planted: correction not scaled back */
#elif ORC_MUTANT == 10
        for (int64_t i = 0; i < n; ++i) x[i] = (float)(x[i] + rn * (double)d32[i]);  /* planted: FP32 update */
#else
        for (int64_t i = 0; i < n; ++i) x[i] += rn * (double)d32[i];
#endif
    }
    info->status = status;
    info->iterations = inner;
    info->restarts = outer;
    info->relres_recurrence = rel;
    info->relres_true = rel;
    free(v32); free(r); free(r32); free(d32);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Mixed-precision CG with reliable updates (the residual replacement of     */
/* Sleijpen and van der Vorst, Computing 56, 1996, applied to CG with FP32   */
/* iterations): CG runs in FP32 on the FP32-rounded values, its iterate      */
/* accumulated in an FP32 correction y.  When the FP32 recurrence residual   */
/* falls below delta times its largest value since the last update, or below */
/* tol ||b||, or the iteration budget is spent, y is added to the FP64 x, the */
/* residual is recomputed as b - A x in FP64 with the FP64 values, and the   */
/* FP32 residual is replaced by its rounding.  The direction p is kept (no   */
/* restart of the Krylov space); beta is formed with the replaced residual.  */
/* The solve ends when the FP64 residual meets tol.  restarts = updates.     */
/* ------------------------------------------------------------------------- */
int orc_cg_reliable(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                    const double *b, double *x, double tol, double delta, int64_t maxit,
                    orc_info *info)
{
    memset(info, 0, sizeof(*info));
    int64_t nnz = rp[n];
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        memset(x, 0, (size_t)n * sizeof(double));
        return 0;
    }
    float *v32 = malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    for (int64_t k = 0; k < nnz; ++k) v32[k] = (float)val[k];
    double *r = malloc(sizeof(double) * (size_t)n);
    size_t fb = sizeof(float) * (size_t)n;
    float *r32 = malloc(fb), *p = malloc(fb), *q = malloc(fb), *y = malloc(fb);
    /* the FP64 residual of the current x */
    orc_spmv_csr(n, rp, col, val, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double rel = nrm2(n, r) / bnorm;
    int status = rel <= tol ? ORC_CONVERGED : ORC_MAX_ITER;
    int64_t it = 0;
    int updates = 0;
    const float ftol = (float)(tol * bnorm);
    for (int64_t i = 0; i < n; ++i) { r32[i] = (float)r[i]; p[i] = r32[i]; y[i] = 0.0f; }
    float rho = dot_f32(n, r32, r32);
    float maxr = sqrtf(rho);
    while (status != ORC_CONVERGED && it < maxit) {
        spmv_f32(n, rp, col, v32, p, q);
        float pq = dot_f32(n, p, q);
        if (pq == 0.0f) { status = ORC_BREAKDOWN; break; }
        float alpha = rho / pq;
        for (int64_t i = 0; i < n; ++i) { y[i] += alpha * p[i]; r32[i] -= alpha * q[i]; }
        float rho1 = dot_f32(n, r32, r32);
        ++it;
        float rn32 = sqrtf(rho1);
        if (rn32 > maxr) maxr = rn32;
        if (rn32 <= ftol || rn32 < (float)delta * maxr || it >= maxit) {
            /* reliable update: fold y into the FP64 x and replace the residual */
            for (int64_t i = 0; i < n; ++i) { x[i] += (double)y[i]; y[i] = 0.0f; }
#if ORC_MUTANT == 15
            /* planted: the FP64 residual is never recomputed (the recurrence is trusted) */
            for (int64_t i = 0; i < n; ++i) r[i] = (double)r32[i];
#else
            orc_spmv_csr(n, rp, col, val, x, r);
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
#endif
            rel = nrm2(n, r) / bnorm;
            ++updates;
            if (rel <= tol) { status = ORC_CONVERGED; break; }
            for (int64_t i = 0; i < n; ++i) r32[i] = (float)r[i];
            rho1 = dot_f32(n, r32, r32);
            maxr = sqrtf(rho1);
#if ORC_MUTANT == 16
            rho = rho1;  /* planted: restart the Krylov space (beta = 0) at every update */
            for (int64_t i = 0; i < n; ++i) p[i] = 0.0f;
#endif
        }
        float beta = rho1 / rho;
        for (int64_t i = 0; i < n; ++i) p[i] = r32[i] + beta * p[i];
        rho = rho1;
    }
    info->status = status;
    info->iterations = it;
    info->restarts = updates;
    info->relres_recurrence = rel;
    info->relres_true = rel;
    free(v32); free(r); free(r32); free(p); free(q); free(y);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Fixed-iteration loops for the CPU baseline timing: k SpMVs, no checks.     */
/* ------------------------------------------------------------------------- */
void orc_spmv_repeat(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                     const double *x, double *y, int reps)
{
    for (int r = 0; r < reps; ++r) spmv_plain(n, rp, col, val, x, y);
}
