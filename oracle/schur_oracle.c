/*
 * CPU oracle for the Schur refinement iteration -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct C. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library; the CUDA library never links
 * or calls it, and this file shares no code with it.
 *
 * Contents (all matrices column-major, element (i,j) at M[i + j*ld]):
 *   - Alg. 2 (Sec. 2.1, "successive substitution"): solves stril(T L - L T) = -E
 *     for strictly lower L, column j = 1..n-1, row i = n..j+1, in float,
 *     double and complex double.
 *   - Alg. 3 (Sec. 2.1, recursive block algorithm) with its triangular
 *     Sylvester sub-solve (eq. "l21"), in double.
 *   - A brute-force solve of the same equation: the n(n-1)/2 x n(n-1)/2 matrix
 *     of the operator L -> stril(T L - L T) assembled column by column from
 *     that definition and solved by Gaussian elimination with partial
 *     pivoting in 128-bit floating point (pins Alg. 2 for n <= 8).
 *   - Residuals ||stril(Q^H A Q)||_F / ||A||_F and ||Q^H Q - I||_F evaluated
 *     with double-double dot products (Sec. 3 reports these two quantities).
 *   - A double-double dot product / GEMM used for the double-double target.
 *   - For the double-double target (hp = double-double, lp = double): Alg. 2
 *     with divisors formed from a double-double diagonal, and the two
 *     residuals (full, or sampled entries) evaluated in 128-bit floating
 *     point.
 *
 * Compile with -ffp-contract=off: every rounding here is the one written.
 * Return codes: 0 ok, 2 two diagonal entries of T coincide (Theorem 1),
 * 3 a non-finite value appeared.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(__x86_64__) || defined(__i386__)
typedef __float128 f128_t;
#else
typedef long double f128_t; /* IEEE binary128 on AArch64 */
#endif

#define SRO_OK 0
#define SRO_NONDISTINCT 2
#define SRO_NONFINITE 3

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* ------------------------------------------------------------------ */
/* Alg. 2 in double. The divisor t_ii - t_jj is formed from dhp if given
 * (the high-precision diagonal), else from T. Every variant computes the
 * columns j < ncols of L (all of them when ncols < 0 or ncols >= n - 1) and
 * leaves the others zero: Alg. 2 forms column j from the columns before it
 * only, so these leading columns are those of the full solve. */
int sro_alg2_f64(int n, const double *T, int ldt, const double *E, int lde,
                 const double *dhp, double *L, int ldl, double cap, int ncols)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) L[IDX(i, j, ldl)] = 0.0;
    const int jend = (ncols < 0 || ncols > n - 1) ? n - 1 : ncols;
    for (int j = 0; j < jend; ++j) {
        for (int i = n - 1; i >= j + 1; --i) {
            double e = E[IDX(i, j, lde)];
            double s1 = 0.0, s2 = 0.0;
            for (int k = i + 1; k < n; ++k) s1 += T[IDX(i, k, ldt)] * L[IDX(k, j, ldl)];
            for (int k = 0; k < j; ++k) s2 += L[IDX(i, k, ldl)] * T[IDX(k, j, ldt)];
            e = e + s1 - s2;
            double di = dhp ? dhp[i] : T[IDX(i, i, ldt)];
            double dj = dhp ? dhp[j] : T[IDX(j, j, ldt)];
            double den = di - dj;
            if (den == 0.0) return SRO_NONDISTINCT;
            double l = -e / den;
            if (cap > 0.0 && fabs(l) > cap) l = 0.0;
            if (!isfinite(l)) return SRO_NONFINITE;
            L[IDX(i, j, ldl)] = l;
        }
    }
    return SRO_OK;
}

/* Alg. 2 in float (the low precision of the mixed form). The divisor is formed
 * in double from dhp and then rounded to float. */
int sro_alg2_f32(int n, const float *T, int ldt, const float *E, int lde,
                 const double *dhp, float *L, int ldl, double cap, int ncols)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) L[IDX(i, j, ldl)] = 0.0f;
    const int jend = (ncols < 0 || ncols > n - 1) ? n - 1 : ncols;
    for (int j = 0; j < jend; ++j) {
        for (int i = n - 1; i >= j + 1; --i) {
            float e = E[IDX(i, j, lde)];
            float s1 = 0.0f, s2 = 0.0f;
            for (int k = i + 1; k < n; ++k) s1 += T[IDX(i, k, ldt)] * L[IDX(k, j, ldl)];
            for (int k = 0; k < j; ++k) s2 += L[IDX(i, k, ldl)] * T[IDX(k, j, ldt)];
            e = e + s1 - s2;
            float den = dhp ? (float)(dhp[i] - dhp[j])
                            : (T[IDX(i, i, ldt)] - T[IDX(j, j, ldt)]);
            if (den == 0.0f) return SRO_NONDISTINCT;
            float l = -e / den;
            if (cap > 0.0 && fabsf(l) > (float)cap) l = 0.0f;
            if (!isfinite(l)) return SRO_NONFINITE;
            L[IDX(i, j, ldl)] = l;
        }
    }
    return SRO_OK;
}

/* Alg. 2 in complex double (interleaved re, im). */
int sro_alg2_c128(int n, const double complex *T, int ldt, const double complex *E, int lde,
                  const double complex *dhp, double complex *L, int ldl, double cap, int ncols)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) L[IDX(i, j, ldl)] = 0.0;
    const int jend = (ncols < 0 || ncols > n - 1) ? n - 1 : ncols;
    for (int j = 0; j < jend; ++j) {
        for (int i = n - 1; i >= j + 1; --i) {
            double complex e = E[IDX(i, j, lde)];
            double complex s1 = 0.0, s2 = 0.0;
            for (int k = i + 1; k < n; ++k) s1 += T[IDX(i, k, ldt)] * L[IDX(k, j, ldl)];
            for (int k = 0; k < j; ++k) s2 += L[IDX(i, k, ldl)] * T[IDX(k, j, ldt)];
            e = e + s1 - s2;
            double complex di = dhp ? dhp[i] : T[IDX(i, i, ldt)];
            double complex dj = dhp ? dhp[j] : T[IDX(j, j, ldt)];
            double complex den = di - dj;
            if (den == 0.0) return SRO_NONDISTINCT;
            double complex l = -e / den;
            if (cap > 0.0 && creal(l) * creal(l) + cimag(l) * cimag(l) > cap * cap) l = 0.0;
            if (!isfinite(creal(l)) || !isfinite(cimag(l))) return SRO_NONFINITE;
            L[IDX(i, j, ldl)] = l;
        }
    }
    return SRO_OK;
}

/* Alg. 2 in complex float with divisors formed in complex double. */
int sro_alg2_c64(int n, const float complex *T, int ldt, const float complex *E, int lde,
                 const double complex *dhp, float complex *L, int ldl, double cap, int ncols)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) L[IDX(i, j, ldl)] = 0.0f;
    const int jend = (ncols < 0 || ncols > n - 1) ? n - 1 : ncols;
    for (int j = 0; j < jend; ++j) {
        for (int i = n - 1; i >= j + 1; --i) {
            float complex e = E[IDX(i, j, lde)];
            float complex s1 = 0.0f, s2 = 0.0f;
            for (int k = i + 1; k < n; ++k) s1 += T[IDX(i, k, ldt)] * L[IDX(k, j, ldl)];
            for (int k = 0; k < j; ++k) s2 += L[IDX(i, k, ldl)] * T[IDX(k, j, ldt)];
            e = e + s1 - s2;
            float complex den = dhp ? (float complex)(dhp[i] - dhp[j])
                                    : (T[IDX(i, i, ldt)] - T[IDX(j, j, ldt)]);
            if (den == 0.0f) return SRO_NONDISTINCT;
            float complex l = -e / den;
            if (cap > 0.0) {
                const float c = (float)cap;
                if (crealf(l) * crealf(l) + cimagf(l) * cimagf(l) > c * c) l = 0.0f;
            }
            if (!isfinite(crealf(l)) || !isfinite(cimagf(l))) return SRO_NONFINITE;
            L[IDX(i, j, ldl)] = l;
        }
    }
    return SRO_OK;
}

/* ------------------------------------------------------------------ */
/* Triangular Sylvester equation T22 X - X T11 = C (T11: n1 x n1, T22: n2 x n2,
 * both upper triangular, X and C: n2 x n1), eq. "l21" of Sec. 2.1. Column b
 * of X satisfies (T22 - t11_bb I) x_b = c_b + sum_{c<b} x_c T11(c,b), an upper
 * triangular system solved by back substitution. */
static int sylv_tri_f64(int n2, int n1, const double *T22, int ld22, const double *T11, int ld11,
                        const double *C, int ldc, double *X, int ldx)
{
    double *rhs = (double *)malloc(sizeof(double) * (size_t)(n2 > 0 ? n2 : 1));
    if (!rhs) return SRO_NONFINITE;
    for (int b = 0; b < n1; ++b) {
        for (int a = 0; a < n2; ++a) {
            double r = C[IDX(a, b, ldc)];
            for (int c = 0; c < b; ++c) r += X[IDX(a, c, ldx)] * T11[IDX(c, b, ld11)];
            rhs[a] = r;
        }
        double tbb = T11[IDX(b, b, ld11)];
        for (int a = n2 - 1; a >= 0; --a) {
            double r = rhs[a];
            for (int c = a + 1; c < n2; ++c) r -= T22[IDX(a, c, ld22)] * X[IDX(c, b, ldx)];
            double den = T22[IDX(a, a, ld22)] - tbb;
            if (den == 0.0) { free(rhs); return SRO_NONDISTINCT; }
            X[IDX(a, b, ldx)] = r / den;
        }
    }
    free(rhs);
    return SRO_OK;
}

/* Alg. 3 in double: E (n x n, strictly lower part used) is overwritten. */
static int alg3_rec(int n, const double *T, int ldt, double *E, int lde, double *L, int ldl, int nmin)
{
    if (n <= nmin) {
        /* Alg. 2 on the block, reading E in place. */
        double *Lb = (double *)calloc((size_t)n * (size_t)n, sizeof(double));
        if (!Lb) return SRO_NONFINITE;
        int rc = sro_alg2_f64(n, T, ldt, E, lde, NULL, Lb, n, 0.0, -1);
        for (int j = 0; j < n; ++j)
            for (int i = j + 1; i < n; ++i) L[IDX(i, j, ldl)] = Lb[IDX(i, j, n)];
        free(Lb);
        return rc;
    }
    int n1 = n / 2, n2 = n - n1;
    const double *T11 = T, *T12 = T + IDX(0, n1, ldt), *T22 = T + IDX(n1, n1, ldt);
    double *E21 = E + IDX(n1, 0, lde);
    double *L21 = L + IDX(n1, 0, ldl);
    /* T22 X - X T11 = -E21 */
    double *C = (double *)malloc(sizeof(double) * (size_t)n2 * (size_t)n1);
    if (!C) return SRO_NONFINITE;
    for (int b = 0; b < n1; ++b)
        for (int a = 0; a < n2; ++a) C[IDX(a, b, n2)] = -E21[IDX(a, b, lde)];
    int rc = sylv_tri_f64(n2, n1, T22, ldt, T11, ldt, C, n2, L21, ldl);
    free(C);
    if (rc) return rc;
    /* E11 <- E11 + stril(T12 L21) */
    for (int j = 0; j < n1; ++j)
        for (int i = j + 1; i < n1; ++i) {
            double s = 0.0;
            for (int k = 0; k < n2; ++k) s += T12[IDX(i, k, ldt)] * L21[IDX(k, j, ldl)];
            E[IDX(i, j, lde)] += s;
        }
    /* E22 <- E22 - stril(L21 T12) */
    for (int j = 0; j < n2; ++j)
        for (int i = j + 1; i < n2; ++i) {
            double s = 0.0;
            for (int k = 0; k < n1; ++k) s += L21[IDX(i, k, ldl)] * T12[IDX(k, j, ldt)];
            E[IDX(n1 + i, n1 + j, lde)] -= s;
        }
    rc = alg3_rec(n1, T11, ldt, E, lde, L, ldl, nmin);
    if (rc) return rc;
    return alg3_rec(n2, T22, ldt, E + IDX(n1, n1, lde), lde, L + IDX(n1, n1, ldl), ldl, nmin);
}

int sro_alg3_f64(int n, const double *T, int ldt, double *E, int lde, double *L, int ldl, int nmin)
{
    if (nmin < 2) nmin = 2;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) L[IDX(i, j, ldl)] = 0.0;
    return alg3_rec(n, T, ldt, E, lde, L, ldl, nmin);
}

/* ------------------------------------------------------------------ */
/* Brute force: unknowns are the strictly lower entries of L, numbered
 * column by column. Column u of the operator matrix is stril(T U - U T) for
 * the unit matrix U carrying a one at unknown u, evaluated by a full triple
 * loop. The square system is solved in 128-bit arithmetic. Result returned as
 * a double-double pair (hi + lo). Only for small n (N = n(n-1)/2 <= 1000). */
static f128_t qabs(f128_t x) { return x < 0 ? -x : x; }

int sro_kron_solve(int n, const double *T, int ldt, const double *E, int lde,
                   double *Lhi, double *Llo, int ldl)
{
    int N = n * (n - 1) / 2;
    if (N == 0) return SRO_OK;
    int *ui = (int *)malloc(sizeof(int) * N), *uj = (int *)malloc(sizeof(int) * N);
    f128_t *M = (f128_t *)calloc((size_t)N * (size_t)(N + 1), sizeof(f128_t));
    f128_t *U = (f128_t *)calloc((size_t)n * (size_t)n, sizeof(f128_t));
    f128_t *R = (f128_t *)calloc((size_t)n * (size_t)n, sizeof(f128_t));
    if (!ui || !uj || !M || !U || !R) return SRO_NONFINITE;
    int u = 0;
    for (int j = 0; j < n; ++j)
        for (int i = j + 1; i < n; ++i) { ui[u] = i; uj[u] = j; ++u; }
    /* rows: equation for each strictly lower (i,j); columns: unknowns; last column: rhs */
    for (int c = 0; c < N; ++c) {
        memset(U, 0, sizeof(f128_t) * (size_t)n * (size_t)n);
        U[IDX(ui[c], uj[c], n)] = 1;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                f128_t s = 0;
                for (int k = 0; k < n; ++k)
                    s += (f128_t)T[IDX(i, k, ldt)] * U[IDX(k, j, n)] - U[IDX(i, k, n)] * (f128_t)T[IDX(k, j, ldt)];
                R[IDX(i, j, n)] = s;
            }
        for (int r = 0; r < N; ++r) M[IDX(r, c, N)] = R[IDX(ui[r], uj[r], n)];
    }
    for (int r = 0; r < N; ++r) M[IDX(r, N, N)] = -(f128_t)E[IDX(ui[r], uj[r], lde)];
    /* Gaussian elimination with partial pivoting. The operator is singular
     * exactly when two diagonal entries of T coincide (Theorem 1); eliminating
     * a singular matrix in 128-bit arithmetic leaves a pivot at the rounding
     * level of the elimination rather than an exact zero, so a pivot below
     * N * 2^-112 * max|M| counts as zero. */
    f128_t mmax = 0;
    for (int c = 0; c < N; ++c)
        for (int r = 0; r < N; ++r)
            if (qabs(M[IDX(r, c, N)]) > mmax) mmax = qabs(M[IDX(r, c, N)]);
    const f128_t ptol = (f128_t)N * mmax * (f128_t)ldexp(1.0, -112);
    int rc = SRO_OK;
    for (int c = 0; c < N; ++c) {
        int p = c;
        for (int r = c + 1; r < N; ++r)
            if (qabs(M[IDX(r, c, N)]) > qabs(M[IDX(p, c, N)])) p = r;
        if (qabs(M[IDX(p, c, N)]) <= ptol) { rc = SRO_NONDISTINCT; break; }
        if (p != c)
            for (int k = c; k <= N; ++k) {
                f128_t t = M[IDX(c, k, N)];
                M[IDX(c, k, N)] = M[IDX(p, k, N)];
                M[IDX(p, k, N)] = t;
            }
        for (int r = c + 1; r < N; ++r) {
            f128_t f = M[IDX(r, c, N)] / M[IDX(c, c, N)];
            if (f == 0) continue;
            for (int k = c; k <= N; ++k) M[IDX(r, k, N)] -= f * M[IDX(c, k, N)];
        }
    }
    if (rc == SRO_OK) {
        f128_t *x = (f128_t *)calloc((size_t)N, sizeof(f128_t));
        for (int c = N - 1; c >= 0; --c) {
            f128_t s = M[IDX(c, N, N)];
            for (int k = c + 1; k < N; ++k) s -= M[IDX(c, k, N)] * x[k];
            x[c] = s / M[IDX(c, c, N)];
        }
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) { Lhi[IDX(i, j, ldl)] = 0.0; Llo[IDX(i, j, ldl)] = 0.0; }
        for (int c = 0; c < N; ++c) {
            double hi = (double)x[c];
            double lo = (double)(x[c] - (f128_t)hi);
            Lhi[IDX(ui[c], uj[c], ldl)] = hi;
            Llo[IDX(ui[c], uj[c], ldl)] = lo;
        }
        free(x);
    }
    free(ui); free(uj); free(M); free(U); free(R);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Double-double arithmetic: Knuth's TwoSum and an FMA-based TwoProd. */
typedef struct { double hi, lo; } dd_t;

static inline dd_t two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd_t r = {s, e};
    return r;
}
static inline dd_t fast_two_sum(double a, double b)
{
    double s = a + b;
    double e = b - (s - a);
    dd_t r = {s, e};
    return r;
}
static inline dd_t two_prod(double a, double b)
{
    double p = a * b;
    double e = fma(a, b, -p);
    dd_t r = {p, e};
    return r;
}
static inline dd_t dd_add(dd_t a, dd_t b)
{
    dd_t s = two_sum(a.hi, b.hi);
    dd_t t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
static inline dd_t dd_mul_d(dd_t a, double b)
{
    dd_t p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return fast_two_sum(p.hi, p.lo);
}
static inline dd_t dd_mul(dd_t a, dd_t b)
{
    dd_t p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}

/* C = op(A) * B in double-double, where A, B are double-double (hi, lo planes;
 * lo planes may be NULL for plain doubles). transA = 1 uses A^T. C (hi, lo)
 * is m x n. */
void sro_gemm_dd(int transA, int m, int n, int k,
                 const double *Ahi, const double *Alo, int lda,
                 const double *Bhi, const double *Blo, int ldb,
                 double *Chi, double *Clo, int ldc)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < m; ++i) {
            dd_t s = {0.0, 0.0};
            for (int l = 0; l < k; ++l) {
                size_t ia = transA ? IDX(l, i, lda) : IDX(i, l, lda);
                dd_t a = {Ahi[ia], Alo ? Alo[ia] : 0.0};
                dd_t b = {Bhi[IDX(l, j, ldb)], Blo ? Blo[IDX(l, j, ldb)] : 0.0};
                s = dd_add(s, dd_mul(a, b));
            }
            Chi[IDX(i, j, ldc)] = s.hi;
            Clo[IDX(i, j, ldc)] = s.lo;
        }
    }
}

/* Residuals of a real decomposition, evaluated in double-double:
 *   r_T = ||stril(Q^T A Q)||_F / ||A||_F,  r_Q = ||Q^T Q - I||_F. */
/* r_T counts the entries below the diagonal blocks: for a quasi-triangular
 * form (blk[k] = 2 at the first row of a 2 x 2 block, see sro_alg2_quasi_f64)
 * the coupling entry (k+1, k) of each 2 x 2 block is part of T, not of the
 * residual; blk NULL: every block 1 x 1 (stril). */
static void residuals_dd_blk(int n, const double *A, int lda, const double *Q, int ldq, const int *blk,
                             double *r_T, double *r_Q);

void sro_residuals_dd(int n, const double *A, int lda, const double *Q, int ldq,
                      double *r_T, double *r_Q)
{
    residuals_dd_blk(n, A, lda, Q, ldq, NULL, r_T, r_Q);
}

void sro_residuals_dd_quasi(int n, const double *A, int lda, const double *Q, int ldq, const int *blk,
                            double *r_T, double *r_Q)
{
    residuals_dd_blk(n, A, lda, Q, ldq, blk, r_T, r_Q);
}

static void residuals_dd_blk(int n, const double *A, int lda, const double *Q, int ldq, const int *blk,
                             double *r_T, double *r_Q)
{
    double *Mhi = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double *Mlo = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    /* M = A Q in double-double */
    sro_gemm_dd(0, n, n, n, A, NULL, lda, Q, NULL, ldq, Mhi, Mlo, n);
    double st = 0.0, so = 0.0, sa = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : st, so)
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
            if (i > j && !(blk && i == j + 1 && blk[j] == 2)) { /* (Q^T M)(i,j) */
                dd_t s = {0.0, 0.0};
                for (int l = 0; l < n; ++l) {
                    dd_t m = {Mhi[IDX(l, j, n)], Mlo[IDX(l, j, n)]};
                    s = dd_add(s, dd_mul_d(m, Q[IDX(l, i, ldq)]));
                }
                double v = s.hi + s.lo;
                st += v * v;
            }
            if (i <= j) { /* (Q^T Q - I)(i,j), symmetric */
                dd_t s = {0.0, 0.0};
                for (int l = 0; l < n; ++l) s = dd_add(s, two_prod(Q[IDX(l, i, ldq)], Q[IDX(l, j, ldq)]));
                if (i == j) s = dd_add(s, (dd_t){-1.0, 0.0});
                double v = s.hi + s.lo;
                so += (i == j ? 1.0 : 2.0) * v * v;
            }
        }
    }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) sa += A[IDX(i, j, lda)] * A[IDX(i, j, lda)];
    *r_T = sqrt(st) / sqrt(sa);
    *r_Q = sqrt(so);
    free(Mhi); free(Mlo);
}

/* Selected entries of Q^T A Q and of Q^T Q - I in double-double, for sampled
 * checks at sizes where the full residual is too slow. For sample s the pair
 * (rows[s], cols[s]) is evaluated, O(n^2) work per sample. Outputs are
 * hi + lo rounded to double. */
void sro_sample_entries_dd(int n, const double *A, int lda, const double *Q, int ldq,
                           int ns, const int *rows, const int *cols,
                           double *tq, double *yq)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < ns; ++s) {
        int i = rows[s], j = cols[s];
        dd_t acc = {0.0, 0.0};
        for (int l = 0; l < n; ++l) {
            dd_t aq = {0.0, 0.0};
            for (int k = 0; k < n; ++k) aq = dd_add(aq, two_prod(A[IDX(l, k, lda)], Q[IDX(k, j, ldq)]));
            acc = dd_add(acc, dd_mul_d(aq, Q[IDX(l, i, ldq)]));
        }
        tq[s] = acc.hi + acc.lo;
        dd_t g = {0.0, 0.0};
        for (int l = 0; l < n; ++l) g = dd_add(g, two_prod(Q[IDX(l, i, ldq)], Q[IDX(l, j, ldq)]));
        if (i == j) g = dd_add(g, (dd_t){-1.0, 0.0});
        yq[s] = g.hi + g.lo;
    }
}

/* Complex form of sro_sample_entries_dd (interleaved complex128 input; tq, yq
   receive 2 ns doubles, re and im of each sampled entry):
   (Q^H A Q)(i, j) = sum_l conj(Q(l, i)) sum_k A(l, k) Q(k, j), (Q^H Q - I)(i, j). */
void sro_sample_entries_dd_c(int n, const double *A, int lda, const double *Q, int ldq,
                             int ns, const int *rows, const int *cols,
                             double *tq, double *yq)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < ns; ++s) {
        int i = rows[s], j = cols[s];
        dd_t tr = {0.0, 0.0}, ti = {0.0, 0.0};
        for (int l = 0; l < n; ++l) {
            dd_t ar = {0.0, 0.0}, ai = {0.0, 0.0};   /* (A Q)(l, j) */
            for (int k = 0; k < n; ++k) {
                double xr = A[2 * IDX(l, k, lda)], xi = A[2 * IDX(l, k, lda) + 1];
                double qr = Q[2 * IDX(k, j, ldq)], qi = Q[2 * IDX(k, j, ldq) + 1];
                ar = dd_add(ar, two_prod(xr, qr));
                ar = dd_add(ar, two_prod(-xi, qi));
                ai = dd_add(ai, two_prod(xr, qi));
                ai = dd_add(ai, two_prod(xi, qr));
            }
            double cr = Q[2 * IDX(l, i, ldq)], ci = -Q[2 * IDX(l, i, ldq) + 1];   /* conj(Q(l, i)) */
            tr = dd_add(tr, dd_mul_d(ar, cr));
            tr = dd_add(tr, dd_mul_d(ai, -ci));
            ti = dd_add(ti, dd_mul_d(ai, cr));
            ti = dd_add(ti, dd_mul_d(ar, ci));
        }
        tq[2 * s] = tr.hi + tr.lo;
        tq[2 * s + 1] = ti.hi + ti.lo;
        dd_t gr = {0.0, 0.0}, gi = {0.0, 0.0};
        for (int l = 0; l < n; ++l) {
            double cr = Q[2 * IDX(l, i, ldq)], ci = -Q[2 * IDX(l, i, ldq) + 1];
            double qr = Q[2 * IDX(l, j, ldq)], qi = Q[2 * IDX(l, j, ldq) + 1];
            gr = dd_add(gr, two_prod(cr, qr));
            gr = dd_add(gr, two_prod(-ci, qi));
            gi = dd_add(gi, two_prod(cr, qi));
            gi = dd_add(gi, two_prod(ci, qr));
        }
        if (i == j) gr = dd_add(gr, (dd_t){-1.0, 0.0});
        yq[2 * s] = gr.hi + gr.lo;
        yq[2 * s + 1] = gi.hi + gi.lo;
    }
}

/* Complex residuals in double-double (interleaved complex128 input). */
void sro_residuals_dd_c(int n, const double *A, int lda, const double *Q, int ldq,
                        double *r_T, double *r_Q)
{
    /* M = A Q, complex, in double-double: separate re/im planes */
    size_t nn = (size_t)n * (size_t)n;
    double *Mr = (double *)malloc(sizeof(double) * nn), *Mrl = (double *)malloc(sizeof(double) * nn);
    double *Mi = (double *)malloc(sizeof(double) * nn), *Mil = (double *)malloc(sizeof(double) * nn);
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            dd_t sr = {0.0, 0.0}, si = {0.0, 0.0};
            for (int l = 0; l < n; ++l) {
                double ar = A[2 * IDX(i, l, lda)], ai = A[2 * IDX(i, l, lda) + 1];
                double qr = Q[2 * IDX(l, j, ldq)], qi = Q[2 * IDX(l, j, ldq) + 1];
                sr = dd_add(sr, two_prod(ar, qr));
                sr = dd_add(sr, two_prod(-ai, qi));
                si = dd_add(si, two_prod(ar, qi));
                si = dd_add(si, two_prod(ai, qr));
            }
            Mr[IDX(i, j, n)] = sr.hi; Mrl[IDX(i, j, n)] = sr.lo;
            Mi[IDX(i, j, n)] = si.hi; Mil[IDX(i, j, n)] = si.lo;
        }
    double st = 0.0, so = 0.0, sa = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : st, so)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            if (i > j) { /* conj(Q(:,i))^T M(:,j) */
                dd_t sr = {0.0, 0.0}, si = {0.0, 0.0};
                for (int l = 0; l < n; ++l) {
                    double qr = Q[2 * IDX(l, i, ldq)], qi = -Q[2 * IDX(l, i, ldq) + 1];
                    dd_t mr = {Mr[IDX(l, j, n)], Mrl[IDX(l, j, n)]};
                    dd_t mi = {Mi[IDX(l, j, n)], Mil[IDX(l, j, n)]};
                    sr = dd_add(sr, dd_mul_d(mr, qr));
                    sr = dd_add(sr, dd_mul_d(mi, -qi));
                    si = dd_add(si, dd_mul_d(mi, qr));
                    si = dd_add(si, dd_mul_d(mr, qi));
                }
                double vr = sr.hi + sr.lo, vi = si.hi + si.lo;
                st += vr * vr + vi * vi;
            }
            if (i <= j) {
                dd_t sr = {0.0, 0.0}, si = {0.0, 0.0};
                for (int l = 0; l < n; ++l) {
                    double ar = Q[2 * IDX(l, i, ldq)], ai = -Q[2 * IDX(l, i, ldq) + 1];
                    double br = Q[2 * IDX(l, j, ldq)], bi = Q[2 * IDX(l, j, ldq) + 1];
                    sr = dd_add(sr, two_prod(ar, br));
                    sr = dd_add(sr, two_prod(-ai, bi));
                    si = dd_add(si, two_prod(ar, bi));
                    si = dd_add(si, two_prod(ai, br));
                }
                if (i == j) sr = dd_add(sr, (dd_t){-1.0, 0.0});
                double vr = sr.hi + sr.lo, vi = si.hi + si.lo;
                so += (i == j ? 1.0 : 2.0) * (vr * vr + vi * vi);
            }
        }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double ar = A[2 * IDX(i, j, lda)], ai = A[2 * IDX(i, j, lda) + 1];
            sa += ar * ar + ai * ai;
        }
    *r_T = sqrt(st) / sqrt(sa);
    *r_Q = sqrt(so);
    free(Mr); free(Mrl); free(Mi); free(Mil);
}

/* Thread count of the OpenMP loops above (1 = serial). */
void sro_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int sro_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Double-double working precision (hp = double-double, lp = double). */

/* Alg. 2 in double with the divisors of a double-double diagonal:
 * t_ii - t_jj is formed in double-double from (dhi, dlo) and rounded once to
 * double (the reading "form the divisor in hp, then round" of the FP64 forms,
 * one precision level up). */
int sro_alg2_f64_dd(int n, const double *T, int ldt, const double *E, int lde,
                    const double *dhi, const double *dlo, double *L, int ldl, double cap)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) L[IDX(i, j, ldl)] = 0.0;
    for (int j = 0; j < n - 1; ++j) {
        for (int i = n - 1; i >= j + 1; --i) {
            double e = E[IDX(i, j, lde)];
            double s1 = 0.0, s2 = 0.0;
            for (int k = i + 1; k < n; ++k) s1 += T[IDX(i, k, ldt)] * L[IDX(k, j, ldl)];
            for (int k = 0; k < j; ++k) s2 += L[IDX(i, k, ldl)] * T[IDX(k, j, ldt)];
            e = e + s1 - s2;
            dd_t di = {dhi[i], dlo[i]}, mdj = {-dhi[j], -dlo[j]};
            dd_t dd = dd_add(di, mdj);
            double den = dd.hi + dd.lo;
            if (den == 0.0) return SRO_NONDISTINCT;
            double l = -e / den;
            if (cap > 0.0 && fabs(l) > cap) l = 0.0;
            if (!isfinite(l)) return SRO_NONFINITE;
            L[IDX(i, j, ldl)] = l;
        }
    }
    return SRO_OK;
}

/* Residuals of a double-double decomposition in 128-bit floating point:
 *   r_T = ||stril(Q^T A Q)||_F / ||A||_F,  r_Q = ||Q^T Q - I||_F,
 * A = Ahi + Alo, Q = Qhi + Qlo (the lo planes may be NULL). */
static inline f128_t q_of(const double *hi, const double *lo, size_t k)
{
    return (f128_t)hi[k] + (lo ? (f128_t)lo[k] : (f128_t)0);
}

void sro_residuals_q(int n, const double *Ahi, const double *Alo, int lda, const double *Qhi,
                     const double *Qlo, int ldq, double *r_T, double *r_Q)
{
    size_t nn = (size_t)n * (size_t)n;
    f128_t *Q = (f128_t *)malloc(sizeof(f128_t) * nn), *M = (f128_t *)malloc(sizeof(f128_t) * nn);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) Q[IDX(i, j, n)] = q_of(Qhi, Qlo, IDX(i, j, ldq));
    /* M = A Q */
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            f128_t s = 0;
            for (int l = 0; l < n; ++l) s += q_of(Ahi, Alo, IDX(i, l, lda)) * Q[IDX(l, j, n)];
            M[IDX(i, j, n)] = s;
        }
    double st = 0.0, so = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : st, so)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            if (i > j) {
                f128_t s = 0;
                for (int l = 0; l < n; ++l) s += Q[IDX(l, i, n)] * M[IDX(l, j, n)];
                double v = (double)s;
                st += v * v;
            }
            if (i <= j) {
                f128_t s = 0;
                for (int l = 0; l < n; ++l) s += Q[IDX(l, i, n)] * Q[IDX(l, j, n)];
                if (i == j) s -= 1;
                double v = (double)s;
                so += (i == j ? 1.0 : 2.0) * v * v;
            }
        }
    double sa = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double a = (double)q_of(Ahi, Alo, IDX(i, j, lda));
            sa += a * a;
        }
    *r_T = sqrt(st) / sqrt(sa);
    *r_Q = sqrt(so);
    free(Q); free(M);
}

/* Sampled entries (rows[s], cols[s]) of Q^T A Q and of Q^T Q - I in 128-bit
 * floating point for double-double A and Q, returned as double-double pairs
 * (t_hi + t_lo, y_hi + y_lo). O(n^2) work per sample. */
void sro_sample_entries_q(int n, const double *Ahi, const double *Alo, int lda, const double *Qhi,
                          const double *Qlo, int ldq, int ns, const int *rows, const int *cols,
                          double *t_hi, double *t_lo, double *y_hi, double *y_lo)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < ns; ++s) {
        int i = rows[s], j = cols[s];
        f128_t t = 0;
        for (int l = 0; l < n; ++l) {
            f128_t aq = 0;
            for (int k = 0; k < n; ++k) aq += q_of(Ahi, Alo, IDX(l, k, lda)) * q_of(Qhi, Qlo, IDX(k, j, ldq));
            t += q_of(Qhi, Qlo, IDX(l, i, ldq)) * aq;
        }
        f128_t g = 0;
        for (int l = 0; l < n; ++l) g += q_of(Qhi, Qlo, IDX(l, i, ldq)) * q_of(Qhi, Qlo, IDX(l, j, ldq));
        if (i == j) g -= 1;
        t_hi[s] = (double)t;
        t_lo[s] = (double)(t - (f128_t)t_hi[s]);
        y_hi[s] = (double)g;
        y_lo[s] = (double)(g - (f128_t)y_hi[s]);
    }
}

/* ------------------------------------------------------------------ */
/* Alg. 2 for the real quasi-triangular Schur form (Sec. 3: real Schur
 * decompositions with 2 x 2 diagonal blocks holding complex-conjugate pairs).
 * blk[k] = 2 when a 2 x 2 diagonal block starts at row k (and blk[k + 1] = 0),
 * 1 for a 1 x 1 block. T holds the block upper triangular part (with the
 * coupling entries t_{k+1,k} of the 2 x 2 blocks), E the strictly block-lower
 * part, L receives the strictly block-lower solution of
 *     sbl(T L - L T) = -E
 * (sbl: the entries below the diagonal blocks). Block column J is taken left to
 * right and block rows I bottom to top, as Alg. 2 does entries:
 *     C_IJ = E_IJ + T(I, after I) L(after I, J) - L(I, before J) T(before J, J)
 * entry by entry in the order of Alg. 2's sums, then T_II X - X T_JJ = -C_IJ is
 * solved through its Kronecker matrix K = I (x) T_II - T_JJ^T (x) I of order
 * p q <= 4 (vec(X) column-major): its diagonal entries t_rr - t_cc are formed
 * from the high-precision diagonal dhp and rounded once, its other entries
 * are entries of T; Gaussian elimination with partial pivoting (the first
 * largest pivot) in the low precision, a zero pivot meaning a shared
 * eigenvalue (SRO_NONDISTINCT). With every block 1 x 1 this is Alg. 2 step
 * for step: x = (-c) / (t_ii - t_jj). */
#define SRO_ALG2_QUASI(NAME, R, ABS)                                                                  \
int NAME(int n, const R *T, int ldt, const R *E, int lde, const double *dhp, const int *blk,         \
         R *L, int ldl, double cap)                                                                  \
{                                                                                                    \
    for (int j = 0; j < n; ++j)                                                                      \
        for (int i = 0; i < n; ++i) L[IDX(i, j, ldl)] = 0;                                           \
    for (int j0 = 0; j0 < n; j0 += blk[j0]) {                                                        \
        const int q = blk[j0];                                                                       \
        if (q != 1 && q != 2) return SRO_NONFINITE;                                                  \
        /* block rows below the block column, bottom to top (the second row of  \
           a 2 x 2 block has blk = 0) */                                                             \
        for (int ib = n - 1; ib >= j0 + q;) {                                                        \
            const int i0 = blk[ib] == 0 ? ib - 1 : ib, p = blk[i0];                                  \
            ib = i0 - 1;                                                                             \
            R c[2][2];                                                                               \
            for (int r = 0; r < p; ++r)                                                              \
                for (int cc = 0; cc < q; ++cc) {                                                     \
                    const int i = i0 + r, j = j0 + cc;                                               \
                    R e = E[IDX(i, j, lde)];                                                         \
                    R s1 = 0, s2 = 0;                                                                \
                    for (int k = i0 + p; k < n; ++k) s1 += T[IDX(i, k, ldt)] * L[IDX(k, j, ldl)];    \
                    for (int k = 0; k < j0; ++k) s2 += L[IDX(i, k, ldl)] * T[IDX(k, j, ldt)];        \
                    c[r][cc] = e + s1 - s2;                                                          \
                }                                                                                    \
            /* Kronecker system K vec(X) = -vec(C), index r + cc p */                                \
            const int m = p * q;                                                                     \
            R K[4][4], rhs[4];                                                                       \
            for (int u = 0; u < m; ++u) {                                                            \
                const int ru = u % p, cu = u / p;                                                    \
                rhs[u] = -c[ru][cu];                                                                 \
                for (int v = 0; v < m; ++v) {                                                        \
                    const int rv = v % p, cv = v / p;                                                \
                    R kv = 0;                                                                        \
                    if (u == v) {                                                                    \
                        kv = (R)(dhp[i0 + ru] - dhp[j0 + cu]);                                       \
                    } else {                                                                         \
                        if (cu == cv) kv = T[IDX(i0 + ru, i0 + rv, ldt)];                            \
                        if (ru == rv) kv = -T[IDX(j0 + cv, j0 + cu, ldt)];                           \
                    }                                                                                \
                    K[u][v] = kv;                                                                    \
                }                                                                                    \
            }                                                                                        \
            for (int k = 0; k < m; ++k) {                                                            \
                int piv = k;                                                                         \
                for (int u = k + 1; u < m; ++u)                                                      \
                    if (ABS(K[u][k]) > ABS(K[piv][k])) piv = u;                                      \
                if (K[piv][k] == 0) return SRO_NONDISTINCT;                                          \
                if (piv != k) {                                                                      \
                    for (int v = 0; v < m; ++v) { R t = K[k][v]; K[k][v] = K[piv][v]; K[piv][v] = t; } \
                    R t = rhs[k]; rhs[k] = rhs[piv]; rhs[piv] = t;                                   \
                }                                                                                    \
                for (int u = k + 1; u < m; ++u) {                                                    \
                    const R f = K[u][k] / K[k][k];                                                   \
                    for (int v = k; v < m; ++v) K[u][v] -= f * K[k][v];                              \
                    rhs[u] -= f * rhs[k];                                                            \
                }                                                                                    \
            }                                                                                        \
            R x[4];                                                                                  \
            for (int u = m - 1; u >= 0; --u) {                                                       \
                R sacc = rhs[u];                                                                     \
                for (int v = u + 1; v < m; ++v) sacc -= K[u][v] * x[v];                              \
                x[u] = sacc / K[u][u];                                                               \
            }                                                                                        \
            for (int u = 0; u < m; ++u) {                                                            \
                R xv = x[u];                                                                         \
                if (cap > 0.0 && ABS(xv) > (R)cap) xv = 0;                                           \
                if (!isfinite(xv)) return SRO_NONFINITE;                                             \
                L[IDX(i0 + u % p, j0 + u / p, ldl)] = xv;                                            \
            }                                                                                        \
        }                                                                                            \
    }                                                                                                \
    return SRO_OK;                                                                                   \
}

SRO_ALG2_QUASI(sro_alg2_quasi_f64, double, fabs)
SRO_ALG2_QUASI(sro_alg2_quasi_f32, float, fabsf)
