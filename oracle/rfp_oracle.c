/*
 * Plain CPU oracle for Cholesky factorization, solution and inversion of a
 * symmetric positive definite matrix held in Rectangular Full Packed Format
 * (Gustavson, Wasniewski, Dongarra, Langou, "Rectangular Full Packed Format
 * for Cholesky's Algorithm: Factorization, Solution and Inversion").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the
 * CUDA library.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Everything here is written for obviousness, not speed: plain loops, IEEE
 * binary64, no blocking, no reordering beyond what each definition states.
 * It is compiled with -ffp-contract=off so that every a*b+c rounds twice, as
 * written.  OpenMP is used only across loop iterations that are independent
 * by definition (rows of one Cholesky column, right-hand sides, columns of
 * the identity); it changes no summation order.
 *
 * Functions and the passages they follow:
 *   oracle_pack / oracle_unpack  - Section 2 (Eq. 1 block split) and the
 *       element placements of Fig. 4 (N=7 lower, no transpose), Fig. 5
 *       (full -> RFPF, N=6,7) and Fig. 6 (all eight layouts).  The rectangle
 *       A_R is assembled from the blocks of A exactly as drawn; the TRANSR='T'
 *       layouts are the transpose of A_R (Section 2, "A_R^T resides in the
 *       transpose of array AR").
 *   oracle_potrf_rowmajor - textbook Cholesky A = L L^T (Eq. 2), column by
 *       column: l_jj = sqrt(a_jj - sum_p l_jp^2), l_ij = (a_ij - sum_p
 *       l_ip l_jp) / l_jj.  info = first j whose pivot is <= 0 or NaN.
 *   oracle_pftrf - Section 3: the factor of A in RFPF is L (UPLO='L') or
 *       U = L^T (UPLO='U') placed in the same layout, so it is computed as
 *       unpack -> Cholesky -> pack.
 *   oracle_pftrs - Section 4, Eqs. 5-8: L Y = B by forward substitution,
 *       then L^T X = Y by back substitution (U^T Y = B, U X = Y for 'U').
 *   oracle_pftri - Section 5, Eq. 9: W = L^{-1} by forward substitution on
 *       the columns of I, then A^{-1} = W^T W; its UPLO triangle is placed
 *       in the same layout.
 *   oracle_*_residual / backward error - error measures (Higham's normwise
 *       definitions, the reference the paper cites for stability), with
 *       inner products evaluated by the compensated Dot2 algorithm of Ogita,
 *       Rump and Oishi so that the measure itself is accurate to ~u^2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((int64_t)(i) + (int64_t)(j) * (int64_t)(ld))

static int is_lower(char uplo) { return uplo == 'L' || uplo == 'l'; }
static int is_trans(char transr) { return transr == 'T' || transr == 't'; }

/* Shape of A_R: LDAR rows and nc = ceil(N/2) columns (Section 7 text). */
static void ar_shape(int64_t n, int64_t *ldar, int64_t *nc)
{
    *ldar = (n % 2 == 1) ? n : n + 1;
    *nc = (n + 1) / 2;
}

/*
 * Assemble A_R (col-major, LDAR x nc) from the UPLO triangle of the
 * column-major full matrix A.  get_not_put selects direction:
 *   1: AR <- A   (TRTTF direction, used by pack)
 *   0: A  <- AR  (TFTTR direction, used by unpack)
 * The three placements per case are read off Figs. 4-6.
 */
static void ar_blocks(int get_not_put, char uplo, int64_t n, double *A,
                      int64_t lda, double *AR, int64_t ldar)
{
#define MOVE(r, c, i, j)                                          \
    do {                                                          \
        if (get_not_put) AR[IDX(r, c, ldar)] = A[IDX(i, j, lda)]; \
        else A[IDX(i, j, lda)] = AR[IDX(r, c, ldar)];             \
    } while (0)
    if (is_lower(uplo)) {
        if (n % 2 == 1) {
            /* N odd, lower (Fig. 4, Fig. 6.1 left): n1 = ceil(N/2).
             *  - lower triangle of A11 in AR(0:n1, 0:n1)
             *  - A21 (n2 x n1) below it, AR(n1:N, 0:n1)
             *  - upper triangle of A22^T in AR(0:n2, 1:n2+1)          */
            int64_t n1 = (n + 1) / 2, n2 = n - n1;
            for (int64_t j = 0; j < n1; ++j)
                for (int64_t i = j; i < n1; ++i) MOVE(i, j, i, j);
            for (int64_t j = 0; j < n1; ++j)
                for (int64_t i = 0; i < n2; ++i) MOVE(n1 + i, j, n1 + i, j);
            for (int64_t c = 0; c < n2; ++c)     /* A22^T(r,c) = A22(c,r) */
                for (int64_t r = 0; r <= c; ++r) MOVE(r, c + 1, n1 + c, n1 + r);
        } else {
            /* N = 2k even, lower (Fig. 5.2, Fig. 6.2 left):
             *  - upper triangle of A22^T in AR(0:k, 0:k)
             *  - lower triangle of A11 one row down, AR(1:k+1, 0:k)
             *  - A21 (k x k) below, AR(k+1:N+1, 0:k)                  */
            int64_t k = n / 2;
            for (int64_t c = 0; c < k; ++c)
                for (int64_t r = 0; r <= c; ++r) MOVE(r, c, k + c, k + r);
            for (int64_t j = 0; j < k; ++j)
                for (int64_t i = j; i < k; ++i) MOVE(1 + i, j, i, j);
            for (int64_t j = 0; j < k; ++j)
                for (int64_t i = 0; i < k; ++i) MOVE(k + 1 + i, j, k + i, j);
        }
    } else {
        /* Upper (Figs. 5.3, 5.4 and Fig. 6 right), n1 = floor(N/2):
         *  - A12 (n1 x n2) in AR(0:n1, 0:n2)
         *  - upper triangle of A22 in AR(n1:n1+n2, 0:n2)
         *  - lower triangle of A11^T one row lower, AR(n1+1:2n1+1, 0:n1) */
        int64_t n1 = n / 2, n2 = n - n1;
        for (int64_t c = 0; c < n2; ++c)
            for (int64_t r = 0; r < n1; ++r) MOVE(r, c, r, n1 + c);
        for (int64_t c = 0; c < n2; ++c)
            for (int64_t r = 0; r <= c; ++r) MOVE(n1 + r, c, n1 + r, n1 + c);
        for (int64_t c = 0; c < n1; ++c)   /* A11^T(r,c) = A11(c,r) */
            for (int64_t r = c; r < n1; ++r) MOVE(n1 + 1 + r, c, c, r);
    }
#undef MOVE
}

/* TRTTF: copy the UPLO triangle of A (col-major, lda) into arf. */
int oracle_pack(char transr, char uplo, int64_t n, const double *A, int64_t lda,
                double *arf)
{
    if (n <= 0) return 0;
    int64_t ldar, nc;
    ar_shape(n, &ldar, &nc);
    double *AR = (double *)calloc((size_t)(ldar * nc), sizeof(double));
    if (!AR) return -1;
    ar_blocks(1, uplo, n, (double *)A, lda, AR, ldar);
    for (int64_t c = 0; c < nc; ++c)
        for (int64_t r = 0; r < ldar; ++r) {
            if (is_trans(transr)) arf[c + r * nc] = AR[IDX(r, c, ldar)];
            else arf[r + c * ldar] = AR[IDX(r, c, ldar)];
        }
    free(AR);
    return 0;
}

/* TFTTR: write the UPLO triangle of A from arf; the other triangle is left
 * untouched. */
int oracle_unpack(char transr, char uplo, int64_t n, const double *arf,
                  double *A, int64_t lda)
{
    if (n <= 0) return 0;
    int64_t ldar, nc;
    ar_shape(n, &ldar, &nc);
    double *AR = (double *)malloc((size_t)(ldar * nc) * sizeof(double));
    if (!AR) return -1;
    for (int64_t c = 0; c < nc; ++c)
        for (int64_t r = 0; r < ldar; ++r)
            AR[IDX(r, c, ldar)] = is_trans(transr) ? arf[c + r * nc] : arf[r + c * ldar];
    ar_blocks(0, uplo, n, A, lda, AR, ldar);
    free(AR);
    return 0;
}

/* ---- dense helpers on a row-major n x n working array ------------------ */

/* Row-major symmetric working copy S[i*n+j] of the matrix stored in arf. */
static double *unpack_symmetric_rowmajor(char transr, char uplo, int64_t n,
                                         const double *arf)
{
    double *F = (double *)calloc((size_t)(n * n), sizeof(double)); /* col-major */
    double *S = (double *)malloc((size_t)(n * n) * sizeof(double));
    if (!F || !S) { free(F); free(S); return NULL; }
    oracle_unpack(transr, uplo, n, arf, F, n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            int take_ij = is_lower(uplo) ? (i >= j) : (i <= j);
            S[i * n + j] = take_ij ? F[IDX(i, j, n)] : F[IDX(j, i, n)];
        }
    free(F);
    return S;
}

/* Lower-triangular factor held in a row-major array: for UPLO='L' the stored
 * triangle is L; for UPLO='U' it is U and L = U^T. */
static double *unpack_factor_rowmajor(char transr, char uplo, int64_t n,
                                      const double *arf)
{
    double *F = (double *)calloc((size_t)(n * n), sizeof(double));
    double *L = (double *)calloc((size_t)(n * n), sizeof(double));
    if (!F || !L) { free(F); free(L); return NULL; }
    oracle_unpack(transr, uplo, n, arf, F, n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j)
            L[i * n + j] = is_lower(uplo) ? F[IDX(i, j, n)] : F[IDX(j, i, n)];
    free(F);
    return L;
}

/* Place the lower triangle of row-major M (L, or a symmetric matrix) into arf:
 * UPLO='L' stores M(i,j), i>=j; UPLO='U' stores A(i,j) = M(j,i), i<=j. */
static int pack_lower_rowmajor(char transr, char uplo, int64_t n,
                               const double *M, double *arf)
{
    double *F = (double *)calloc((size_t)(n * n), sizeof(double));
    if (!F) return -1;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j) {
            if (is_lower(uplo)) F[IDX(i, j, n)] = M[i * n + j];
            else F[IDX(j, i, n)] = M[i * n + j];
        }
    int rc = oracle_pack(transr, uplo, n, F, n, arf);
    free(F);
    return rc;
}

/*
 * Textbook Cholesky on a row-major array S (lower triangle used, overwritten
 * by L).  Column j: first the pivot l_jj, then every l_ij, i > j.  Returns 0
 * or the 1-based index of the first pivot that is <= 0 or NaN.
 */
int oracle_potrf_rowmajor(int64_t n, double *S)
{
    for (int64_t j = 0; j < n; ++j) {
        double s = S[j * n + j];
        for (int64_t p = 0; p < j; ++p) s -= S[j * n + p] * S[j * n + p];
        if (!(s > 0.0)) return (int)(j + 1);
        double ljj = sqrt(s);
        S[j * n + j] = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            double t = S[i * n + j];
            for (int64_t p = 0; p < j; ++p) t -= S[i * n + p] * S[j * n + p];
            S[i * n + j] = t / ljj;
        }
    }
    return 0;
}

/* PFTRF: overwrite arf with the Cholesky factor in the same layout. */
int oracle_pftrf(char transr, char uplo, int64_t n, double *arf)
{
    if (n <= 0) return 0;
    double *S = unpack_symmetric_rowmajor(transr, uplo, n, arf);
    if (!S) return -1;
    int info = oracle_potrf_rowmajor(n, S);
    if (info == 0) {
        for (int64_t i = 0; i < n; ++i)          /* keep the lower triangle */
            for (int64_t j = i + 1; j < n; ++j) S[i * n + j] = 0.0;
        pack_lower_rowmajor(transr, uplo, n, S, arf);
    }
    free(S);
    return info;
}

/* PFTRS: B (col-major n x nrhs, ldb) is overwritten by X with A X = B, A's
 * factor held in arf. */
int oracle_pftrs(char transr, char uplo, int64_t n, int64_t nrhs,
                 const double *arf, double *B, int64_t ldb)
{
    if (n <= 0 || nrhs <= 0) return 0;
    double *L = unpack_factor_rowmajor(transr, uplo, n, arf);
    if (!L) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < nrhs; ++c) {
        double *b = B + c * ldb;
        for (int64_t i = 0; i < n; ++i) {          /* L y = b */
            double t = b[i];
            for (int64_t p = 0; p < i; ++p) t -= L[i * n + p] * b[p];
            b[i] = t / L[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) {     /* L^T x = y */
            double t = b[i];
            for (int64_t p = i + 1; p < n; ++p) t -= L[p * n + i] * b[p];
            b[i] = t / L[i * n + i];
        }
    }
    free(L);
    return 0;
}

/* PFTRI: arf (holding the factor) is overwritten by the UPLO triangle of
 * A^{-1} = W^T W, W = L^{-1}.  info = first zero diagonal of the factor. */
int oracle_pftri(char transr, char uplo, int64_t n, double *arf)
{
    if (n <= 0) return 0;
    double *L = unpack_factor_rowmajor(transr, uplo, n, arf);
    if (!L) return -1;
    for (int64_t i = 0; i < n; ++i)
        if (L[i * n + i] == 0.0) { free(L); return (int)(i + 1); }
    double *W = (double *)calloc((size_t)(n * n), sizeof(double));
    double *M = (double *)calloc((size_t)(n * n), sizeof(double));
    if (!W || !M) { free(L); free(W); free(M); return -1; }
    /* column c of W solves L w = e_c (w_i = 0 for i < c) */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < n; ++c)
        for (int64_t i = c; i < n; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int64_t p = c; p < i; ++p) t -= L[i * n + p] * W[p * n + c];
            W[i * n + c] = t / L[i * n + i];
        }
    /* M = W^T W; M(i,j) = sum_{k >= max(i,j)} W(k,i) W(k,j), lower part */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j) {
            double t = 0.0;
            for (int64_t k = i; k < n; ++k) t += W[k * n + i] * W[k * n + j];
            M[i * n + j] = t;
        }
    pack_lower_rowmajor(transr, uplo, n, M, arf);
    free(L); free(W); free(M);
    return 0;
}

/* ---- error measures ---------------------------------------------------- */

/* Error-free transformations (Knuth TwoSum; TwoProduct via one fma). */
static inline void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b, z = x - a;
    *s = x;
    *e = (a - (x - z)) + (b - z);
}
static inline void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

/* Dot2 accumulator: value represented as hi + lo. */
typedef struct { double hi, lo; } acc2;
static inline void acc2_add_prod(acc2 *s, double a, double b)
{
    double p, ep, t, et;
    two_prod(a, b, &p, &ep);
    two_sum(s->hi, p, &t, &et);
    s->hi = t;
    s->lo += et + ep;
}
static inline double acc2_value(acc2 s) { return s.hi + s.lo; }

/* ||A - L L^T||_F / ||A||_F.  A: col-major symmetric (full, lda), L: col-major
 * lower triangular (full, ldl; upper part ignored). */
double oracle_factor_residual(int64_t n, const double *A, int64_t lda,
                              const double *L, int64_t ldl)
{
    double num = 0.0, den = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : num, den)
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
            int64_t r = i > j ? i : j, c = i > j ? j : i; /* symmetric entry */
            acc2 s = {A[IDX(r, c, lda)], 0.0};
            for (int64_t p = 0; p <= c; ++p)
                acc2_add_prod(&s, -L[IDX(r, p, ldl)], L[IDX(c, p, ldl)]);
            double d = acc2_value(s), a = A[IDX(r, c, lda)];
            num += d * d;
            den += a * a;
        }
    return den > 0 ? sqrt(num) / sqrt(den) : sqrt(num);
}

/* Normwise backward error of each column (Rigal-Gaches):
 * ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf); returns the max. */
double oracle_solve_backward_error(int64_t n, int64_t nrhs, const double *A,
                                   int64_t lda, const double *X, int64_t ldx,
                                   const double *B, int64_t ldb)
{
    double anorm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = 0.0;
        for (int64_t j = 0; j < n; ++j) r += fabs(A[IDX(i, j, lda)]);
        if (r > anorm) anorm = r;
    }
    double worst = 0.0;
    for (int64_t c = 0; c < nrhs; ++c) {
        double rmax = 0.0, xmax = 0.0, bmax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : rmax)
        for (int64_t i = 0; i < n; ++i) {
            acc2 s = {B[IDX(i, c, ldb)], 0.0};
            for (int64_t j = 0; j < n; ++j)
                acc2_add_prod(&s, -A[IDX(i, j, lda)], X[IDX(j, c, ldx)]);
            double r = fabs(acc2_value(s));
            if (r > rmax) rmax = r;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (fabs(X[IDX(i, c, ldx)]) > xmax) xmax = fabs(X[IDX(i, c, ldx)]);
            if (fabs(B[IDX(i, c, ldb)]) > bmax) bmax = fabs(B[IDX(i, c, ldb)]);
        }
        double den = anorm * xmax + bmax;
        double e = den > 0 ? rmax / den : rmax;
        if (e > worst) worst = e;
    }
    return worst;
}

/* ||A X - I||_1 / (||A||_1 ||X||_1), A and X col-major full symmetric. */
double oracle_inverse_residual(int64_t n, const double *A, int64_t lda,
                               const double *X, int64_t ldx)
{
    double anorm = 0.0, xnorm = 0.0, rnorm = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double sa = 0.0, sx = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            sa += fabs(A[IDX(i, j, lda)]);
            sx += fabs(X[IDX(i, j, ldx)]);
        }
        if (sa > anorm) anorm = sa;
        if (sx > xnorm) xnorm = sx;
    }
#pragma omp parallel for schedule(dynamic, 4) reduction(max : rnorm)
    for (int64_t j = 0; j < n; ++j) {
        double col = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            acc2 s = {(i == j) ? -1.0 : 0.0, 0.0};
            for (int64_t p = 0; p < n; ++p)
                acc2_add_prod(&s, A[IDX(i, p, lda)], X[IDX(p, j, ldx)]);
            col += fabs(acc2_value(s));
        }
        if (col > rnorm) rnorm = col;
    }
    double den = anorm * xnorm;
    return den > 0 ? rnorm / den : rnorm;
}
