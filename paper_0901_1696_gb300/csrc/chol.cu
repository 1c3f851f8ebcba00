// Blocked PFTRF, PFTRS and PFTRI on the RFP blocks (Sections 3, 4 and 5).
//
// Each routine is the paper's 2 x 2 block algorithm on the logical lower
// factor L = [L11 0; L21 L22] (T1 = L11, S = L21, T2 = L22 as views of the
// caller's array).  The full-format LAPACK / Level-3 BLAS calls of Fig. 4
// are replaced by tiled kernels with 64-wide diagonal tiles:
//   PFTRF: POTRF(T1); S <- S L11^{-T}; T2 <- T2 - S S^T; POTRF(T2)
//   PFTRS: L11 Y1 = B1; B2 -= L21 Y1; L22 Y2 = B2;
//          L22^T X2 = Y2; Y1 -= L21^T X2; L11^T X1 = Y1
//   PFTRI: W21 = -L22^{-1} L21 L11^{-1}; T1 <- W11^T W11 + W21^T W21;
//          S <- W22^T W21; T2 <- W22^T W22
// Every step works in place on the caller's array.  FP64 steps take small
// stream-ordered scratch from a library pool: the sync words of the one-launch
// kernels and, for triangles up to order 1024, PFTRI's W = L^{-1} and split-K
// chunks.  The in-place triangular products are ordered so that no kernel
// reads a tile another CTA of the same launch writes (right-looking blocked
// TRTRI and LAUUM below).
#include <algorithm>

#include "rfp_internal.cuh"

namespace rfp {

constexpr int64_t kNb = 64;   // diagonal tile width

#define RFP_TRY(x)                               \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) return e_;        \
    } while (0)

// op(V) Y = alpha X in place (V the m x m lower triangle, X an m x nrhs view,
// op = transpose when `trans`) as one launch of the block substitution
// (rfp_solve.cu) in FP64.  Returns false when it did not run (FP32, or no
// scratch, e.g. under stream capture): the caller then runs its multi-launch
// form.  *err receives the launch's result when it ran.
template <typename T>
bool solve_one_launch(cudaStream_t st, View<T> V, int64_t m, View<T> X, int64_t nrhs, bool trans,
                      T alpha, const int32_t *abort, cudaError_t *err)
{
    if constexpr (sizeof(T) == 8) {
        int32_t *sync = nullptr;
        if (solve_scratch_acquire(st, rfp_solve_sync_words(nrhs), &sync) != cudaSuccess) {
            (void)cudaGetLastError();   // the failed scratch request is not the caller's error
            return false;
        }
        const cudaError_t e = rfp_solve(st, V, V, V, m, 0, X, nrhs, trans, sync, abort, alpha);
        const cudaError_t e2 = solve_scratch_release(st, sync);
        *err = e != cudaSuccess ? e : e2;
        return true;
    }
    return false;
}

// C (lower m x m) = alpha A B^T + beta C with K-long operands: the SYRK of
// PFTRF step 3 and PFTRI's T1 update.  In FP64, when the lower 32 x 32 tiles
// are too few to fill the device twice over and K is long, K is split into
// chunks summed by a second kernel (pool scratch; not under graph capture):
// otherwise one CTA's serial K loop bounds the launch (n = 1001: 136 tiles
// of K = 501, about 124 us on one SM, against about 100 us for the whole
// product on all of them).
template <typename T>
cudaError_t update_lower(cudaStream_t st, View<T> C, View<T> A, View<T> B, int64_t m, int64_t K,
                         T alpha, T beta, const int32_t *abort)
{
    if constexpr (sizeof(T) == 8) {
        const int64_t t = (m + 31) / 32, tiles = t * (t + 1) / 2, sms = device_sm_count();
        if (m > 0 && tiles < 2 * sms && K >= 256) {
            int64_t splits = std::min<int64_t>(8, std::max<int64_t>(2, (4 * sms + tiles - 1) / tiles));
            splits = std::min<int64_t>(splits, K / 64);
            int32_t *buf = nullptr;
            if (solve_scratch_acquire(st, (size_t)(splits * m * m) * 2, &buf) == cudaSuccess) {
                const cudaError_t e = gemm_nt_splitk(st, C, A, B, m, m, K, alpha, beta, MASK_LOWER,
                                                     MASK_NONE, MASK_NONE, abort, (int)splits,
                                                     reinterpret_cast<double *>(buf));
                const cudaError_t e2 = solve_scratch_release(st, buf);
                return e != cudaSuccess ? e : e2;
            }
            (void)cudaGetLastError();   // the failed scratch request is not the caller's error
        }
    }
    return gemm_nt(st, C, A, B, m, m, K, alpha, beta, MASK_LOWER, MASK_NONE, MASK_NONE, abort);
}

// ---- triangle-level building blocks ----------------------------------------

// Right-looking blocked Cholesky of the m x m lower triangle V in place
// (LAPACK POTRF 'L' on one RFP triangle).  Failure index offset by `base`.
template <typename T>
cudaError_t potrf_blocked(cudaStream_t st, View<T> V, int64_t m, int32_t *info,
                                 int64_t base)
{
    if constexpr (sizeof(T) == 8) {
        // FP64: panel 0 as below, then one lookahead launch per panel step
        // (potrf_step.cu, panels potrf_step_width(m) wide); the multi-launch
        // form when no scratch can be had.
        int32_t *sync = nullptr;
        if (m > kNb && solve_scratch_acquire(st, potrf_step_sync_words(m), &sync) == cudaSuccess) {
            const int64_t pw = potrf_step_width(m);
            cudaError_t e = cudaMemsetAsync(sync, 0, potrf_step_sync_words(m) * sizeof(int32_t), st);
            if (e == cudaSuccess) e = potrf_tile(st, V, (int)pw, info, base);
            if (e == cudaSuccess)
                e = trsm_strip(st, V.sub(pw, 0), V, m - pw, (int)pw, 1, T(1), info);
            for (int64_t k0 = 0; e == cudaSuccess && k0 + pw < m; k0 += pw)
                e = potrf_step(st, V, m, k0, info, base, sync + 2 * (k0 / pw));
            const cudaError_t e2 = solve_scratch_release(st, sync);
            return e != cudaSuccess ? e : e2;
        }
        if (m > kNb) (void)cudaGetLastError();   // the failed scratch request is not the caller's error
    }
    for (int64_t k0 = 0; k0 < m; k0 += kNb) {
        const int64_t k1 = std::min(k0 + kNb, m), w = k1 - k0;
        RFP_TRY(potrf_tile(st, V.sub(k0, k0), (int)w, info, base + k0));
        if (k1 < m) {
            RFP_TRY(trsm_strip(st, V.sub(k1, k0), V.sub(k0, k0), m - k1, (int)w, 1, T(1), info));
            RFP_TRY(gemm_nt(st, V.sub(k1, k1), V.sub(k1, k0), V.sub(k1, k0), m - k1, m - k1, w,
                            T(-1), T(1), MASK_LOWER, MASK_NONE, MASK_NONE, info));
        }
    }
    return cudaSuccess;
}

// X (rows x m) <- X L^{-T}, L the m x m lower triangle V (right-looking).
template <typename T>
cudaError_t trsm_right_lower_trans(cudaStream_t st, View<T> X, int64_t rows, View<T> V,
                                          int64_t m, const int32_t *abort, bool unit)
{
    for (int64_t k0 = 0; k0 < m; k0 += kNb) {
        const int64_t k1 = std::min(k0 + kNb, m), w = k1 - k0;
        RFP_TRY(trsm_strip(st, X.sub(0, k0), V.sub(k0, k0), rows, (int)w, 1, T(1), abort, unit));
        if (k1 < m)
            RFP_TRY(gemm_nt(st, X.sub(0, k1), X.sub(0, k0), V.sub(k1, k0), rows, m - k1, w,
                            T(-1), T(1), MASK_NONE, MASK_NONE, MASK_NONE, abort));
    }
    return cudaSuccess;
}

// X (rows x m) <- alpha X L^{-1}, L the m x m lower triangle V (columns from
// the right).
template <typename T>
cudaError_t trsm_right_lower_notrans(cudaStream_t st, View<T> X, int64_t rows, View<T> V,
                                            int64_t m, T alpha, const int32_t *abort, bool unit)
{
    const int64_t nblk = (m + kNb - 1) / kNb;
    for (int64_t b = nblk - 1; b >= 0; --b) {
        const int64_t k0 = b * kNb, k1 = std::min(k0 + kNb, m), w = k1 - k0;
        const T a = (b == nblk - 1) ? alpha : T(1);
        RFP_TRY(trsm_strip(st, X.sub(0, k0), V.sub(k0, k0), rows, (int)w, 0, a, abort, unit));
        if (k0 > 0)   // X(:, 0:k0) = a X(:, 0:k0) - X_b L(k0:k1, 0:k0)
            RFP_TRY(gemm_nt(st, X, X.sub(0, k0), V.sub(k0, 0).t(), rows, k0, w, T(-1), a,
                            MASK_NONE, MASK_NONE, MASK_NONE, abort));
    }
    return cudaSuccess;
}

// L X = B in place, B (m x nrhs), L the m x m lower triangle V (forward).
template <typename T>
cudaError_t trsm_left_lower_notrans(cudaStream_t st, View<T> B, int64_t nrhs, View<T> V,
                                           int64_t m, const int32_t *abort, bool unit)
{
    for (int64_t k0 = 0; k0 < m; k0 += kNb) {
        const int64_t k1 = std::min(k0 + kNb, m), w = k1 - k0;
        // L_pp X_p = B_p  <=>  X_p^T L_pp^T = B_p^T
        RFP_TRY(trsm_strip(st, B.sub(k0, 0).t(), V.sub(k0, k0), nrhs, (int)w, 1, T(1), abort, unit));
        if (k1 < m)   // B(k1:m) -= L(k1:m, p) X_p
            RFP_TRY(gemm_nt(st, B.sub(k1, 0), V.sub(k1, k0), B.sub(k0, 0).t(), m - k1, nrhs, w,
                            T(-1), T(1), MASK_NONE, MASK_NONE, MASK_NONE, abort));
    }
    return cudaSuccess;
}

// L^T X = B in place, B (m x nrhs), L the m x m lower triangle V (backward).
template <typename T>
cudaError_t trsm_left_lower_trans(cudaStream_t st, View<T> B, int64_t nrhs, View<T> V,
                                         int64_t m, const int32_t *abort, bool unit)
{
    const int64_t nblk = (m + kNb - 1) / kNb;
    for (int64_t b = nblk - 1; b >= 0; --b) {
        const int64_t k0 = b * kNb, k1 = std::min(k0 + kNb, m), w = k1 - k0;
        // L_pp^T X_p = B_p  <=>  X_p^T L_pp = B_p^T
        RFP_TRY(trsm_strip(st, B.sub(k0, 0).t(), V.sub(k0, k0), nrhs, (int)w, 0, T(1), abort, unit));
        if (k0 > 0)   // B(0:k0) -= L(p, 0:k0)^T X_p
            RFP_TRY(gemm_nt(st, B, V.sub(k0, 0).t(), B.sub(k0, 0).t(), k0, nrhs, w, T(-1), T(1),
                            MASK_NONE, MASK_NONE, MASK_NONE, abort));
    }
    return cudaSuccess;
}

// Triangles of order kNb < m <= kSmallInverse are inverted (FP64, outside
// graph capture) by one launch of the block substitution L W = I into pool
// scratch, and their W^T W formed by one split-K product: each a fixed
// number of launches instead of a serial chain of them per 64-wide panel,
// which bounds these orders on GB300's FP64 pipe.
constexpr int64_t kSmallInverse = 1024;

// W = L^{-1}: W = I in scratch, L W = I with a lower-triangular right-hand
// side (solution lower triangular), W's lower triangle back into V.  Returns
// false when it did not run (FP32, order out of range, no scratch); *err
// receives the result when it ran.
template <typename T>
bool trtri_by_solve(cudaStream_t st, View<T> V, int64_t m, const int32_t *abort, cudaError_t *err)
{
    if constexpr (sizeof(T) == 8) {
        if (m <= kNb || m > kSmallInverse) return false;
        const size_t wwords = (size_t)(m * m) * 2, swords = rfp_solve_sync_words(m);
        int32_t *buf = nullptr;
        if (solve_scratch_acquire(st, wwords + swords, &buf) != cudaSuccess) {
            (void)cudaGetLastError();   // the failed scratch request is not the caller's error
            return false;
        }
        View<double> W{reinterpret_cast<double *>(buf), 1, m};
        cudaError_t e = identity_fill(st, W, m, abort);
        if (e == cudaSuccess)
            e = rfp_solve(st, V, V, V, m, 0, W, m, false, buf + wwords, abort, 1.0, true);
        if (e == cudaSuccess) e = lower_copy(st, V, W, m, abort);
        const cudaError_t e2 = solve_scratch_release(st, buf);
        *err = e != cudaSuccess ? e : e2;
        return true;
    }
    return false;
}

// Lower triangle of W^T W in place, as one split-K product: C(i, j) =
// sum_{k >= max(i, j)} W(k, i) W(k, j) (both operands W^T, masked to k >= row),
// the chunk products into scratch, their sum into V's lower triangle by the
// second kernel.  Same conditions as trtri_by_solve.
template <typename T>
bool lauum_by_product(cudaStream_t st, View<T> V, int64_t m, const int32_t *abort, cudaError_t *err)
{
    if constexpr (sizeof(T) == 8) {
        if (m <= kNb || m > kSmallInverse) return false;
        const int splits = (int)std::min<int64_t>(8, std::max<int64_t>(2, (m + 127) / 128));
        int32_t *buf = nullptr;
        if (solve_scratch_acquire(st, (size_t)splits * (size_t)(m * m) * 2, &buf) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        const cudaError_t e = gemm_nt_splitk(st, V, V.t(), V.t(), m, m, m, 1.0, 0.0, MASK_LOWER,
                                             MASK_UPPER, MASK_UPPER, abort, splits,
                                             reinterpret_cast<double *>(buf));
        const cudaError_t e2 = solve_scratch_release(st, buf);
        *err = e != cudaSuccess ? e : e2;
        return true;
    }
    return false;
}

// In-place W = L^{-1} on an m x m lower triangle V.  Right-looking over the
// block columns p: with X = C_{p-1}^{-1} ... C_1^{-1} held where L was
// consumed, step p applies C_p^{-1} (block column p of L):
//   W_pp = L_pp^{-1};  X(p, :p) <- W_pp X(p, :p);
//   X(i>p, :p) -= L(i, p) X(p, :p);  X(i>p, p) <- -L(i, p) W_pp.
template <typename T>
cudaError_t trtri_blocked(cudaStream_t st, View<T> V, int64_t m, const int32_t *abort)
{
    cudaError_t err = cudaSuccess;
    if (trtri_by_solve(st, V, m, abort, &err)) return err;
    for (int64_t k0 = 0; k0 < m; k0 += kNb) {
        const int64_t k1 = std::min(k0 + kNb, m), w = k1 - k0;
        RFP_TRY(trtri_tile(st, V.sub(k0, k0), (int)w, abort));
        if (k0 > 0)
            RFP_TRY(gemm_nt(st, V.sub(k0, 0), V.sub(k0, k0), V.sub(k0, 0).t(), w, k0, w, T(1),
                            T(0), MASK_NONE, MASK_LOWER, MASK_NONE, abort, GEMM_INPLACE_COLS));
        if (k1 < m) {
            if (k0 > 0)
                RFP_TRY(gemm_nt(st, V.sub(k1, 0), V.sub(k1, k0), V.sub(k0, 0).t(), m - k1, k0, w,
                                T(-1), T(1), MASK_NONE, MASK_NONE, MASK_NONE, abort));
            RFP_TRY(gemm_nt(st, V.sub(k1, k0), V.sub(k1, k0), V.sub(k0, k0).t(), m - k1, w, w,
                            T(-1), T(0), MASK_NONE, MASK_NONE, MASK_UPPER, abort, GEMM_INPLACE_ROWS));
        }
    }
    return cudaSuccess;
}

// In-place lower triangle of W^T W on an m x m lower triangle V holding W.
// Block row q contributes W(q, :)^T W(q, :) to rows <= q; processed in
// increasing q, rows < q already hold partial sums, row q still holds W.
template <typename T>
cudaError_t lauum_blocked(cudaStream_t st, View<T> V, int64_t m, const int32_t *abort)
{
    cudaError_t err = cudaSuccess;
    if (lauum_by_product(st, V, m, abort, &err)) return err;
    for (int64_t k0 = 0; k0 < m; k0 += kNb) {
        const int64_t k1 = std::min(k0 + kNb, m), w = k1 - k0;
        if (k0 > 0) {
            RFP_TRY(gemm_nt(st, V, V.sub(k0, 0).t(), V.sub(k0, 0).t(), k0, k0, w, T(1), T(1),
                            MASK_LOWER, MASK_NONE, MASK_NONE, abort));
            RFP_TRY(gemm_nt(st, V.sub(k0, 0), V.sub(k0, k0).t(), V.sub(k0, 0).t(), w, k0, w,
                            T(1), T(0), MASK_NONE, MASK_UPPER, MASK_NONE, abort, GEMM_INPLACE_COLS));
        }
        RFP_TRY(lauum_tile(st, V.sub(k0, k0), (int)w, abort));
    }
    return cudaSuccess;
}

// S <- -L22^{-1} S L11^{-1} (Sec. 5, W21 = -W22 L21 W11, reading R9): first
// S <- -S L11^{-1}, i.e. L11^T S^T = -S^T, then S <- L22^{-1} S.  In FP64
// each is one launch of the block substitution.
template <typename T>
cudaError_t w21_solves(cudaStream_t st, View<T> t1, View<T> s, View<T> t2, int64_t n1, int64_t n2,
                       const int32_t *info)
{
    cudaError_t e = cudaSuccess;
    if (solve_one_launch(st, t1, n1, s.t(), n2, true, T(-1), info, &e)) RFP_TRY(e);
    else RFP_TRY(trsm_right_lower_notrans(st, s, n2, t1, n1, T(-1), info));
    if (solve_one_launch(st, t2, n2, s, n1, false, T(1), info, &e)) RFP_TRY(e);
    else RFP_TRY(trsm_left_lower_notrans(st, s, n1, t2, n2, info));
    return cudaSuccess;
}

// ---- the three routines --------------------------------------------------------

template <typename T>
cudaError_t pftrf_impl(cudaStream_t st, const Layout &L, T *arf, int32_t *info)
{
    View<T> t1 = block_view(arf, L, L.t1), s = block_view(arf, L, L.s), t2 = block_view(arf, L, L.t2);
    stage_begin(st);
    RFP_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), st));
    // step 1: L11 L11^T = A11
    RFP_TRY(potrf_blocked(st, t1, L.n1, info, 0));
    stage_mark(st, "pftrf.potrf_t1");
    if (L.n2 > 0 && L.n1 > 0) {
        // step 2: L21 L11^T = A21, i.e. L11 L21^T = A21^T: in FP64 one launch
        // of the block substitution with T1 and the n2 columns of S^T
        // (rfp_solve.cu); the multi-launch form when no scratch can be had.
        cudaError_t e = cudaSuccess;
        if (solve_one_launch(st, t1, L.n1, s.t(), L.n2, false, T(1), info, &e)) RFP_TRY(e);
        else RFP_TRY(trsm_right_lower_trans(st, s, L.n2, t1, L.n1, info));
        stage_mark(st, "pftrf.trsm_s");
        // step 3: A22 <- A22 - L21 L21^T (lower triangle of T2)
        RFP_TRY(update_lower(st, t2, s, s, L.n2, L.n1, T(-1), T(1), info));
        stage_mark(st, "pftrf.syrk_t2");
    }
    // step 4: L22 L22^T = A22
    RFP_TRY(potrf_blocked(st, t2, L.n2, info, L.n1));
    stage_mark(st, "pftrf.potrf_t2");
    return cudaSuccess;
}

template <typename T>
cudaError_t pftrs_impl(cudaStream_t st, const Layout &L, const T *arf_c, T *Bp, int64_t ldb,
                       int64_t nrhs)
{
    T *arf = const_cast<T *>(arf_c);   // read only below
    View<T> t1 = block_view(arf, L, L.t1), s = block_view(arf, L, L.s), t2 = block_view(arf, L, L.t2);
    View<T> B{Bp, 1, ldb};
    View<T> B1 = B, B2 = B.sub(L.n1, 0);
    stage_begin(st);
    if constexpr (sizeof(T) == 8) {
        // One launch per direction over the whole factor (rfp_solve.cu);
        // the multi-launch form below when no scratch can be had (stream
        // capture).
        int32_t *sync = nullptr;
        if (solve_scratch_acquire(st, rfp_solve_sync_words(nrhs), &sync) == cudaSuccess) {
            cudaError_t e = rfp_solve(st, t1, s, t2, L.n1, L.n2, B, nrhs, false, sync);
            stage_mark(st, "pftrs.forward");
            if (e == cudaSuccess) e = rfp_solve(st, t1, s, t2, L.n1, L.n2, B, nrhs, true, sync);
            stage_mark(st, "pftrs.backward");
            const cudaError_t e2 = solve_scratch_release(st, sync);
            return e != cudaSuccess ? e : e2;
        }
        (void)cudaGetLastError();   // the failed scratch request is not the caller's error
    }
    // L Y = B
    RFP_TRY(trsm_left_lower_notrans(st, B1, nrhs, t1, L.n1, (const int32_t *)nullptr));
    RFP_TRY(gemm_nt(st, B2, s, B1.t(), L.n2, nrhs, L.n1, T(-1), T(1), MASK_NONE, MASK_NONE,
                    MASK_NONE, (const int32_t *)nullptr));
    RFP_TRY(trsm_left_lower_notrans(st, B2, nrhs, t2, L.n2, (const int32_t *)nullptr));
    stage_mark(st, "pftrs.forward");
    // L^T X = Y
    RFP_TRY(trsm_left_lower_trans(st, B2, nrhs, t2, L.n2, (const int32_t *)nullptr));
    RFP_TRY(gemm_nt(st, B1, s.t(), B2.t(), L.n1, nrhs, L.n2, T(-1), T(1), MASK_NONE, MASK_NONE,
                    MASK_NONE, (const int32_t *)nullptr));
    RFP_TRY(trsm_left_lower_trans(st, B1, nrhs, t1, L.n1, (const int32_t *)nullptr));
    stage_mark(st, "pftrs.backward");
    return cudaSuccess;
}

template <typename T>
cudaError_t pftri_impl(cudaStream_t st, const Layout &L, T *arf, int32_t *info)
{
    View<T> t1 = block_view(arf, L, L.t1), s = block_view(arf, L, L.s), t2 = block_view(arf, L, L.t2);
    stage_begin(st);
    RFP_TRY(check_diag(st, t1, L.n1, t2, L.n2, info));
    if (L.n1 > 0 && L.n2 > 0) {
        // W21 = -L22^{-1} L21 L11^{-1}: two in-place solves with the factor
        RFP_TRY(w21_solves(st, t1, s, t2, L.n1, L.n2, info));
    }
    stage_mark(st, "pftri.w21");
    // T1 <- W11^T W11 + W21^T W21
    RFP_TRY(trtri_blocked(st, t1, L.n1, info));
    stage_mark(st, "pftri.trtri_t1");
    RFP_TRY(lauum_blocked(st, t1, L.n1, info));
    stage_mark(st, "pftri.lauum_t1");
    if (L.n1 > 0 && L.n2 > 0) {
        RFP_TRY(update_lower(st, t1, s.t(), s.t(), L.n1, L.n2, T(1), T(1), info));
        stage_mark(st, "pftri.syrk_t1");
        // S <- W22^T W21 = L22^{-T} W21 (T2 still holds L22)
        cudaError_t e = cudaSuccess;
        if (solve_one_launch(st, t2, L.n2, s, L.n1, true, T(1), info, &e)) RFP_TRY(e);
        else RFP_TRY(trsm_left_lower_trans(st, s, L.n1, t2, L.n2, info));
        stage_mark(st, "pftri.trmm_s");
    }
    // T2 <- W22^T W22
    RFP_TRY(trtri_blocked(st, t2, L.n2, info));
    stage_mark(st, "pftri.trtri_t2");
    RFP_TRY(lauum_blocked(st, t2, L.n2, info));
    stage_mark(st, "pftri.lauum_t2");
    return cudaSuccess;
}

// ---- the rest of the LAPACK 3.2 RFP routine set (Table lapack) --------------

// TFTRI: the inverse of the triangle in place, i.e. stage 1 of PFTRI
// (Section 5): W11 = L11^{-1}, W21 = -W22 L21 W11, W22 = L22^{-1}.
template <typename T>
cudaError_t tftri_impl(cudaStream_t st, const Layout &L, T *arf, int32_t *info)
{
    View<T> t1 = block_view(arf, L, L.t1), s = block_view(arf, L, L.s), t2 = block_view(arf, L, L.t2);
    RFP_TRY(check_diag(st, t1, L.n1, t2, L.n2, info));
    if (L.n1 > 0 && L.n2 > 0) RFP_TRY(w21_solves(st, t1, s, t2, L.n1, L.n2, info));
    RFP_TRY(trtri_blocked(st, t1, L.n1, info));
    return trtri_blocked(st, t2, L.n2, info);
}

// SFRK: with op(A) split at n1 into A1 (rows 0..n1) and A2, the three blocks
// of C are C11 = alpha A1 A1^T + beta C11 (lower), C21 = alpha A2 A1^T +
// beta C21 and C22 = alpha A2 A2^T + beta C22 (lower): the paper's SYRK /
// GEMM step 3 on each block.
template <typename T>
cudaError_t sfrk_impl(cudaStream_t st, const Layout &L, T *arf, View<T> opA, int64_t k, T alpha,
                      T beta)
{
    View<T> t1 = block_view(arf, L, L.t1), s = block_view(arf, L, L.s), t2 = block_view(arf, L, L.t2);
    const int32_t *none = nullptr;
    View<T> A1 = opA, A2 = opA.sub(L.n1, 0);
    if (L.n1 > 0)
        RFP_TRY(gemm_nt(st, t1, A1, A1, L.n1, L.n1, k, alpha, beta, MASK_LOWER, MASK_NONE,
                        MASK_NONE, none));
    if (L.n1 > 0 && L.n2 > 0)
        RFP_TRY(gemm_nt(st, s, A2, A1, L.n2, L.n1, k, alpha, beta, MASK_NONE, MASK_NONE, MASK_NONE,
                        none));
    if (L.n2 > 0)
        RFP_TRY(gemm_nt(st, t2, A2, A2, L.n2, L.n2, k, alpha, beta, MASK_LOWER, MASK_NONE,
                        MASK_NONE, none));
    return cudaSuccess;
}

// TFSM: Section 4's block substitutions with an arbitrary right-hand-side
// block, from either side.  alpha is applied first (alpha = 0: B = 0).
template <typename T>
cudaError_t tfsm_impl(cudaStream_t st, const Layout &L, const T *arf_c, bool left, bool opT,
                      bool unit, int64_t m, int64_t nc, T alpha, T *Bp, int64_t ldb)
{
    T *arf = const_cast<T *>(arf_c);   // read only below
    View<T> t1 = block_view(arf, L, L.t1), s = block_view(arf, L, L.s), t2 = block_view(arf, L, L.t2);
    View<T> B{Bp, 1, ldb};
    const int32_t *none = nullptr;
    if (m <= 0 || nc <= 0) return cudaSuccess;
    if (alpha != T(1))   // B = alpha B (a K = 0 product: C = 0 + beta C)
        RFP_TRY(gemm_nt(st, B, B, B, m, nc, 0, T(0), alpha, MASK_NONE, MASK_NONE, MASK_NONE, none));
    if (alpha == T(0)) return cudaSuccess;
    const int64_t n1 = L.n1, n2 = L.n2;
    if (left) {   // op(A) is m x m; B1 = rows [0, n1)
        View<T> B1 = B, B2 = B.sub(n1, 0);
        if (!opT) {   // L X = B
            RFP_TRY(trsm_left_lower_notrans(st, B1, nc, t1, n1, none, unit));
            if (n1 > 0 && n2 > 0)
                RFP_TRY(gemm_nt(st, B2, s, B1.t(), n2, nc, n1, T(-1), T(1), MASK_NONE, MASK_NONE,
                                MASK_NONE, none));
            RFP_TRY(trsm_left_lower_notrans(st, B2, nc, t2, n2, none, unit));
        } else {      // L^T X = B
            RFP_TRY(trsm_left_lower_trans(st, B2, nc, t2, n2, none, unit));
            if (n1 > 0 && n2 > 0)
                RFP_TRY(gemm_nt(st, B1, s.t(), B2.t(), n1, nc, n2, T(-1), T(1), MASK_NONE,
                                MASK_NONE, MASK_NONE, none));
            RFP_TRY(trsm_left_lower_trans(st, B1, nc, t1, n1, none, unit));
        }
    } else {      // op(A) is nc x nc; B1 = columns [0, n1)
        View<T> B1 = B, B2 = B.sub(0, n1);
        if (!opT) {   // X L = B: X2 = B2 L22^{-1}, B1 -= X2 L21, X1 = B1 L11^{-1}
            RFP_TRY(trsm_right_lower_notrans(st, B2, m, t2, n2, T(1), none, unit));
            if (n1 > 0 && n2 > 0)
                RFP_TRY(gemm_nt(st, B1, B2, s.t(), m, n1, n2, T(-1), T(1), MASK_NONE, MASK_NONE,
                                MASK_NONE, none));
            RFP_TRY(trsm_right_lower_notrans(st, B1, m, t1, n1, T(1), none, unit));
        } else {      // X L^T = B: X1 = B1 L11^{-T}, B2 -= X1 L21^T, X2 = B2 L22^{-T}
            RFP_TRY(trsm_right_lower_trans(st, B1, m, t1, n1, none, unit));
            if (n1 > 0 && n2 > 0)
                RFP_TRY(gemm_nt(st, B2, B1, s, m, n2, n1, T(-1), T(1), MASK_NONE, MASK_NONE,
                                MASK_NONE, none));
            RFP_TRY(trsm_right_lower_trans(st, B2, m, t2, n2, none, unit));
        }
    }
    return cudaSuccess;
}

#define RFP_SURFACE_ORCH_INST(T)                                                                  \
    template cudaError_t tftri_impl<T>(cudaStream_t, const Layout &, T *, int32_t *);             \
    template cudaError_t sfrk_impl<T>(cudaStream_t, const Layout &, T *, View<T>, int64_t, T, T); \
    template cudaError_t tfsm_impl<T>(cudaStream_t, const Layout &, const T *, bool, bool, bool,  \
                                      int64_t, int64_t, T, T *, int64_t);
RFP_SURFACE_ORCH_INST(float)
RFP_SURFACE_ORCH_INST(double)
#undef RFP_SURFACE_ORCH_INST


#define RFP_BLOCKED_INST(T)                                                                      \
    template cudaError_t potrf_blocked<T>(cudaStream_t, View<T>, int64_t, int32_t *, int64_t);     \
    template cudaError_t trsm_right_lower_trans<T>(cudaStream_t, View<T>, int64_t, View<T>, int64_t, \
                                                   const int32_t *, bool);                         \
    template cudaError_t trsm_right_lower_notrans<T>(cudaStream_t, View<T>, int64_t, View<T>,      \
                                                     int64_t, T, const int32_t *, bool);           \
    template cudaError_t trsm_left_lower_notrans<T>(cudaStream_t, View<T>, int64_t, View<T>,       \
                                                    int64_t, const int32_t *, bool);               \
    template cudaError_t trsm_left_lower_trans<T>(cudaStream_t, View<T>, int64_t, View<T>, int64_t, \
                                                  const int32_t *, bool);
RFP_BLOCKED_INST(float)
RFP_BLOCKED_INST(double)
#undef RFP_BLOCKED_INST

template cudaError_t pftrf_impl<double>(cudaStream_t, const Layout &, double *, int32_t *);
template cudaError_t pftrf_impl<float>(cudaStream_t, const Layout &, float *, int32_t *);
template cudaError_t pftrs_impl<double>(cudaStream_t, const Layout &, const double *, double *,
                                        int64_t, int64_t);
template cudaError_t pftrs_impl<float>(cudaStream_t, const Layout &, const float *, float *,
                                       int64_t, int64_t);
template cudaError_t pftri_impl<double>(cudaStream_t, const Layout &, double *, int32_t *);
template cudaError_t pftri_impl<float>(cudaStream_t, const Layout &, float *, int32_t *);

}  // namespace rfp
