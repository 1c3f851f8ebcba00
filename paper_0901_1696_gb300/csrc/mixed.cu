// Mixed-precision solve of A X = B for an SPD matrix held in FP64 RFPF:
// factor a low-precision copy, refine in FP64 (the precision direction of
// the project; the method of Sections 3-4 is unchanged apart from the
// precision of its Level-3 steps).
//
//   1. W = fl32(A) (lower triangle of the logical matrix, FP32, full storage)
//   2. W = L L^T in FP32 storage: the blocked Cholesky of Section 3 on W by
//      512-wide panels (factor_panels) with the SYRK updates in
//        RFP_PREC_FP32: FP32 FMA (SIMT), the s-precision kernels,
//        RFP_PREC_TF32 / RFP_PREC_BF16: tcgen05 tensor cores (rfp_ssyrk_tc's
//        kernel) on 512-wide panels converted to TF32 / BF16, FP32 accumulate;
//        RFP_PREC_TF32X3: the same kernel on a split panel P = hi + lo (both
//        TF32), C -= hi hi^T + lo hi^T + hi lo^T (three products, one launch);
//        RFP_PREC_BF16X6: P = hi + mid + lo (all BF16), the six products
//        above 2^-24 in one kind::f16 launch;
//      the diagonal blocks and the panel solves stay in FP32.
//   3. X = 0, R = B; repeat: D = (L L^T)^{-1} fl32(R) (FP32 block solves of
//      Section 4, one launch each, the 128-wide diagonal blocks applied as
//      inverses formed once),
//      X += D (FP64), R = B - A X with A read from the FP64 RFP array (FP64),
//      until max_j ||r_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf) <= tol
//      or max_iter steps.  Convergence is decided on the device: every later
//      kernel of the fixed launch sequence returns at once.
#include "mixed_internal.cuh"

namespace rfp {

namespace {
constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
int64_t ldw_for(int64_t n) { return (n + 31) / 32 * 32; }
size_t panel_elem(int prec) { return (prec == RFP_PREC_BF16 || prec == RFP_PREC_BF16X6) ? 2 : 4; }
size_t inv_elems(int64_t n) { return (size_t)((n + kInvBlock - 1) / kInvBlock) * kInvBlock * kInvBlock; }
}  // namespace

size_t mixed_workspace_bytes(int64_t n, int64_t nrhs, int prec)
{
    size_t b = 0;
    b += up((size_t)ldw_for(n) * (size_t)n * sizeof(float));                  // W
    b += up(inv_elems(n) * sizeof(float));                                    // Inv
    if (prec != RFP_PREC_FP32) b += up((size_t)n * panel_cols(prec) * panel_elem(prec));   // P
    b += up((size_t)n * (size_t)nrhs * sizeof(double));                       // R
    b += up((size_t)n * (size_t)nrhs * sizeof(float));                        // D
    b += up((size_t)nrhs * sizeof(double));                                   // berr
    b += up(sizeof(double)) + up(sizeof(int32_t)) + up(sizeof(int32_t));      // anorm, stop, tc_err
    b += up(wavefront_sync_words(n, nrhs) * sizeof(int32_t));                 // solve sync
    if (residual_splits(n) > 1)
        b += up((size_t)residual_splits(n) * (size_t)n * (size_t)nrhs * sizeof(double));
    return b;
}

bool mixed_carve(void *work, size_t bytes, int64_t n, int64_t nrhs, int prec, MixedWork *w)
{
    if (reinterpret_cast<uintptr_t>(work) % kAlign) return false;
    if (bytes < mixed_workspace_bytes(n, nrhs, prec)) return false;
    char *p = static_cast<char *>(work);
    w->ldw = ldw_for(n);
    w->W = reinterpret_cast<float *>(p);
    p += up((size_t)w->ldw * (size_t)n * sizeof(float));
    w->Inv = reinterpret_cast<float *>(p);
    p += up(inv_elems(n) * sizeof(float));
    w->P = nullptr;
    if (prec != RFP_PREC_FP32) {
        w->P = p;
        p += up((size_t)n * panel_cols(prec) * panel_elem(prec));
    }
    w->R = reinterpret_cast<double *>(p);
    p += up((size_t)n * (size_t)nrhs * sizeof(double));
    w->D = reinterpret_cast<float *>(p);
    p += up((size_t)n * (size_t)nrhs * sizeof(float));
    w->berr = reinterpret_cast<double *>(p);
    p += up((size_t)nrhs * sizeof(double));
    w->anorm = reinterpret_cast<double *>(p);
    p += up(sizeof(double));
    w->stop = reinterpret_cast<int32_t *>(p);
    p += up(sizeof(int32_t));
    w->tc_err = reinterpret_cast<int32_t *>(p);
    p += up(sizeof(int32_t));
    w->sync = reinterpret_cast<int32_t *>(p);
    p += up(wavefront_sync_words(n, nrhs) * sizeof(int32_t));
    w->splits = residual_splits(n);
    w->splitk = w->splits > 1 ? reinterpret_cast<double *>(p) : nullptr;
    return true;
}

#define RFP_TRY(x)                        \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

// Blocked right-looking Cholesky of the FP32 working matrix by 512-wide
// panels (Section 3's algorithm on W).  Per panel:
//   1. Cholesky of the diagonal block (blocked by 64-wide tiles);
//   2. inverses of its 128-wide diagonal blocks, kept in w.Inv (they serve
//      the panel solve here and the refinement's block solves later);
//   3. the panel solve L21 = A21 L11^{-T} by 128-column blocks: subtract the
//      finished columns (GEMM), then multiply by the block's inverse (an
//      in-place GEMM): every step is one wide launch;
//   4. the trailing update A22 -= L21 L21^T: FP32 FMA for RFP_PREC_FP32,
//      else on the tensor cores from the converted or split panel.
static cudaError_t factor_panels(cudaStream_t st, View<float> W, int64_t n, int prec,
                                 const MixedWork &w, int32_t *info)
{
    for (int64_t j0 = 0; j0 < n; j0 += kMixedPanel) {
        const int64_t j1 = std::min(j0 + kMixedPanel, n), nb = j1 - j0;
        View<float> L11 = W.sub(j0, j0);
        float *inv0 = w.Inv + (j0 / kInvBlock) * kInvBlock * kInvBlock;
        RFP_TRY(potrf_blocked<float>(st, L11, nb, info, j0));
        RFP_TRY(inv_diag_blocks(st, L11, nb, inv0, info));
        if (j1 >= n) break;
        const int64_t m = n - j1;
        View<float> X = W.sub(j1, j0);
        for (int64_t c0 = 0; c0 < nb; c0 += kInvBlock) {
            const int64_t cw = std::min(kInvBlock, nb - c0);
            if (c0 > 0)   // X_c -= X(:, 0:c0) L11(c0:c0+cw, 0:c0)^T
                RFP_TRY(gemm_nt(st, X.sub(0, c0), X, L11.sub(c0, 0), m, cw, c0, -1.0f, 1.0f,
                                MASK_NONE, MASK_NONE, MASK_NONE, info));
            // X_c <- X_c W_c^T with W_c = L11(c0.., c0..)^{-1} (lower): in place
            View<float> Wc{inv0 + (c0 / kInvBlock) * kInvBlock * kInvBlock, 1, kInvBlock};
            RFP_TRY(gemm_nt(st, X.sub(0, c0), X.sub(0, c0), Wc, m, cw, cw, 1.0f, 0.0f, MASK_NONE,
                            MASK_NONE, MASK_LOWER, info, GEMM_INPLACE_ROWS));
        }
        if (prec == RFP_PREC_FP32) {
            RFP_TRY(gemm_nt(st, W.sub(j1, j1), X, X, m, m, nb, -1.0f, 1.0f, MASK_LOWER, MASK_NONE,
                            MASK_NONE, info));
            continue;
        }
        // panel -> K-contiguous low-precision copy P (row r, column k at P[r*pitch + k])
        if (prec == RFP_PREC_BF16) {
            View<__nv_bfloat16> P{static_cast<__nv_bfloat16 *>(w.P), kMixedPanel, 1};
            RFP_TRY((convert<float, __nv_bfloat16>(st, X, P, m, nb, false, info)));
        } else if (prec == RFP_PREC_TF32) {
            View<float> P{static_cast<float *>(w.P), kMixedPanel, 1};
            RFP_TRY((convert<float, float>(st, X, P, m, nb, false, info)));
        } else if (prec == RFP_PREC_TF32X3) {
            RFP_TRY(split_tf32(st, X, static_cast<float *>(w.P), m, nb, kMixedPanel, info));
        } else {
            __nv_bfloat16 *QA = static_cast<__nv_bfloat16 *>(w.P), *QB = QA + (size_t)m * 6 * kMixedPanel;
            RFP_TRY(split_bf16x3(st, X, QA, QB, m, nb, kMixedPanel, info));
        }
        if (prec == RFP_PREC_BF16X6) {
            const __nv_bfloat16 *QA = static_cast<const __nv_bfloat16 *>(w.P),
                                *QB = QA + (size_t)m * 6 * kMixedPanel;
            RFP_TRY(tc_gemm_nt(st, RFP_PREC_BF16, QA, m, 6 * kMixedPanel, 0, QB, m, 6 * kMixedPanel, 0,
                               W.sub(j1, j1), m, m, 6 * kMixedPanel, -1.0f, 1.0f, MASK_LOWER,
                               w.tc_err));
        } else if (prec == RFP_PREC_TF32X3) {
            // A = segments 1..3 = [hi | lo | hi], B = segments 0..2 = [hi | hi | lo]
            const float *Q = static_cast<const float *>(w.P);
            RFP_TRY(tc_gemm_nt(st, RFP_PREC_TF32, Q + kMixedPanel, m, 4 * kMixedPanel, 0, Q, m,
                               4 * kMixedPanel, 0, W.sub(j1, j1), m, m, 3 * kMixedPanel, -1.0f, 1.0f,
                               MASK_LOWER, w.tc_err));
        } else {
            RFP_TRY(tc_gemm_nt(st, prec, w.P, m, kMixedPanel, 0, w.P, m, kMixedPanel, 0,
                               W.sub(j1, j1), m, m, nb, -1.0f, 1.0f, MASK_LOWER, w.tc_err));
        }
    }
    return cudaSuccess;
}

// R = B - A X with A read from its FP64 RFP blocks (A11 = T1, A21 = S,
// A22 = T2 as stored lower triangles; the strict upper halves come from
// the transposed views).
static cudaError_t residual(cudaStream_t st, const RfpViews &v, View<double> B, View<double> X,
                            View<double> R, int64_t nrhs, const int32_t *stop, int splits,
                            double *work)
{
    // the products have nrhs columns and a long K: split K so they fill the GPU
    auto gemm = [&](View<double> C, View<double> A, View<double> Bop, int64_t M, int64_t K,
                    int amask) {
        return gemm_nt_splitk<double>(st, C, A, Bop, M, nrhs, K, -1.0, 1.0, MASK_NONE, amask,
                                      MASK_NONE, stop, splits, work);
    };
    const int64_t n1 = v.n1, n2 = v.n2;
    RFP_TRY((convert<double, double>(st, B, R, n1 + n2, nrhs, false, stop)));
    View<double> R1 = R, R2 = R.sub(n1, 0), X1 = X, X2 = X.sub(n1, 0);
    if (n1 > 0) {
        RFP_TRY(gemm(R1, v.t1, X1.t(), n1, n1, MASK_LOWER));
        RFP_TRY(gemm(R1, v.t1.t(), X1.t(), n1, n1, MASK_STRICT_UPPER));
    }
    if (n1 > 0 && n2 > 0) {
        RFP_TRY(gemm(R1, v.s.t(), X2.t(), n1, n2, MASK_NONE));
        RFP_TRY(gemm(R2, v.s, X1.t(), n2, n1, MASK_NONE));
    }
    if (n2 > 0) {
        RFP_TRY(gemm(R2, v.t2, X2.t(), n2, n2, MASK_LOWER));
        RFP_TRY(gemm(R2, v.t2.t(), X2.t(), n2, n2, MASK_STRICT_UPPER));
    }
    return cudaSuccess;
}

cudaError_t pfsv_mixed_impl(cudaStream_t st, const Layout &L, const double *arf_c, const double *Bp,
                            int64_t ldb, double *Xp, int64_t ldx, int64_t nrhs, int prec,
                            int max_iter, double tol, const MixedWork &w,
                            rfp_mixed_status_t *status)
{
    double *arf = const_cast<double *>(arf_c);     // read only
    RfpViews v{block_view(arf, L, L.t1), block_view(arf, L, L.s), block_view(arf, L, L.t2), L.n1,
               L.n2};
    const int64_t n = L.n;
    View<float> W{w.W, 1, w.ldw};
    View<double> B{const_cast<double *>(Bp), 1, ldb}, X{Xp, 1, ldx}, R{w.R, 1, n};
    View<float> D{w.D, 1, n};

    RFP_TRY(cudaMemsetAsync(status, 0, sizeof(rfp_mixed_status_t), st));
    RFP_TRY(cudaMemsetAsync(w.stop, 0, sizeof(int32_t), st));
    RFP_TRY(cudaMemsetAsync(w.tc_err, 0, sizeof(int32_t), st));
    stage_begin(st);
    RFP_TRY(anorm_inf(st, v, n, w.anorm));
    // 1. W = fl32(A), logical lower triangle
    RFP_TRY((convert<double, float>(st, v.t1, W, L.n1, L.n1, true, nullptr)));
    RFP_TRY((convert<double, float>(st, v.s, W.sub(L.n1, 0), L.n2, L.n1, false, nullptr)));
    RFP_TRY((convert<double, float>(st, v.t2, W.sub(L.n1, L.n1), L.n2, L.n2, true, nullptr)));
    stage_mark(st, "mixed.convert");
    // 2. factor
    int32_t *info = &status->info;
    RFP_TRY(factor_panels(st, W, n, prec, w, info));
    RFP_TRY(stop_on_failure(st, status, w.tc_err, w.stop));
    stage_mark(st, "mixed.factor");
    // 3. refinement (step marks: "mixed.solve", "mixed.residual" per iteration)
    RFP_TRY(fill(st, X, n, nrhs, 0.0));
    RFP_TRY((convert<double, double>(st, B, R, n, nrhs, false, w.stop)));
    stage_mark(st, "mixed.setup");
    for (int it = 0; it < max_iter; ++it) {
        RFP_TRY((convert<double, float>(st, R, D, n, nrhs, false, w.stop)));
        RFP_TRY(trsm_wavefront(st, W, n, w.Inv, w.D, n, nrhs, false, w.sync, w.tc_err, w.stop));
        RFP_TRY(trsm_wavefront(st, W, n, w.Inv, w.D, n, nrhs, true, w.sync, w.tc_err, w.stop));
        RFP_TRY(stop_on_failure(st, status, w.tc_err, w.stop));
        RFP_TRY(add_correction(st, X, D, n, nrhs, w.stop));
        stage_mark(st, "mixed.solve");
        RFP_TRY(residual(st, v, B, X, R, nrhs, w.stop, w.splits, w.splitk));
        RFP_TRY(backward_error(st, R, X, B, n, nrhs, w.anorm, w.berr, tol, status, w.stop));
        stage_mark(st, "mixed.residual");
    }
    return cudaSuccess;
}

}  // namespace rfp
