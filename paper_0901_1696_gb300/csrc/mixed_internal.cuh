// Internal declarations of the mixed-precision solve (mixed.cu,
// mixed_kernels.cu).
#pragma once

#include <cuda_bf16.h>

#include <algorithm>

#include "../../include/rfp.h"
#include "rfp_internal.cuh"

namespace rfp {

// The three logical-lower blocks of an FP64 RFP array.
struct RfpViews {
    View<double> t1, s, t2;
    int64_t n1, n2;
};

template <typename Ts, typename Td>
cudaError_t convert(cudaStream_t st, View<Ts> src, View<Td> dst, int64_t rows, int64_t cols,
                    bool tri, const int32_t *stop);
// Q rows of four K-segments [hi | hi | lo | hi] (width seg) of the rows x cols
// FP32 block src, hi = x truncated to TF32, lo = x - hi.
cudaError_t split_tf32(cudaStream_t st, View<float> src, float *Q, int64_t rows, int64_t cols,
                       int64_t seg, const int32_t *stop);
// QA / QB rows of six K-segments (width seg) of the three-way BF16 split of
// the rows x cols FP32 block src: QA [hi|hi|mid|mid|hi|lo], QB [hi|mid|hi|mid|lo|hi].
cudaError_t split_bf16x3(cudaStream_t st, View<float> src, __nv_bfloat16 *QA, __nv_bfloat16 *QB,
                         int64_t rows, int64_t cols, int64_t seg, const int32_t *stop);
cudaError_t add_correction(cudaStream_t st, View<double> X, View<float> D, int64_t n, int64_t nrhs,
                           const int32_t *stop);
cudaError_t fill(cudaStream_t st, View<double> X, int64_t n, int64_t nrhs, double v);
cudaError_t anorm_inf(cudaStream_t st, const RfpViews &v, int64_t n, double *out);
cudaError_t backward_error(cudaStream_t st, View<double> R, View<double> X, View<double> B,
                           int64_t n, int64_t nrhs, const double *anorm, double *berr_col,
                           double tol, rfp_mixed_status_t *status, int32_t *stop);
cudaError_t stop_on_failure(cudaStream_t st, rfp_mixed_status_t *status, const int32_t *tc_err,
                            int32_t *stop);

// Workspace carve-up of the mixed-precision solve (mixed.cu).
struct MixedWork {
    float *W;          // FP32 working matrix / factor, ldw x n column-major (lower used)
    int64_t ldw;
    float *Inv;        // inverses of the factor's diagonal blocks, ceil(n / kInvBlock) x kInvBlock^2
    void *P;           // low-precision panel, n x kPanel, K-contiguous
    double *R;         // FP64 residual, n x nrhs
    float *D;          // FP32 correction, n x nrhs
    double *berr;      // per-column backward errors (nrhs)
    double *anorm;     // ||A||_inf
    int32_t *stop;     // refinement stop word
    int32_t *tc_err;   // tensor-core / solve kernel error word
    int32_t *sync;     // task counter and ready flags of the one-launch solves
    double *splitk;    // split-K slices of the residual products (residual_splits x n x nrhs)
    int splits;
};

// K chunks of the residual products: one per 2048 of the larger block's
// order, at most 8 (1 = no split, no buffer).
inline int residual_splits(int64_t n)
{
    const int64_t k = ((n + 1) / 2) / 2048;
    return (int)(k < 1 ? 1 : (k > 8 ? 8 : k));
}

constexpr int64_t kMixedPanel = 512;   // panel width of the tensor-core factorization

// Columns of the panel buffer P per row: the split-TF32 mode keeps four
// segments, the split-BF16 mode two operands (QA, QB) of six segments each.
inline int64_t panel_cols(int prec)
{
    return prec == RFP_PREC_TF32X3 ? 4 * kMixedPanel
                                   : (prec == RFP_PREC_BF16X6 ? 12 * kMixedPanel : kMixedPanel);
}

size_t mixed_workspace_bytes(int64_t n, int64_t nrhs, int prec);
// Checks of rfp_dpfsv_mixed's arguments other than its workspace (arguments
// 13 and 14): 0 if they pass, else -i in rfp_dpfsv_mixed's numbering (status
// is argument 15).  Pointer and leading-dimension checks only when n > 0 and
// nrhs > 0.
int mixed_check_args(char transr, char uplo, int64_t n, int64_t nrhs, const double *arf,
                     const double *B, int64_t ldb, const double *X, int64_t ldx, int prec,
                     int max_iter, double tol, const rfp_mixed_status_t *status);
bool mixed_carve(void *work, size_t bytes, int64_t n, int64_t nrhs, int prec, MixedWork *w);
cudaError_t pfsv_mixed_impl(cudaStream_t st, const Layout &L, const double *arf, const double *B,
                            int64_t ldb, double *X, int64_t ldx, int64_t nrhs, int prec,
                            int max_iter, double tol, const MixedWork &w,
                            rfp_mixed_status_t *status);

}  // namespace rfp
