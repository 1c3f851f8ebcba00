// Internal declarations of the RFPF CUDA library (not part of the C ABI).
//
// Everything in this library works on "views": a matrix whose element (i, j)
// lives at p[i*rs + j*cs].  The three RFPF blocks T1, S and T2 are views of
// the caller's array, so a transposed block is just a view with its strides
// swapped, and every algorithm below is written once, on the logical lower
// factor L = [L11 0; L21 L22] (Section 3, Eq. 3), for all eight layouts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rfp {

template <typename T>
struct View {
    T *p;
    int64_t rs, cs;
    __host__ __device__ View sub(int64_t i, int64_t j) const { return {p + i * rs + j * cs, rs, cs}; }
    __host__ __device__ View t() const { return {p, cs, rs}; }   // transpose
    __host__ __device__ T &operator()(int64_t i, int64_t j) const { return p[i * rs + j * cs]; }
};

// One block of the RFP array: element (i, j) at off + i + j*ld (trans = 0) or
// off + j + i*ld (trans = 1).
struct Block {
    int64_t off;
    int trans;
};

// Block split and placement of one of the eight layouts (see make_layout).
struct Layout {
    int64_t n, n1, n2, ld;
    Block t1, s, t2;
};

bool make_layout(char transr, char uplo, int64_t n, Layout *out);

template <typename T>
inline View<T> block_view(T *arf, const Layout &L, const Block &b)
{
    return b.trans ? View<T>{arf + b.off, L.ld, 1} : View<T>{arf + b.off, 1, L.ld};
}

// Operand / output triangle masks used by the tile GEMM.
// STRICT variants exclude the diagonal (operands only).
enum Mask : int { MASK_NONE = 0, MASK_LOWER = 1, MASK_UPPER = 2, MASK_STRICT_LOWER = 3,
                  MASK_STRICT_UPPER = 4 };

// Does a triangle mask keep operand element (r, c)?
__host__ __device__ inline bool mask_keeps(int mask, int64_t r, int64_t c)
{
    switch (mask) {
    case MASK_LOWER: return r >= c;
    case MASK_UPPER: return r <= c;
    case MASK_STRICT_LOWER: return r > c;
    case MASK_STRICT_UPPER: return r < c;
    default: return true;
    }
}

#ifdef __CUDACC__
// 1 / sqrt(d) for a normal, finite d > 0 by Newton-Raphson iteration for the
// reciprocal square root, y <- y (3/2 - (d/2) y^2): d = m 4^k with m in
// [1, 4) (exponent split), a single-precision seed for m (about 23 correct
// bits), two double-precision steps (each doubles the correct bits; the
// last one's rounding leaves an error of a few ulp), and the scale 2^-k.
// Other d (zero, negative, subnormal, infinite, NaN) take 1 / sqrt(d).  On
// GB300's narrow FP64 pipe this is a few dependent multiply-adds where a
// square root followed by a division is two long instruction sequences; the
// Cholesky pivots use it for both l_jj = d y and the column scale y.
__device__ __forceinline__ double rsqrt_newton(double d)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;
    if (!(d > 0.0) || e <= -1023 || e >= 1024) return 1.0 / sqrt(d);
    const int k = e >> 1;                                           // floor(e / 2)
    const double m = __longlong_as_double((long long)((bits & 0x000fffffffffffffull) |
                                                      ((unsigned long long)(e - 2 * k + 1023) << 52)));
    double y = (double)rsqrtf((float)m);
    const double h = 0.5 * m;
#pragma unroll
    for (int it = 0; it < 2; ++it) y = fma(y, fma(-h * y, y, 0.5), y);
    return y * __longlong_as_double((long long)((unsigned long long)(1023 - k) << 52));
}
#endif

// Records e as the calling thread's last CUDA error (rfp_last_cuda_error) and
// returns the library's CUDA-failure status (1); cudaSuccess returns 0.
int finish_cuda(cudaError_t e);

// ---- instrumentation (api.cu): launch counter and optional step timing ----
void note_launch();                                   // one kernel enqueued
void stage_begin(cudaStream_t st);                    // start of a timed routine
void stage_mark(cudaStream_t st, const char *name);   // end of one of its steps

// ---- launchers (all enqueue on `st`, return cudaSuccess or the launch error)

// In-place gemm_nt calls (A or B aliasing C): which elements of C a CTA
// must own whole, so that it reads only what it writes itself.
//   GEMM_INPLACE_COLS  C(:, j) is computed from C(:, j) (M <= 64): a CTA
//                      holds all M rows of its columns;
//   GEMM_INPLACE_ROWS  C(i, :) is computed from C(i, :) (N <= 64): a CTA
//                      holds all N columns of its rows.
enum { GEMM_INPLACE_NONE = 0, GEMM_INPLACE_COLS = 1, GEMM_INPLACE_ROWS = 2 };

// Tile shape of one gemm_nt launch.  Out-of-place: the large tile (64 x 64
// FP64, 128 x 128 FP32) or the small one (32 x 32 FP64, 64 x 64 FP32),
// whichever has the smaller estimated time: waves x (CTAs per SM) x (tile
// area), the CTAs of a wave sharing their SM's pipes and each doing work
// proportional to its tile area.  The small tile must win by 5%.  In-place
// FP64 calls take 64 x 16 column strips (GEMM_INPLACE_COLS) or 16 x 64 row
// strips (GEMM_INPLACE_ROWS): four times the CTAs of the 64 x 64 tile, each
// with a quarter of its serial work, since these products sit on the
// latency-bound chain of the blocked triangle inverse and LAUUM.  In-place
// FP32 calls take the large tile, which covers a 64-wide block either way.
enum { GEMM_TILE_BIG = 0, GEMM_TILE_SMALL = 1, GEMM_TILE_COLSTRIP = 2, GEMM_TILE_ROWSTRIP = 3 };
struct GemmTileChoice {
    int bm, bn;
    int kind;
};
inline GemmTileChoice gemm_tile_choice(int64_t M, int64_t N, int cmode, int inplace,
                                       int elem_size, int num_sms, int occ_big, int occ_small,
                                       int64_t splits = 1)   // CTAs per tile (split K)
{
    const int big = elem_size == 8 ? 64 : 128, sml = elem_size == 8 ? 32 : 64;
    if (inplace != GEMM_INPLACE_NONE) {
        if (elem_size == 8 && inplace == GEMM_INPLACE_COLS && M <= 64) return {64, 16, GEMM_TILE_COLSTRIP};
        if (elem_size == 8 && inplace == GEMM_INPLACE_ROWS && N <= 64) return {16, 64, GEMM_TILE_ROWSTRIP};
        return {big, big, GEMM_TILE_BIG};
    }
    auto ctas = [&](int64_t t) {
        const int64_t gm = (M + t - 1) / t, gn = (N + t - 1) / t;
        if (cmode != MASK_LOWER) return gm * gn;
        int64_t c = 0;   // tiles with some i >= j
        for (int64_t by = 0; by < gm; ++by) {
            const int64_t last_n = (by * t + t - 1) / t;   // column tiles 0..last_n
            c += (last_n + 1 < gn ? last_n + 1 : gn);
        }
        return c;
    };
    auto est = [&](int64_t c, int occ, int t) {
        occ = occ > 0 ? occ : 1;
        c *= splits > 1 ? splits : 1;
        const int64_t slots = (int64_t)num_sms * occ;
        return (double)((c + slots - 1) / slots) * occ * (double)t * t;
    };
    if (est(ctas(sml), occ_small, sml) < 0.95 * est(ctas(big), occ_big, big))
        return {sml, sml, GEMM_TILE_SMALL};
    return {big, big, GEMM_TILE_BIG};
}
int device_sm_count();   // SMs of the current device (cached per device)
// Resident CTAs per SM of the large / small gemm_nt configuration for
// element size elem_size (cached per device).
void gemm_occupancy(int elem_size, int *occ_big, int *occ_small);

// C(M x N) = alpha * A(M x K) * B(N x K)^T + beta * C.  cmode MASK_LOWER
// writes only i >= j.  amask / bmask treat an operand as triangular (entries
// outside the triangle read as zero and are never loaded).  A or B may
// alias C when `inplace` says which of C's dimensions is tied (the C
// elements each CTA reads are then among those it writes).  abort: if
// non-null and *abort != 0 at kernel start, the kernel does nothing.
template <typename T>
cudaError_t gemm_nt(cudaStream_t st, View<T> C, View<T> A, View<T> B, int64_t M, int64_t N,
                    int64_t K, T alpha, T beta, int cmode, int amask, int bmask,
                    const int32_t *abort, int inplace = GEMM_INPLACE_NONE);

// gemm_nt with K split into `splits` chunks (one launch, grid z = chunk), the
// chunk products written to work (splits x M x N, dense) and summed into C in
// a fixed order by a second kernel.  For products with few output tiles and a
// long K.  splits <= 1 or work == nullptr falls back to gemm_nt.  With
// splits >= 2 and a work array, C may alias A or B: the chunk products
// write only `work`, and C is written by the second kernel after them.
template <typename T>
cudaError_t gemm_nt_splitk(cudaStream_t st, View<T> C, View<T> A, View<T> B, int64_t M, int64_t N,
                           int64_t K, T alpha, T beta, int cmode, int amask, int bmask,
                           const int32_t *abort, int splits, T *work);

// Solve X * op(Ltri) = alpha * X in place for an M x w strip (w <= 64);
// op = transpose when transL != 0.  Rows are independent.  unit: Ltri has a
// unit diagonal, which is not read.
template <typename T>
cudaError_t trsm_strip(cudaStream_t st, View<T> X, View<T> Ltri, int64_t M, int w, int transL,
                       T alpha, const int32_t *abort, bool unit = false);

// In-place Cholesky of one w x w lower tile (w <= 64).  On a pivot <= 0 or
// NaN at local column j, sets *info = base + j + 1 (when *info was 0).
template <typename T>
cudaError_t potrf_tile(cudaStream_t st, View<T> A, int w, int32_t *info, int64_t base);

// In-place inverse of one w x w lower-triangular tile.
template <typename T>
cudaError_t trtri_tile(cudaStream_t st, View<T> A, int w, const int32_t *abort);

// In-place lower triangle of W^T W for one w x w lower-triangular tile W.
template <typename T>
cudaError_t lauum_tile(cudaStream_t st, View<T> A, int w, const int32_t *abort);

// W = I (m x m), and dst's lower triangle = src's (m x m views), in FP64;
// nothing is done if abort is non-null and non-zero at launch.
cudaError_t identity_fill(cudaStream_t st, View<double> W, int64_t m, const int32_t *abort);
cudaError_t lower_copy(cudaStream_t st, View<double> dst, View<double> src, int64_t m,
                       const int32_t *abort);

// *info = first j (1-based) with a zero diagonal in T1 then T2, else 0.
template <typename T>
cudaError_t check_diag(cudaStream_t st, View<T> t1, int64_t n1, View<T> t2, int64_t n2,
                       int32_t *info);

// Tensor-core GEMM update (tc_gemm.cu): C (FP32 view, M x N) = alpha A B^T +
// beta C, A / B K-contiguous low-precision matrices (kind 0: BF16, kind 1:
// FP32 read as TF32) with a_rows / b_rows rows `pitch` elements apart (pitch
// * element size a multiple of 16 bytes, base 16-byte aligned); rows
// a_row0.. / b_row0.. are used.  cmode MASK_LOWER with M == N launches only
// the lower-triangular tiles.  *err receives a non-zero code if a bounded
// wait inside the kernel expires.
cudaError_t tc_gemm_nt(cudaStream_t st, int kind, const void *A, int64_t a_rows,
                       int64_t a_pitch_elems, int a_row0, const void *B, int64_t b_rows,
                       int64_t b_pitch_elems, int b_row0, View<float> C, int64_t M, int64_t N,
                       int64_t K, float alpha, float beta, int cmode, int *err);

// Batched PFTRF + PFTRS (batched.cu).
size_t batch_plan_bytes(int64_t batch);
int batch_plan(int64_t batch, const struct rfp_batch_entry *h, int64_t arf_len, int64_t b_len,
               void *d_plan, cudaStream_t st, int64_t *bad);
template <typename T>
cudaError_t batched_run(int64_t batch, const void *d_plan, T *arf, T *B, int32_t *info,
                        cudaStream_t st);

// TRTTF / TFTTR copies.
template <typename T>
cudaError_t pack_copy(cudaStream_t st, const Layout &L, bool lowerA, T *A, int64_t lda, T *arf,
                      bool unpack);

// Blocked triangle building blocks (chol.cu), instantiated for float and
// double.  V is an m x m lower triangle; `abort` / `info` as for the kernels.
template <typename T>
cudaError_t potrf_blocked(cudaStream_t st, View<T> V, int64_t m, int32_t *info, int64_t base);
// The blocked solves take unit = true for a unit-diagonal triangle (its
// diagonal is not read).
template <typename T>   // X (rows x m) <- X L^{-T}
cudaError_t trsm_right_lower_trans(cudaStream_t st, View<T> X, int64_t rows, View<T> V, int64_t m,
                                   const int32_t *abort, bool unit = false);
template <typename T>   // X (rows x m) <- alpha X L^{-1}
cudaError_t trsm_right_lower_notrans(cudaStream_t st, View<T> X, int64_t rows, View<T> V,
                                     int64_t m, T alpha, const int32_t *abort, bool unit = false);
template <typename T>   // L X = B, B m x nrhs
cudaError_t trsm_left_lower_notrans(cudaStream_t st, View<T> B, int64_t nrhs, View<T> V, int64_t m,
                                    const int32_t *abort, bool unit = false);
template <typename T>   // L^T X = B
cudaError_t trsm_left_lower_trans(cudaStream_t st, View<T> B, int64_t nrhs, View<T> V, int64_t m,
                                  const int32_t *abort, bool unit = false);

// Inverses of the diagonal blocks of width kInvBlock of the m x m FP32 lower
// triangle V: Inv[b] = (block b)^{-1} for b = 0 .. ceil(m / kInvBlock) - 1,
// each kInvBlock x kInvBlock column-major with zeros above the diagonal and
// outside the block's order (one launch, one CTA per block).  kInvBlock is the
// height of the large FP32 GEMM tile, so a product with a block inverse runs
// in place in one row of CTAs.
constexpr int64_t kInvBlock = 128;
cudaError_t inv_diag_blocks(cudaStream_t st, View<float> V, int64_t m, float *Inv,
                            const int32_t *abort);

// One-launch FP32 block triangular solve (trsm_wavefront.cu): L X = B
// (trans = false) or L^T X = B (trans = true) in place on X (n x nrhs,
// column-major, ldx), L the n x n lower triangle of the column-major view Lv
// (unit row stride, column stride a multiple of 4, 16-byte aligned) and Inv
// its inverted diagonal blocks from inv_diag_blocks.  sync: device scratch of
// wavefront_sync_words(n, nrhs) int32 (cleared by the call, stream-ordered);
// err: error word, set to 4 if a wait between tasks expired; stop: if set at
// launch, nothing is done.
size_t wavefront_sync_words(int64_t n, int64_t nrhs);
cudaError_t trsm_wavefront(cudaStream_t st, View<float> Lv, int64_t n, const float *Inv, float *X,
                           int64_t ldx, int64_t nrhs, bool trans, int32_t *sync, int32_t *err,
                           const int32_t *stop);

// One-launch FP64 block substitution with a logical lower factor
// (rfp_solve.cu): L Y = X (trans = false) or L^T Y = X (trans = true) in
// place on X (n x nrhs, any strides), n = n1 + n2, L = [T1 0; S T2] given by
// its RFP block views (n2 = 0: L is T1 alone).  sync: device scratch of
// rfp_solve_sync_words(nrhs) int32 (cleared by the call, stream-ordered).
// abort: if non-null and non-zero when the launch starts, nothing is done.
// alpha scales the right-hand side (op(L) Y = alpha X).  If a wait between
// tasks expires (2 s), the blocks of X not computed are set to NaN.
// lower_rhs (forward, n2 = 0 only): X is lower triangular (column c zero in
// rows < c), so the solution is too; blocks above a column group's first
// row are neither read nor written, which cuts the work of L W = I from
// n^3 / 2 to about n^3 / 6 multiply-adds.
size_t rfp_solve_sync_words(int64_t nrhs);
cudaError_t rfp_solve(cudaStream_t st, View<double> t1, View<double> s, View<double> t2, int64_t n1,
                      int64_t n2, View<double> X, int64_t nrhs, bool trans, int32_t *sync,
                      const int32_t *abort = nullptr, double alpha = 1.0, bool lower_rhs = false);
// One panel step of the FP64 lookahead Cholesky of an m x m lower triangle V
// (potrf_step.cu), panel k = [k0, k0 + pw) already factored, pw =
// potrf_step_width(m) (32 or 64): the trailing update with it, and the
// factorization of panel k + 1 (its diagonal tile and the rows below), in
// one launch.  sync: 2 int32 per step, zero before the launch
// (potrf_step_sync_words(m) for all steps of one factorization).  info as
// for potrf_tile (global index base + column + 1; the launch does nothing if
// *info is already non-zero).
int potrf_step_width(int64_t m);
// Tile width (32 or 64) of a lookahead step's bulk update of the trailing
// triangle of order `rest` (rows below the next panel), with `slots`
// resident step CTAs on the device: the 32-wide tile when it wins by 5% on
// waves x tile area (a bulk tile's time grows with its area), i.e. when the
// 64-wide tiles are too few to fill the device.
inline int potrf_step_bulk_tile(int64_t rest, int64_t slots)
{
    if (rest <= 0) return 64;
    slots = slots > 0 ? slots : 1;
    auto est = [&](int64_t t) {
        const int64_t r = (rest + t - 1) / t, tiles = r * (r + 1) / 2;
        return (double)((tiles + slots - 1) / slots) * (double)(t * t);
    };
    return est(32) < 0.95 * est(64) ? 32 : 64;
}
size_t potrf_step_sync_words(int64_t m);
cudaError_t potrf_step(cudaStream_t st, View<double> V, int64_t m, int64_t k0, int32_t *info,
                       int64_t base, int32_t *sync);
// Stream-ordered scratch (`words` int32, 256-byte aligned) for the sync
// words and work arrays of the FP64 one-launch forms, from a library-private
// memory pool.  cudaErrorNotSupported while `st` is being captured into a
// graph.
cudaError_t solve_scratch_acquire(cudaStream_t st, size_t words, int32_t **out);
cudaError_t solve_scratch_release(cudaStream_t st, int32_t *p);

// The rest of the LAPACK 3.2 RFP routine set (surface.cu kernels, chol.cu
// orchestration), all on the logical lower triangle's three block views.
// TP <-> RFP copy (lowerTP: the packed array holds the lower triangle).
template <typename T>
cudaError_t tp_copy(cudaStream_t st, const Layout &L, T *arf, T *ap, bool lowerTP, bool to_rfp);
// Norm of the symmetric matrix: which 0 max |a|, 1 one / infinity norm,
// 2 Frobenius; work holds 2n elements; *out (device) receives the norm.
template <typename T>
cudaError_t sym_norm(cudaStream_t st, const Layout &L, const T *arf, int which, T *work, T *out);
// Save the diagonal to work and set it to 1 (save), or put it back.
template <typename T>
cudaError_t unit_diag(cudaStream_t st, const Layout &L, T *arf, T *work, bool save);
// TFTRI: W = L^{-1} in place (blocks W11, W21, W22); *info = first zero diagonal.
template <typename T>
cudaError_t tftri_impl(cudaStream_t st, const Layout &L, T *arf, int32_t *info);
// SFRK: C = alpha op(A) op(A)^T + beta C on C's RFP blocks; op(A) is the
// n x k view opA.
template <typename T>
cudaError_t sfrk_impl(cudaStream_t st, const Layout &L, T *arf, View<T> opA, int64_t k, T alpha,
                      T beta);
// TFSM: B (m x nc) = alpha op(A)^{-1} B (left) or alpha B op(A)^{-1}, op(A) =
// L (opT false) or L^T (opT true) for the logical lower L of the RFP triangle.
template <typename T>
cudaError_t tfsm_impl(cudaStream_t st, const Layout &L, const T *arf, bool left, bool opT,
                      bool unit, int64_t m, int64_t nc, T alpha, T *B, int64_t ldb);

// Blocked algorithms on the RFP blocks (Sections 3-5).
template <typename T>
cudaError_t pftrf_impl(cudaStream_t st, const Layout &L, T *arf, int32_t *info);
template <typename T>
cudaError_t pftrs_impl(cudaStream_t st, const Layout &L, const T *arf, T *B, int64_t ldb,
                       int64_t nrhs);
template <typename T>
cudaError_t pftri_impl(cudaStream_t st, const Layout &L, T *arf, int32_t *info);

}  // namespace rfp
