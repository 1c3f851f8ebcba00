/*
 * rfp.h - C ABI of the GB300 (sm_103a) library for Cholesky factorization,
 * solution and inversion of a symmetric positive definite matrix held in
 * Rectangular Full Packed Format (RFPF).
 *
 * Method: Gustavson, Wasniewski, Dongarra, Langou, "Rectangular Full Packed
 * Format for Cholesky's Algorithm: Factorization, Solution and Inversion".
 * Names and argument order follow the LAPACK 3.2 calling sequences listed in
 * the paper's Table "lapack" (PFTRF, PFTRS, PFTRI, TRTTF, TFTTR), with a
 * stream argument added and INFO moved to device memory.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - transr: 'N' (array A_R, LDAR x ceil(N/2), column-major) or 'T' (its
 *    transpose, ceil(N/2) x LDAR); LDAR = N for odd N and N+1 for even N
 *    (Section 7).  'C' is rejected: the library is real only.
 *  - uplo: 'L' or 'U', which triangle of the symmetric matrix is stored
 *    (Section 2, Eq. 1).  Lower/upper case letters are both accepted.
 *  - The RFP array holds exactly n(n+1)/2 elements, no padding.
 *  - Every pointer except `info` arguments is a DEVICE pointer owned by the
 *    caller, aligned to its element size; `info` is a device int32.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All work is enqueued on it; no entry point synchronizes the device.
 *  - Return value: an immediate host-side result.
 *      0   success (work enqueued),
 *     -i   argument i is invalid (LAPACK convention, 1-based), nothing enqueued,
 *     >0   library error (RFP_ERR_*): a CUDA call failed; the stream's state
 *          is then whatever CUDA reports.
 *    Numerical failure is reported asynchronously through *info (see
 *    rfp_dpftrf / rfp_dpftri).
 *  - n = 0 (and nrhs = 0 for the solve) return 0 immediately.
 *  - The numerical routines allocate no device memory of their own beyond
 *    what each entry point's comment states (workspaces are caller-owned and
 *    sized by a query).  The serving loop is the exception: rfp_serve_create
 *    allocates its arena and pinned result slots once, and rfp_serve_destroy
 *    frees them.
 *  - The s-variants (float) have the same shapes and semantics in IEEE
 *    binary32 arithmetic.
 */
#ifndef RFP_H
#define RFP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RFP_OK 0
#define RFP_ERR_CUDA 1      /* a CUDA runtime call or kernel launch failed */

/*
 * Block descriptor of one RFPF layout (host only; no GPU needed).
 *
 * The logical lower factor is L = [L11 0; L21 L22] (for UPLO='U', L = U^T),
 * split at n1 as drawn in Figs. 4-6: n1 = ceil(N/2) for 'L', floor(N/2) for
 * 'U', n2 = N - n1.  Block X in {T1: L11 (n1 x n1, lower), S: L21 (n2 x n1),
 * T2: L22 (n2 x n2, lower)} has its element (i, j) at array position
 *     X_off + i + j*ld   if X_trans == 0,
 *     X_off + j + i*ld   if X_trans == 1.
 * ld = LDAR for transr='N' and ceil(N/2) for transr='T'.
 * Returns 0, or -1 / -2 / -3 for an invalid transr / uplo / n.
 */
typedef struct rfp_layout {
    int64_t n, n1, n2, ld;
    int64_t t1_off, s_off, t2_off;
    int32_t t1_trans, s_trans, t2_trans;
} rfp_layout_t;

int rfp_layout(char transr, char uplo, int64_t n, rfp_layout_t *out);

/*
 * rfp_dpack (TRTTF, Table "lapack"): copy the UPLO triangle of the
 * column-major n x n matrix A (leading dimension lda >= max(1,n)) into the
 * RFP array arf.  The other triangle of A is never read.  Bit-exact copy.
 * Arguments: 1 transr, 2 uplo, 3 n, 4 A, 5 lda, 6 arf, 7 stream.
 */
int rfp_dpack(char transr, char uplo, int64_t n, const double *A, int64_t lda,
              double *arf, void *stream);
int rfp_spack(char transr, char uplo, int64_t n, const float *A, int64_t lda,
              float *arf, void *stream);

/*
 * rfp_dunpack (TFTTR, Table "lapack"): write the UPLO triangle of A from
 * arf; the other triangle of A is left untouched.  Bit-exact copy.
 * Arguments: 1 transr, 2 uplo, 3 n, 4 arf, 5 A, 6 lda, 7 stream.
 */
int rfp_dunpack(char transr, char uplo, int64_t n, const double *arf, double *A,
                int64_t lda, void *stream);
int rfp_sunpack(char transr, char uplo, int64_t n, const float *arf, float *A,
                int64_t lda, void *stream);

/*
 * rfp_dpftrf (PFTRF, Section 3, Eqs. 2-4, Fig. 4): Cholesky factorization
 * A = L L^T (uplo 'L') or A = U^T U (uplo 'U') in place; arf then holds the
 * factor in the same layout.  Four steps on the blocks: Cholesky of T1,
 * triangular solve of S, symmetric rank-n1 update of T2, Cholesky of T2.
 * *info (device) is set to 0, or to j > 0 when the leading minor of order j
 * is not positive definite (a pivot <= 0 or NaN); arf is then unspecified.
 * FP64 scratch: the triangle factorizations run one launch per panel step
 * (panels 32 columns wide up to triangle order 4096, 64 beyond; trailing
 * update and the next panel's factorization together) and step 2 runs as one
 * launch; they take stream-ordered scratch from a library-private memory pool
 * (8 bytes per panel step, and 8 + 4 ceil(n2 / 16) bytes for step 2), and
 * step 3 below order about 1540 splits its K into chunks held there (up to
 * 8 n2^2 doubles), all returned on `stream` when the call's work is done.
 * While `stream` is being captured into a CUDA graph, the routine runs its
 * multi-launch form instead, which takes none.
 * Arguments: 1 transr, 2 uplo, 3 n, 4 arf, 5 info, 6 stream.
 */
int rfp_dpftrf(char transr, char uplo, int64_t n, double *arf, int32_t *info,
               void *stream);
int rfp_spftrf(char transr, char uplo, int64_t n, float *arf, int32_t *info,
               void *stream);

/*
 * rfp_dpftrs (PFTRS, Section 4, Eqs. 5-8, Fig. 4): solve A X = B with the
 * factor computed by rfp_dpftrf.  B is column-major n x nrhs (ldb >=
 * max(1,n)) and is overwritten by X.  Forward: L11 Y1 = B1, B2 -= L21 Y1,
 * L22 Y2 = B2; backward: L22^T X2 = Y2, Y1 -= L21^T X2, L11^T X1 = Y1, where
 * B1 is rows [0, n1) of B.
 * FP64: each direction is one launch over the whole factor; it takes
 * 8 + 4 ceil(nrhs / 16) bytes of stream-ordered scratch from the same pool
 * as rfp_dpftrf (the multi-launch form under graph capture).  The FP32
 * variant uses the multi-launch form always.
 * Arguments: 1 transr, 2 uplo, 3 n, 4 nrhs, 5 arf, 6 B, 7 ldb, 8 stream.
 */
int rfp_dpftrs(char transr, char uplo, int64_t n, int64_t nrhs, const double *arf,
               double *B, int64_t ldb, void *stream);
int rfp_spftrs(char transr, char uplo, int64_t n, int64_t nrhs, const float *arf,
               float *B, int64_t ldb, void *stream);

/*
 * rfp_dpftri (PFTRI, Section 5, Eqs. 9-11, Fig. 4): overwrite the factor in
 * arf with the UPLO triangle of A^{-1} = W^T W (W = L^{-1}), same layout.
 * *info (device) is set to 0, or to j > 0 when the j-th diagonal entry of the
 * factor is exactly zero; arf is then unspecified.
 * FP64: the three solves with the factor (W21 and S <- L22^-T W21) run as
 * one launch each, with scratch as for rfp_dpftrs.  A triangle T1 or T2 of
 * order m, 64 < m <= 1024, is inverted by one solve L W = I and its W^T W
 * formed by one split-K product, through up to 9 m^2 doubles of scratch from
 * the same pool; larger triangles, and every triangle under graph capture,
 * use the in-place blocked forms.
 * Arguments: 1 transr, 2 uplo, 3 n, 4 arf, 5 info, 6 stream.
 */
int rfp_dpftri(char transr, char uplo, int64_t n, double *arf, int32_t *info,
               void *stream);
int rfp_spftri(char transr, char uplo, int64_t n, float *arf, int32_t *info,
               void *stream);

/*
 * rfp_ssyrk_tc: the SYRK of PFTRF step 3 (Fig. 4, T2 <- T2 - S S^T) on the
 * tcgen05 tensor cores, the building block of the mixed-precision modes.
 * C (n x n, FP32, column-major, ldc >= max(1,n)) <- alpha * A * A^T + beta * C
 * on the lower triangle (uplo must be 'L'; the strict upper triangle of C is
 * not touched).  A is n x k stored K-contiguous (element (i, p) at
 * A[i*lda + p]) in the precision `prec`: RFP_PREC_BF16 (bfloat16, tensor-core
 * kind::f16) or RFP_PREC_TF32 (float read as TF32, kind::tf32); products are
 * accumulated in FP32.  A must be 16-byte aligned and lda * element size a
 * multiple of 16 bytes.  beta == 0 does not read C.  *d_err (device int32)
 * is set non-zero if a bounded wait inside the kernel expired (C is then
 * unspecified); it is not cleared by the call.
 * Arguments: 1 uplo, 2 n, 3 k, 4 alpha, 5 A, 6 lda, 7 prec, 8 beta, 9 C,
 * 10 ldc, 11 d_err, 12 stream.
 */
#define RFP_PREC_BF16 0
#define RFP_PREC_TF32 1
int rfp_ssyrk_tc(char uplo, int64_t n, int64_t k, float alpha, const void *A, int64_t lda,
                 int prec, float beta, float *C, int64_t ldc, int32_t *d_err, void *stream);

/*
 * rfp_dpfsv_mixed: solve A X = B for the SPD matrix A held in FP64 RFPF
 * (arf, any of the eight layouts, left unchanged) by factoring a
 * low-precision copy and refining in FP64.  This is the mixed-precision
 * direction of the project: the algorithms of Sections 3-4 are unchanged
 * apart from the precision of their Level-3 steps; there is no counterpart
 * in the paper (its routines are FP64 or FP32 throughout).
 *   prec RFP_PREC_FP32: FP32 factorization on the FP32 FMA pipes;
 *   prec RFP_PREC_TF32 / RFP_PREC_BF16: FP32 storage, the SYRK updates of
 *        512-wide panels on tcgen05 tensor cores from TF32 / BF16 operands
 *        with FP32 accumulation;
 *   prec RFP_PREC_TF32X3: as RFP_PREC_TF32, but each panel value is split
 *        into two TF32 parts (hi = tf32(x), lo = tf32(x - hi), both rounded
 *        to nearest) and the update sums the three products
 *        hi hi^T + lo hi^T + hi lo^T on the tensor cores: FP32's 24 bits per
 *        operand instead of TF32's 11 (panel buffer four times larger);
 *   prec RFP_PREC_BF16X6: the BF16 tensor cores with FP32-accurate updates:
 *        each panel value is split into three BF16 parts (hi + mid + lo,
 *        Henry, Tang and Heinecke's bfloat16 splitting) and the update sums
 *        the six products hi hi, hi mid, mid hi, mid mid, hi lo, lo hi (panel
 *        buffer twelve times a BF16 panel).
 * Refinement: X = 0, R = B, then up to max_iter times D = (L L^T)^{-1} R in
 * FP32, X += D in FP64, R = B - A X in FP64 from arf; it stops as soon as
 * max_j ||r_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf) <= tol, decided on
 * the device (no host synchronization).  B (n x nrhs, ldb) is read only; X
 * (n x nrhs, ldx) receives the solution.
 * work: caller-owned device workspace of at least rfp_dpfsv_mixed_workspace
 * bytes, 256-byte aligned (FP32 copy of A in full storage, 4 n^2 bytes, plus
 * O(n * (512 + nrhs)) panel and residual buffers).
 * status (device, caller-owned) receives: info (first failing pivot of the
 * low-precision factorization, 0 if none), iterations, converged (1/0),
 * tc_error (non-zero if a tensor-core kernel's bounded wait expired),
 * backward_error (last value of the criterion above).
 * Arguments: 1 transr, 2 uplo, 3 n, 4 nrhs, 5 arf, 6 B, 7 ldb, 8 X, 9 ldx,
 * 10 prec, 11 max_iter, 12 tol, 13 work, 14 work_bytes, 15 status, 16 stream.
 */
#define RFP_PREC_FP32 2
#define RFP_PREC_TF32X3 3
#define RFP_PREC_BF16X6 4
typedef struct rfp_mixed_status {
    int32_t info, iterations, converged, tc_error;
    double backward_error;
} rfp_mixed_status_t;
size_t rfp_dpfsv_mixed_workspace(int64_t n, int64_t nrhs, int prec);
int rfp_dpfsv_mixed(char transr, char uplo, int64_t n, int64_t nrhs, const double *arf,
                    const double *B, int64_t ldb, double *X, int64_t ldx, int prec, int max_iter,
                    double tol, void *work, size_t work_bytes, rfp_mixed_status_t *status,
                    void *stream);

/*
 * rfp_dpfsv_mixed_noalloc: rfp_dpfsv_mixed for callers that cannot allocate
 * device memory (code running inside a memory pool it does not own, plugins
 * whose host application forbids device allocations after start-up, loops
 * that must not block or fail on an allocation).  The paper has no
 * counterpart; this is an interface variant of rfp_dpfsv_mixed.
 * The workspace is a fixed 32 MiB array inside the library; no call
 * allocates anything.  The array is reserved on a device when the library's
 * code for it is loaded there: under CUDA's default lazy module loading that
 * is the first call on that device (CUDA_MODULE_LOADING=EAGER: when the
 * context is created).  Make that first call at start-up, while memory is
 * free; the device then holds the array until the process exits.
 * Same arguments and results as rfp_dpfsv_mixed without work / work_bytes:
 * 1 transr, 2 uplo, 3 n, 4 nrhs, 5 arf, 6 B, 7 ldb, 8 X, 9 ldx, 10 prec,
 * 11 max_iter, 12 tol, 13 status, 14 stream.  Problems whose
 * rfp_dpfsv_mixed_workspace exceeds rfp_dpfsv_mixed_noalloc_capacity() are
 * rejected once every argument has passed rfp_dpfsv_mixed's checks (which
 * come first, with the same codes): -3 if n does not fit even with
 * nrhs = 1, else -4 (for example
 * n = 2048 with nrhs <= 256 fits in the FP32, TF32 and BF16 modes; the
 * split modes, whose panel buffers are larger, fit n = 1664 (split-TF32)
 * and n = 1472 (split-BF16) with nrhs <= 256).
 * All calls share the array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it; serialize them.  The array keeps
 * the previous call's contents; the solve itself clears what must start at
 * zero.  The first call on each device looks up the array's device address
 * (set-up, once per device and context: again after a device reset or in a
 * context the caller created); make it before any stream capture.  A CUDA
 * failure of that set-up returns RFP_ERR_CUDA and is named by
 * rfp_last_cuda_error.
 */
size_t rfp_dpfsv_mixed_noalloc_capacity(void);
int rfp_dpfsv_mixed_noalloc(char transr, char uplo, int64_t n, int64_t nrhs, const double *arf,
                            const double *B, int64_t ldb, double *X, int64_t ldx, int prec,
                            int max_iter, double tol, rfp_mixed_status_t *status, void *stream);

/*
 * Batched PFTRF + PFTRS (the batching direction of the project): many
 * independent SPD matrices, each of its own order n <= 512 and its own RFPF
 * layout, factored (Section 3) and solved (Section 4) by ONE persistent
 * kernel launch.  All RFP arrays live in one caller buffer `arf` and all
 * right-hand sides in one buffer `B`, at element offsets given per matrix.
 *
 * rfp_batch_entry_t, one per matrix:
 *   n       order, 0 <= n <= 512
 *   arf     element offset of its RFP array (n(n+1)/2 elements) in arf
 *   b       element offset of its right-hand sides (column-major, ldb) in B
 *   nrhs    0 (factor only) to 32 (solved 8 columns per pass); ldb >= max(1, n)
 *           when nrhs > 0
 *   transr, uplo   its layout ('N'/'T', 'L'/'U')
 *   nb      panel width 16, 24 or 32 (0 = 32), e.g. from the package's
 *           autotuner; a launch reserves shared memory for the plan's widest
 *           panel (in FP64, plans whose panels are all <= 24 columns wide run
 *           two CTAs per SM)
 *
 * rfp_batch_plan (host, not capturable): validates every entry against the
 * buffer lengths arf_len / b_len (elements), orders the matrices largest
 * first, and copies the resulting table into d_plan (device, caller-owned,
 * rfp_batch_plan_bytes(batch) bytes, 256-byte aligned); it synchronizes
 * `stream`.  Returns 0, -2 if an entry is invalid (its index is written to
 * *bad_entry when bad_entry is not NULL), -5 / -6 for a bad d_plan /
 * plan_bytes, or RFP_ERR_CUDA.  A plan can be reused for any number of runs
 * with the same entries, in FP64 or FP32.  The library remembers, per d_plan
 * address, the widest panel of the plan last written there; a run on a plan
 * copied to another address is sized for 32-column panels (same results).
 * Arguments: 1 batch, 2 h_entries, 3 arf_len, 4 b_len, 5 d_plan, 6 plan_bytes,
 * 7 bad_entry, 8 stream.
 *
 * rfp_dpfsv_batched / rfp_spfsv_batched: one memset of the plan's work
 * counter and one kernel launch on `stream` (so the call can be captured in a
 * CUDA graph and replayed); each matrix is overwritten by its factor, its
 * right-hand sides by the solutions, and d_info[k] (device, one int32 per
 * entry, in entry order) receives 0 or the 1-based index of the first
 * failing pivot (the solve of that matrix is then skipped).  Runs that share
 * a plan must not overlap on the GPU (they share its counter).
 * Arguments: 1 batch, 2 d_plan, 3 arf, 4 B, 5 d_info, 6 stream.
 */
typedef struct rfp_batch_entry {
    int64_t n, arf, b;
    int32_t nrhs, ldb;
    char transr, uplo;
    int16_t nb;
    int32_t reserved;
} rfp_batch_entry_t;
size_t rfp_batch_plan_bytes(int64_t batch);
int rfp_batch_plan(int64_t batch, const rfp_batch_entry_t *h_entries, int64_t arf_len,
                   int64_t b_len, void *d_plan, size_t plan_bytes, int64_t *bad_entry,
                   void *stream);
int rfp_dpfsv_batched(int64_t batch, const void *d_plan, double *arf, double *B, int32_t *d_info,
                      void *stream);
int rfp_spfsv_batched(int64_t batch, const void *d_plan, float *arf, float *B, int32_t *d_info,
                      void *stream);

/* Text for a return code of this library (static storage, never NULL). */
const char *rfp_status_string(int status);

/*
 * The rest of the LAPACK 3.2 RFP routine set (the paper's table of new
 * routines), with LAPACK's argument order and meaning; "d" FP64, "s" FP32.
 * All arrays are device memory, all calls are asynchronous on `stream`, and
 * the return value is 0, -i for an invalid argument i (checked before
 * anything is enqueued), or RFP_ERR_CUDA.
 *
 * rfp_?tpttf / rfp_?tfttp: standard packed storage (AP, n(n+1)/2 elements,
 *   column-major: UPLO 'U' AP[i + j(j+1)/2] = A(i, j), i <= j; 'L'
 *   AP[i + j(2n-j-1)/2] = A(i, j), i >= j) to RFP and back, bit-exact.
 *   Arguments: 1 transr, 2 uplo, 3 n, 4 source, 5 destination, 6 stream.
 * rfp_?tftri: the inverse of the triangular matrix in RFP, in place (the
 *   first stage of PFTRI).  diag 'N' or 'U'; with 'U' the diagonal is taken
 *   as 1 and is left unchanged, and `work` (n elements) holds it meanwhile.
 *   FP64 takes pool scratch as rfp_dpftri does.
 *   *info (device) = 0, or the first exactly zero diagonal (1-based).
 *   Arguments: 1 transr, 2 uplo, 3 diag, 4 n, 5 arf, 6 info, 7 work, 8 stream.
 * rfp_?sfrk: C := alpha op(A) op(A)^T + beta C for the symmetric C in RFP
 *   (its UPLO triangle), op(A) = A (trans 'N', A n x k, lda >= max(1, n)) or
 *   A^T (trans 'T', A k x n, lda >= max(1, k)), A column-major; beta = 0:
 *   C is not read; alpha = 0 or k = 0: A is not read.
 *   Arguments: 1 transr, 2 uplo, 3 trans, 4 n, 5 k, 6 alpha, 7 A, 8 lda,
 *   9 beta, 10 C, 11 stream.
 * rfp_?tfsm: B := alpha op(A)^{-1} B (side 'L', A of order m) or
 *   alpha B op(A)^{-1} (side 'R', A of order n), A triangular in RFP,
 *   op(A) = A (trans 'N') or A^T ('T'), unit diagonal when diag = 'U' (not
 *   read); B m x n column-major, ldb >= max(1, m); alpha = 0: B := 0 and A
 *   is not read.
 *   Arguments: 1 transr, 2 side, 3 uplo, 4 trans, 5 diag, 6 m, 7 n, 8 alpha,
 *   9 arf, 10 B, 11 ldb, 12 stream.
 * rfp_?lansf: *value (device) = the norm of the symmetric matrix in RFP:
 *   norm 'M' max |a_ij|, '1' / 'O' / 'I' one / infinity norm (equal for a
 *   symmetric matrix), 'F' / 'E' Frobenius norm (scaled sums, no overflow for
 *   finite entries); a NaN entry gives NaN.  work: 2n elements.  The result
 *   does not depend on scheduling (fixed-order reductions).
 *   Arguments: 1 norm, 2 transr, 3 uplo, 4 n, 5 arf, 6 work, 7 value, 8 stream.
 */
int rfp_dtpttf(char transr, char uplo, int64_t n, const double *ap, double *arf, void *stream);
int rfp_stpttf(char transr, char uplo, int64_t n, const float *ap, float *arf, void *stream);
int rfp_dtfttp(char transr, char uplo, int64_t n, const double *arf, double *ap, void *stream);
int rfp_stfttp(char transr, char uplo, int64_t n, const float *arf, float *ap, void *stream);
int rfp_dtftri(char transr, char uplo, char diag, int64_t n, double *arf, int32_t *info,
               double *work, void *stream);
int rfp_stftri(char transr, char uplo, char diag, int64_t n, float *arf, int32_t *info,
               float *work, void *stream);
int rfp_dsfrk(char transr, char uplo, char trans, int64_t n, int64_t k, double alpha,
              const double *A, int64_t lda, double beta, double *C, void *stream);
int rfp_ssfrk(char transr, char uplo, char trans, int64_t n, int64_t k, float alpha,
              const float *A, int64_t lda, float beta, float *C, void *stream);
int rfp_dtfsm(char transr, char side, char uplo, char trans, char diag, int64_t m, int64_t n,
              double alpha, const double *arf, double *B, int64_t ldb, void *stream);
int rfp_stfsm(char transr, char side, char uplo, char trans, char diag, int64_t m, int64_t n,
              float alpha, const float *arf, float *B, int64_t ldb, void *stream);
int rfp_dlansf(char norm, char transr, char uplo, int64_t n, const double *arf, double *work,
               double *value, void *stream);
int rfp_slansf(char norm, char transr, char uplo, int64_t n, const float *arf, float *work,
               float *value, void *stream);

/*
 * Serving loop (the serving direction of the project; the paper has no
 * counterpart): a native scheduler that accepts factor+solve, solve and
 * invert requests of uneven order from any host thread and runs them on one
 * GPU with continuous batching.  One scheduler thread admits requests, oldest
 * first, as soon as a stream slot and device memory are free, so requests
 * that arrive while others run overlap with them on the device:
 *   - factor+solve requests with n <= small_n and nrhs <= 32 whose factor is
 *     not resident go into one launch of the batched kernel
 *     (rfp_dpfsv_batched) whenever one of its two streams is idle (every such
 *     request that arrived meanwhile joins that launch, up to batch_max);
 *   - every other request runs on its own stream (one of `streams`): FP64
 *     PFTRF + PFTRS, the mixed-precision solve (rfp_dpfsv_mixed with
 *     RFP_PREC_BF16X6), or PFTRI on a copy of a resident array.
 * A mixed-mode request of order n <= small_n is served in FP64 (its array is
 * held as an FP64 factor): the FP64 result meets the mixed mode's accuracy,
 * and at these orders FP64 is at least as fast.
 * All device memory is one arena of arena_bytes allocated at creation.  The
 * RFP array of a request with key >= 0 stays resident after it completes
 * (FP64 mode: the factor; mixed mode: the FP64 matrix) and is reused by later
 * requests with that key and the same n / layout / mode (a factor+solve on a
 * resident key skips the upload and the factorization).  Resident arrays are
 * admitted by their RFP bytes n(n+1)/2 * 8 and evicted least recently used
 * first when the arena is needed, never while a request uses them.
 * Results are independent of what else runs: every request computes exactly
 * what the corresponding single call computes.
 *
 * rfp_serve_create: cfg->arena_bytes >= 1 MiB; 1 <= streams <= 64;
 * 1 <= batch_max <= 4096; 0 <= small_n <= 512 (0: no batching); max_iter >= 0
 * and tol > 0 for mixed requests; batch_nb[t][b]: panel width (0 = 16, or
 * 16, 24, 32) for TRANSR t (0 'N', 1 'T') and order bucket b (n in
 * (64 b, 64 (b + 1)]).  Returns 0 (*server set), -1 bad config, -2 null
 * server, RFP_ERR_CUDA (arena, pinned memory or streams could not be made).
 * rfp_serve_submit: queues a copy of *req and returns at once (0, -1 null
 * server, -2 invalid request: layout, op, mode, n < 1, nrhs < 1 for
 * solves, null arrays, or key < 0 for SOLVE / INVERT).  The host arrays must
 * stay valid until the request's completion has been polled; pinned memory
 * makes the copies asynchronous.  arf: the RFP array of A (FACTOR_SOLVE),
 * B: n x nrhs column-major (ld n), X: receives the n x nrhs solution, or for
 * INVERT the n(n+1)/2 RFP array of A^{-1} in the request's layout.
 * rfp_serve_poll: up to max completions, waiting up to timeout_s for the
 * first; returns how many were written.  A completion's status is 0, > 0 the
 * failing pivot index (not SPD), or RFP_SERVE_E*: ETOOLARGE (cannot fit the
 * arena even when empty), ENOKEY (no matching resident array), ENOCONV
 * (mixed refinement did not converge), ECUDA.  Times are seconds on the host
 * clock since creation: submitted, started (enqueued on the GPU), done
 * (observed complete by a host callback after the result copies).
 * gpu_start_ms / gpu_end_ms: device clock (CUDA events, ms since creation)
 * at the start of the request's first GPU operation and the end of its last
 * (for a batched request, its batch's); both 0 if it never reached the GPU.
 * Two requests whose [gpu_start_ms, gpu_end_ms] intervals intersect were in
 * progress on the device at the same time.
 * rfp_serve_destroy: finishes every submitted request, then frees everything.
 */
#define RFP_SERVE_OP_FACTOR_SOLVE 0
#define RFP_SERVE_OP_SOLVE 1
#define RFP_SERVE_OP_INVERT 2
#define RFP_SERVE_MODE_FP64 0
#define RFP_SERVE_MODE_MIXED 1
#define RFP_SERVE_ETOOLARGE (-101)
#define RFP_SERVE_ENOKEY (-102)
#define RFP_SERVE_ENOCONV (-103)
#define RFP_SERVE_ECUDA (-104)
typedef struct rfp_serve_config {
    size_t arena_bytes;
    int32_t streams, batch_max, small_n, max_iter;
    double tol;
    int16_t batch_nb[2][8];
} rfp_serve_config_t;
typedef struct rfp_serve_request {
    int64_t id, key, n;
    int32_t nrhs, op, mode;
    char transr, uplo;
    int16_t reserved;
    const double *arf;
    const double *B;
    double *X;
} rfp_serve_request_t;
typedef struct rfp_serve_completion {
    int64_t id;
    int32_t status, iterations, cache_hit, batched;
    double t_submit, t_start, t_done, backward_error;
    double gpu_start_ms, gpu_end_ms;
} rfp_serve_completion_t;
typedef struct rfp_serve_stats {
    int64_t submitted, completed, batches, batched_requests, cache_hits, evictions, cache_entries;
    size_t cache_bytes, arena_in_use, arena_capacity;
} rfp_serve_stats_t;
int rfp_serve_create(const rfp_serve_config_t *cfg, void **server);
int rfp_serve_submit(void *server, const rfp_serve_request_t *req);
int rfp_serve_poll(void *server, rfp_serve_completion_t *out, int max, double timeout_s);
int rfp_serve_stats(void *server, rfp_serve_stats_t *stats);
int rfp_serve_destroy(void *server);

/* Name of the last CUDA error seen by the calling host thread inside this
 * library ("no error" if none). */
const char *rfp_last_cuda_error(void);

/*
 * Instrumentation (no effect on results).
 *
 * rfp_kernel_launches: number of kernels this library has enqueued in this
 * process so far (all threads).
 *
 * rfp_stage_timing(1) makes the calling host thread record a CUDA event at
 * the start of each later rfp_?pftrf / pftrs / pftri call and one after each
 * of its steps (PFTRF: "pftrf.potrf_t1", "pftrf.trsm_s", "pftrf.syrk_t2",
 * "pftrf.potrf_t2", the four steps of Fig. 4); rfp_stage_timing(0) stops
 * recording.  Either call clears the history.  rfp_stage_times waits for
 * the last recorded event, then writes up to `max` step durations in ms (and
 * the steps' names, static strings) of every call recorded since the last
 * rfp_stage_timing, in order; it returns the number written, 0 if none, or
 * -RFP_ERR_CUDA.  At most 8192 events are kept.  Events are created on the
 * device current when they are first needed.
 */
int64_t rfp_kernel_launches(void);
int rfp_stage_timing(int enable);
int rfp_stage_times(int max, float *ms, const char **names);

#ifdef __cplusplus
}
#endif

#endif /* RFP_H */
