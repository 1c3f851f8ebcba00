// Element-wise and reduction kernels of the mixed-precision solve
// (mixed.cu): precision conversion between strided views, the FP64
// refinement update, the infinity norm of the symmetric matrix held in RFP,
// and the per-column normwise backward error that decides convergence.
// All of them are HBM-bound one-pass kernels; each returns at once when its
// `stop` word is non-zero, so the fixed launch sequence of the refinement
// loop costs nothing after convergence.
#include <cuda_bf16.h>

#include <cfloat>

#include "mixed_internal.cuh"

namespace rfp {

template <typename Td, typename Ts>
__device__ __forceinline__ Td cvt(Ts x);
template <> __device__ __forceinline__ float cvt<float, double>(double x) { return (float)x; }
template <> __device__ __forceinline__ double cvt<double, double>(double x) { return x; }
template <> __device__ __forceinline__ double cvt<double, float>(float x) { return (double)x; }
template <> __device__ __forceinline__ float cvt<float, float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, float>(float x)
{
    return __float2bfloat16_rn(x);
}

constexpr int kCvtTile = 32;

// dst = (Td) src for a rows x cols block (tri: lower triangle only), through a
// 32 x 32 shared-memory tile so both sides walk their unit-stride index.
template <typename Ts, typename Td>
__global__ void __launch_bounds__(256) convert_kernel(View<Ts> src, View<Td> dst, int64_t rows,
                                                      int64_t cols, int tri, const int32_t *stop)
{
    __shared__ Ts tile[kCvtTile][kCvtTile + 1];
    if (stop && *stop) return;
    const int64_t r0 = (int64_t)blockIdx.y * kCvtTile, c0 = (int64_t)blockIdx.x * kCvtTile;
    if (tri && r0 + kCvtTile - 1 < c0) return;
    const int fast = threadIdx.x % kCvtTile, slow0 = threadIdx.x / kCvtTile;   // 8 slow rows
    auto ok = [&](int64_t i, int64_t j) { return i < rows && j < cols && (!tri || i >= j); };
    const bool srow = src.rs == 1, drow = dst.rs == 1;
#pragma unroll
    for (int q = 0; q < kCvtTile / 8; ++q) {
        const int sl = slow0 + 8 * q;
        const int ti = srow ? fast : sl, tj = srow ? sl : fast;
        if (ok(r0 + ti, c0 + tj)) tile[ti][tj] = src(r0 + ti, c0 + tj);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kCvtTile / 8; ++q) {
        const int sl = slow0 + 8 * q;
        const int ti = drow ? fast : sl, tj = drow ? sl : fast;
        if (ok(r0 + ti, c0 + tj)) dst(r0 + ti, c0 + tj) = cvt<Td, Ts>(tile[ti][tj]);
    }
}

template <typename Ts, typename Td>
cudaError_t convert(cudaStream_t st, View<Ts> src, View<Td> dst, int64_t rows, int64_t cols,
                    bool tri, const int32_t *stop)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((cols + kCvtTile - 1) / kCvtTile), (unsigned)((rows + kCvtTile - 1) / kCvtTile));
    convert_kernel<Ts, Td><<<grid, 256, 0, st>>>(src, dst, rows, cols, tri ? 1 : 0, stop);
    note_launch();
    return cudaGetLastError();
}

// Rounding of an FP32 value to TF32 (10 stored mantissa bits), to nearest
// with ties away from zero: add half a TF32 unit to the magnitude, clear the
// 13 low mantissa bits.  Finite inputs only (the panels are bounded).
__device__ __forceinline__ float round_tf32(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// Split of an FP32 panel for three-product TF32 updates: hi = tf32(x),
// lo = tf32(x - hi) (x - hi is exact in FP32 by Sterbenz's lemma), so
// |x - hi - lo| <= 2^-24 |x|: hi + lo carries FP32's precision.  Row r of Q
// holds the four K-segments [hi | hi | lo | hi] of width seg, so that with
// A = Q + seg and B = Q a single K = 3 seg product sums
// hi hi^T + lo hi^T + hi lo^T (the dropped lo lo^T is below 2^-22 |x y|).
__global__ void __launch_bounds__(256) split_tf32_kernel(View<float> src, float *Q, int64_t rows,
                                                         int64_t cols, int64_t seg,
                                                         const int32_t *stop)
{
    __shared__ float tile[kCvtTile][kCvtTile + 1];
    if (stop && *stop) return;
    const int64_t r0 = (int64_t)blockIdx.y * kCvtTile, c0 = (int64_t)blockIdx.x * kCvtTile;
    const int fast = threadIdx.x % kCvtTile, slow0 = threadIdx.x / kCvtTile;
    const bool srow = src.rs == 1;
#pragma unroll
    for (int q = 0; q < kCvtTile / 8; ++q) {
        const int sl = slow0 + 8 * q;
        const int ti = srow ? fast : sl, tj = srow ? sl : fast;
        if (r0 + ti < rows && c0 + tj < cols) tile[ti][tj] = src(r0 + ti, c0 + tj);
    }
    __syncthreads();
    const int64_t pitch = 4 * seg;
#pragma unroll
    for (int q = 0; q < kCvtTile / 8; ++q) {
        const int ti = slow0 + 8 * q, tj = fast;          // k (column) is Q's unit stride
        const int64_t r = r0 + ti, k = c0 + tj;
        if (r < rows && k < cols) {
            const float x = tile[ti][tj];
            const float hi = round_tf32(x);
            const float lo = round_tf32(x - hi);
            float *row = Q + r * pitch + k;
            row[0] = hi;
            row[seg] = hi;
            row[2 * seg] = lo;
            row[3 * seg] = hi;
        }
    }
}

cudaError_t split_tf32(cudaStream_t st, View<float> src, float *Q, int64_t rows, int64_t cols,
                       int64_t seg, const int32_t *stop)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((cols + kCvtTile - 1) / kCvtTile), (unsigned)((rows + kCvtTile - 1) / kCvtTile));
    split_tf32_kernel<<<grid, 256, 0, st>>>(src, Q, rows, cols, seg, stop);
    note_launch();
    return cudaGetLastError();
}

// Split of an FP32 panel into three BF16 parts (Henry, Tang and Heinecke's
// bfloat16 splitting): hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi -
// mid), each difference exact in FP32, so hi + mid + lo carries FP32's 24
// bits.  Row r of QA holds the K-segments [hi | hi | mid | mid | hi | lo] and
// row r of QB [hi | mid | hi | mid | lo | hi] (width seg each), so one
// K = 6 seg product QA QB^T sums the six terms hi hi^T, hi mid^T, mid hi^T,
// mid mid^T, hi lo^T, lo hi^T; the dropped ones are below 2^-24 |x y|.
__global__ void __launch_bounds__(256) split_bf16x3_kernel(View<float> src, __nv_bfloat16 *QA,
                                                           __nv_bfloat16 *QB, int64_t rows,
                                                           int64_t cols, int64_t seg,
                                                           const int32_t *stop)
{
    __shared__ float tile[kCvtTile][kCvtTile + 1];
    if (stop && *stop) return;
    const int64_t r0 = (int64_t)blockIdx.y * kCvtTile, c0 = (int64_t)blockIdx.x * kCvtTile;
    const int fast = threadIdx.x % kCvtTile, slow0 = threadIdx.x / kCvtTile;
    const bool srow = src.rs == 1;
#pragma unroll
    for (int q = 0; q < kCvtTile / 8; ++q) {
        const int sl = slow0 + 8 * q;
        const int ti = srow ? fast : sl, tj = srow ? sl : fast;
        if (r0 + ti < rows && c0 + tj < cols) tile[ti][tj] = src(r0 + ti, c0 + tj);
    }
    __syncthreads();
    const int64_t pitch = 6 * seg;
#pragma unroll
    for (int q = 0; q < kCvtTile / 8; ++q) {
        const int ti = slow0 + 8 * q, tj = fast;
        const int64_t r = r0 + ti, k = c0 + tj;
        if (r < rows && k < cols) {
            const float x = tile[ti][tj];
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            const float r1 = x - __bfloat162float(hi);
            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
            const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
            __nv_bfloat16 *a = QA + r * pitch + k, *b = QB + r * pitch + k;
            a[0] = hi;        b[0] = hi;
            a[seg] = hi;      b[seg] = mid;
            a[2 * seg] = mid; b[2 * seg] = hi;
            a[3 * seg] = mid; b[3 * seg] = mid;
            a[4 * seg] = hi;  b[4 * seg] = lo;
            a[5 * seg] = lo;  b[5 * seg] = hi;
        }
    }
}

cudaError_t split_bf16x3(cudaStream_t st, View<float> src, __nv_bfloat16 *QA, __nv_bfloat16 *QB,
                         int64_t rows, int64_t cols, int64_t seg, const int32_t *stop)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((unsigned)((cols + kCvtTile - 1) / kCvtTile), (unsigned)((rows + kCvtTile - 1) / kCvtTile));
    split_bf16x3_kernel<<<grid, 256, 0, st>>>(src, QA, QB, rows, cols, seg, stop);
    note_launch();
    return cudaGetLastError();
}

// X += (double) D, n x nrhs.
__global__ void axpy_kernel(View<double> X, View<float> D, int64_t n, int64_t nrhs,
                            const int32_t *stop)
{
    if (*stop) return;
    const int64_t total = n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        X(i, j) += (double)D(i, j);
    }
}

cudaError_t add_correction(cudaStream_t st, View<double> X, View<float> D, int64_t n, int64_t nrhs,
                           const int32_t *stop)
{
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n * nrhs + 255) / 256, 4096);
    axpy_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, D, n, nrhs, stop);
    note_launch();
    return cudaGetLastError();
}

__global__ void fill_kernel(View<double> X, int64_t n, int64_t nrhs, double v)
{
    const int64_t total = n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x)
        X(e % n, e / n) = v;
}

cudaError_t fill(cudaStream_t st, View<double> X, int64_t n, int64_t nrhs, double v)
{
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n * nrhs + 255) / 256, 4096);
    fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, n, nrhs, v);
    note_launch();
    return cudaGetLastError();
}

// Element (i, j), i >= j, of the logical lower triangle of A held in RFP.
__device__ __forceinline__ double rfp_lower(const RfpViews &v, int64_t i, int64_t j)
{
    if (j >= v.n1) return v.t2(i - v.n1, j - v.n1);
    if (i >= v.n1) return v.s(i - v.n1, j);
    return v.t1(i, j);
}

// ||A||_inf = max_i sum_j |A(i, j)| of the symmetric matrix: row i of the
// stored lower triangle plus column i below the diagonal.  One warp per row;
// the maximum is combined through the ordered bit pattern of a non-negative
// double, so the result does not depend on the order of the warps.
__global__ void anorm_kernel(RfpViews v, int64_t n, unsigned long long *out)
{
    const int lane = threadIdx.x % 32;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t j = lane; j <= i; j += 32) s += fabs(rfp_lower(v, i, j));
    for (int64_t k = i + 1 + lane; k < n; k += 32) s += fabs(rfp_lower(v, k, i));
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

cudaError_t anorm_inf(cudaStream_t st, const RfpViews &v, int64_t n, double *out)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
    if (e != cudaSuccess || n <= 0) return e;
    const int64_t warps_per_block = 8;
    anorm_kernel<<<(unsigned)((n + warps_per_block - 1) / warps_per_block), 256, 0, st>>>(
        v, n, reinterpret_cast<unsigned long long *>(out));
    note_launch();
    return cudaGetLastError();
}

// max that keeps a NaN (fmax would drop it and could fake convergence)
__device__ __forceinline__ double nanmax(double a, double b)
{
    return (a != a || b != b) ? __longlong_as_double(0x7ff8000000000000ll) : fmax(a, b);
}

// Column j: ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf).
__global__ void __launch_bounds__(256) berr_col_kernel(View<double> R, View<double> X,
                                                       View<double> B, int64_t n,
                                                       const double *anorm, double *berr,
                                                       const int32_t *stop)
{
    __shared__ double red[3][256];
    if (*stop) return;
    const int64_t j = blockIdx.x;
    double r = 0.0, x = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        r = nanmax(r, fabs(R(i, j)));
        x = nanmax(x, fabs(X(i, j)));
        b = nanmax(b, fabs(B(i, j)));
    }
    red[0][threadIdx.x] = r; red[1][threadIdx.x] = x; red[2][threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int q = 0; q < 3; ++q) red[q][threadIdx.x] = nanmax(red[q][threadIdx.x], red[q][threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double den = *anorm * red[1][0] + red[2][0];
        berr[j] = den > 0.0 ? red[0][0] / den : red[0][0];
    }
}

__global__ void berr_final_kernel(const double *berr, int64_t nrhs, double tol,
                                  rfp_mixed_status_t *status, int32_t *stop)
{
    if (*stop) return;
    double m = 0.0;
    for (int64_t j = 0; j < nrhs; ++j) m = nanmax(m, berr[j]);
    status->backward_error = m;
    status->iterations += 1;
    if (m <= tol) {
        status->converged = 1;
        *stop = 1;
    }
}

cudaError_t backward_error(cudaStream_t st, View<double> R, View<double> X, View<double> B,
                           int64_t n, int64_t nrhs, const double *anorm, double *berr_col,
                           double tol, rfp_mixed_status_t *status, int32_t *stop)
{
    berr_col_kernel<<<(unsigned)nrhs, 256, 0, st>>>(R, X, B, n, anorm, berr_col, stop);
    note_launch();
    berr_final_kernel<<<1, 1, 0, st>>>(berr_col, nrhs, tol, status, stop);
    note_launch();
    return cudaGetLastError();
}

// Stop the refinement when the factorization failed; copy the tensor-core
// error word into the status.
__global__ void stop_on_failure_kernel(rfp_mixed_status_t *status, const int32_t *tc_err,
                                       int32_t *stop)
{
    status->tc_error = *tc_err;
    if (status->info != 0 || *tc_err != 0) *stop = 1;
}

cudaError_t stop_on_failure(cudaStream_t st, rfp_mixed_status_t *status, const int32_t *tc_err,
                            int32_t *stop)
{
    stop_on_failure_kernel<<<1, 1, 0, st>>>(status, tc_err, stop);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t convert<double, float>(cudaStream_t, View<double>, View<float>, int64_t,
                                            int64_t, bool, const int32_t *);
template cudaError_t convert<double, double>(cudaStream_t, View<double>, View<double>, int64_t,
                                             int64_t, bool, const int32_t *);
template cudaError_t convert<float, float>(cudaStream_t, View<float>, View<float>, int64_t,
                                           int64_t, bool, const int32_t *);
template cudaError_t convert<float, __nv_bfloat16>(cudaStream_t, View<float>, View<__nv_bfloat16>,
                                                   int64_t, int64_t, bool, const int32_t *);

}  // namespace rfp
