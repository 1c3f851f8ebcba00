// Kernels of the rest of the LAPACK 3.2 RFP routine set (the paper's table
// of new routines): TPTTF / TFTTP (standard packed <-> RFP), LANSF (norms of
// the symmetric matrix in RFP), and the diagonal save / restore that lets
// TFTRI treat a unit diagonal.  Every kernel addresses the RFP array through
// the three block views of the logical lower factor (T1 = L11, S = L21,
// T2 = L22), as the factorization does.
#include "rfp_internal.cuh"

namespace rfp {

namespace {

template <typename T>
struct LowerRfp {   // element (i, j), i >= j, of the logical lower triangle
    View<T> t1, s, t2;
    int64_t n1;
    __device__ __forceinline__ T *at(int64_t i, int64_t j) const
    {
        if (j >= n1) return &t2(i - n1, j - n1);
        if (i >= n1) return &s(i - n1, j);
        return &t1(i, j);
    }
};

// max that propagates NaN (a NaN anywhere makes the norm NaN)
template <typename T>
__device__ __forceinline__ T nanmax(T a, T b)
{
    return (b > a || b != b) ? b : a;
}

template <typename T>
LowerRfp<T> lower_rfp(const Layout &L, T *arf)
{
    return LowerRfp<T>{block_view(arf, L, L.t1), block_view(arf, L, L.s), block_view(arf, L, L.t2),
                       L.n1};
}

// TP <-> RFP, one thread per element of the lower triangle of the logical L,
// 32 x 32 tiles (tiles above the diagonal exit).  For UPLO = 'L', L(i, j) =
// A(i, j) sits at AP[i + j (2n - j - 1) / 2] (consecutive i contiguous); for
// UPLO = 'U', L(i, j) = A(j, i) sits at AP[j + i (i + 1) / 2] (consecutive j
// contiguous).  The fast thread index follows the packed array's unit stride.
template <typename T>
__global__ void __launch_bounds__(256) tp_copy_kernel(LowerRfp<T> L, T *ap, int64_t n, int lowerTP,
                                                      int to_rfp)
{
    const int64_t ti = blockIdx.y, tj = blockIdx.x;
    if (tj > ti) return;
    const int fast = threadIdx.x & 31, slow0 = threadIdx.x >> 5;
    for (int q = 0; q < 4; ++q) {
        const int slow = slow0 + 8 * q;
        const int64_t i = ti * 32 + (lowerTP ? fast : slow), j = tj * 32 + (lowerTP ? slow : fast);
        if (i >= n || j > i) continue;
        const int64_t p = lowerTP ? i + j * (2 * n - j - 1) / 2 : j + i * (i + 1) / 2;
        if (to_rfp) *L.at(i, j) = ap[p];
        else ap[p] = *L.at(i, j);
    }
}

// Per row i of the full symmetric matrix (A(i, j) = L(max, min)), one warp:
// which = 0: w[i] = max_j |a_ij|
// which = 1: w[i] = sum_j |a_ij|
// which = 2: w[i] = s_i = max_j |a_ij|, w[n + i] = sum_j (a_ij / s_i)^2
// Lanes take j = lane, lane + 32, ...; the lane partials are combined by a
// fixed butterfly, so the result does not depend on scheduling.
template <typename T>
__global__ void __launch_bounds__(256) row_norm_kernel(LowerRfp<T> L, int64_t n, int which, T *w)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= n) return;
    auto a = [&](int64_t j) { return j <= i ? *L.at(i, j) : *L.at(j, i); };
    T v = T(0);
    for (int64_t j = lane; j < n; j += 32) {
        const T x = fabs(a(j));
        v = which == 1 ? v + x : nanmax(v, x);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = which == 1 ? v + u : nanmax(v, u);
    }
    if (which != 2) {
        if (lane == 0) w[i] = v;
        return;
    }
    const T scale = v;
    T q = T(0);
    if (scale > T(0))
        for (int64_t j = lane; j < n; j += 32) {
            const T x = a(j) / scale;
            q += x * x;
        }
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) {
        w[i] = scale;
        w[n + i] = q;
    }
}

// One CTA: the norm from the row results, combined in a fixed order
// (per-thread strided partials, then a shared-memory tree).
template <typename T>
__global__ void __launch_bounds__(1024) norm_final_kernel(const T *w, int64_t n, int which, T *out)
{
    __shared__ T red[1024];
    const int tid = threadIdx.x;
    T v = T(0);   // largest row value: the norm for which = 0, 1; the largest row scale for 2
    for (int64_t i = tid; i < n; i += blockDim.x) v = nanmax(v, w[i]);
    red[tid] = v;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (tid < h) red[tid] = nanmax(red[tid], red[tid + h]);
        __syncthreads();
    }
    const T mx = red[0];
    __syncthreads();
    if (which != 2) {
        if (tid == 0) *out = mx;
        return;
    }
    // Frobenius: sqrt(sum_i s_i^2 q_i) = mx sqrt(sum_i (s_i / mx)^2 q_i)
    T q = T(0);
    if (mx > T(0))
        for (int64_t i = tid; i < n; i += blockDim.x) {
            const T r = w[i] / mx;
            q += r * r * w[n + i];
        }
    red[tid] = q;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    if (tid == 0) *out = mx * sqrt(red[0]);
}

// Flat pass over the RFP array for the max and Frobenius norms: every
// element of the logical triangle once, coalesced (thread t of CTA b takes
// elements b * 256 + t + k * G * 256).  CTA b < G writes w[b] = max |a| over
// its elements and, for Frobenius, w[G + b] = sum (a / w[b])^2; CTA G (only
// for Frobenius) does the same over the n diagonal elements (read through
// the views) into w[2G], w[2G + 1].  Fixed-order block reductions.
constexpr int kFlatThreads = 256, kFlatPerThread = 8;

template <typename T>
__global__ void __launch_bounds__(kFlatThreads) flat_norm_kernel(const T *arf, int64_t nt,
                                                                 LowerRfp<T> L, int64_t n, int ssq,
                                                                 T *w, int64_t G)
{
    __shared__ T red[kFlatThreads];
    const int tid = threadIdx.x;
    const bool diag = (int64_t)blockIdx.x == G;
    const int64_t total = diag ? n : nt;
    const int64_t start = diag ? tid : (int64_t)blockIdx.x * kFlatThreads + tid;
    const int64_t stride = diag ? kFlatThreads : G * kFlatThreads;
    auto get = [&](int64_t e) -> T { return diag ? *L.at(e, e) : arf[e]; };
    T v = T(0);
#pragma unroll 4
    for (int64_t e = start; e < total; e += stride) v = nanmax(v, (T)fabs(get(e)));
    red[tid] = v;
    __syncthreads();
    for (int h = kFlatThreads / 2; h > 0; h >>= 1) {
        if (tid < h) red[tid] = nanmax(red[tid], red[tid + h]);
        __syncthreads();
    }
    const T scale = red[0];
    __syncthreads();
    const int64_t slot = diag ? 2 * G : blockIdx.x, qslot = diag ? 2 * G + 1 : G + blockIdx.x;
    if (!ssq) {
        if (tid == 0) w[slot] = scale;
        return;
    }
    T q = T(0);
    if (scale > T(0)) {
#pragma unroll 4
        for (int64_t e = start; e < total; e += stride) {
            const T x = get(e) / scale;
            q += x * x;
        }
    }
    red[tid] = q;
    __syncthreads();
    for (int h = kFlatThreads / 2; h > 0; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    if (tid == 0) {
        w[slot] = scale;
        w[qslot] = red[0];
    }
}

// Combine the flat partials: max, or sqrt(2 S_all - S_diag) from the scaled
// sums (fixed order, one CTA).
template <typename T>
__global__ void __launch_bounds__(1024) flat_final_kernel(const T *w, int64_t G, int ssq, T *out)
{
    __shared__ T red[1024];
    const int tid = threadIdx.x;
    T v = T(0);
    for (int64_t b = tid; b < G; b += blockDim.x) v = nanmax(v, w[b]);
    red[tid] = v;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (tid < h) red[tid] = nanmax(red[tid], red[tid + h]);
        __syncthreads();
    }
    const T mx = red[0];
    __syncthreads();
    if (!ssq) {
        if (tid == 0) *out = mx;
        return;
    }
    T q = T(0);
    if (mx > T(0))
        for (int64_t b = tid; b < G; b += blockDim.x) {
            const T r = w[b] / mx;
            q += r * r * w[G + b];
        }
    red[tid] = q;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    if (tid == 0) {
        T d = T(0);
        if (mx > T(0)) {
            const T r = w[2 * G] / mx;
            d = r * r * w[2 * G + 1];
        }
        const T s = T(2) * red[0] - d;
        *out = mx * sqrt(s > T(0) ? s : T(0));
    }
}

// Unit diagonal for TFTRI: save = true copies the diagonal of L to work[0, n)
// and sets it to 1; save = false puts the saved values back.
template <typename T>
__global__ void unit_diag_kernel(LowerRfp<T> L, int64_t n, T *work, int save)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T *d = L.at(i, i);
    if (save) {
        work[i] = *d;
        *d = T(1);
    } else {
        *d = work[i];
    }
}

}  // namespace

template <typename T>
cudaError_t tp_copy(cudaStream_t st, const Layout &L, T *arf, T *ap, bool lowerTP, bool to_rfp)
{
    if (L.n <= 0) return cudaSuccess;
    const unsigned t = (unsigned)((L.n + 31) / 32);
    tp_copy_kernel<T><<<dim3(t, t), 256, 0, st>>>(lower_rfp(L, arf), ap, L.n, lowerTP ? 1 : 0,
                                                  to_rfp ? 1 : 0);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t sym_norm(cudaStream_t st, const Layout &L, const T *arf, int which, T *work, T *out)
{
    if (L.n <= 0) return cudaMemsetAsync(out, 0, sizeof(T), st);
    T *a = const_cast<T *>(arf);   // read only
    const int64_t nt = L.n * (L.n + 1) / 2;
    if (which != 1 && L.n >= 8) {   // max / Frobenius: flat coalesced pass (work: 2G + 2 <= 2n)
        const int64_t span = (int64_t)kFlatThreads * kFlatPerThread;
        int64_t G = (nt + span - 1) / span;
        const int64_t gmax = L.n - 1;   // 2G + 2 <= 2n
        G = G < gmax ? G : gmax;
        const int ssq = which == 2 ? 1 : 0;
        flat_norm_kernel<T><<<(unsigned)(G + ssq), kFlatThreads, 0, st>>>(a, nt, lower_rfp(L, a),
                                                                          L.n, ssq, work, G);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        flat_final_kernel<T><<<1, 1024, 0, st>>>(work, G, ssq, out);
        note_launch();
        return cudaGetLastError();
    }
    row_norm_kernel<T><<<(unsigned)((L.n + 7) / 8), 256, 0, st>>>(lower_rfp(L, a), L.n, which, work);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    norm_final_kernel<T><<<1, 1024, 0, st>>>(work, L.n, which, out);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t unit_diag(cudaStream_t st, const Layout &L, T *arf, T *work, bool save)
{
    if (L.n <= 0) return cudaSuccess;
    unit_diag_kernel<T><<<(unsigned)((L.n + 255) / 256), 256, 0, st>>>(lower_rfp(L, arf), L.n, work,
                                                                       save ? 1 : 0);
    note_launch();
    return cudaGetLastError();
}

#define RFP_SURFACE_INST(T)                                                                        \
    template cudaError_t tp_copy<T>(cudaStream_t, const Layout &, T *, T *, bool, bool);           \
    template cudaError_t sym_norm<T>(cudaStream_t, const Layout &, const T *, int, T *, T *);      \
    template cudaError_t unit_diag<T>(cudaStream_t, const Layout &, T *, T *, bool);
RFP_SURFACE_INST(float)
RFP_SURFACE_INST(double)
#undef RFP_SURFACE_INST

}  // namespace rfp
