// Batched PFTRF + PFTRS over many independent SPD matrices of uneven order,
// each in its own RFPF layout: one persistent launch.
//
// Every CTA takes matrices from a device work counter (largest first, as
// ordered by rfp_batch_plan) and runs, on that matrix alone, the blocked
// right-looking Cholesky of Section 3 on the logical lower factor held in the
// RFP blocks T1 / S / T2, followed by the forward and back substitutions of
// Section 4 for its right-hand sides.  Per NB-wide panel (NB = 16 or 32, the
// entry's autotuned choice):
//   1. the panel (rows k0..n-1, NB columns) is read into shared memory,
//   2. it is factored there column by column (pivot, scale, rank-1 update of
//      the remaining panel columns): this is both the diagonal POTRF and the
//      panel TRSM,
//   3. it is written back and the trailing lower triangle receives
//      A(i, j) -= P(i, :) P(j, :)^T in 4 x 4 register tiles.
// Orders up to 512 (the panel then takes 128 KB of shared memory in FP64).
// A failing pivot stores the global 1-based index in info[entry] and skips
// that matrix's solve.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/rfp.h"
#include "rfp_internal.cuh"

namespace rfp {

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchMaxN = 512;

struct PlanEntry {           // device table row (sorted by n descending)
    int64_t n, arf, b;
    int32_t nrhs, ldb, nb, index;
    Block t1, s, t2;
    int64_t n1, ld;
};

struct PlanHeader {
    int32_t counter;         // next table row to take
    int32_t pad[63];         // keeps the table 256-byte aligned
};

template <typename T>
struct Mat {
    View<T> t1, s, t2;
    int64_t n1;
    __device__ __forceinline__ T *at(int64_t i, int64_t j) const   // i >= j
    {
        if (j >= n1) return &t2(i - n1, j - n1);
        if (i >= n1) return &s(i - n1, j);
        return &t1(i, j);
    }
};

template <typename T>
__device__ __forceinline__ View<T> bview(T *base, const Block &b, int64_t ld)
{
    return b.trans ? View<T>{base + b.off, ld, 1} : View<T>{base + b.off, 1, ld};
}

// Factor one matrix in place; returns 0 or the 1-based failing index.
template <typename T, int NB>
__device__ int factor_one(const Mat<T> &A, int64_t n, T *P /* smem (kBatchMaxN) x (NB + 1) */,
                          int *s_fail)
{
    constexpr int LDP = NB + 1;
    const int tid = threadIdx.x;
    for (int64_t k0 = 0; k0 < n; k0 += NB) {
        const int kb = (int)(n - k0 < NB ? n - k0 : NB);
        const int rows = (int)(n - k0);
        // 1. panel -> shared memory (lower part of the diagonal block only)
        for (int e = tid; e < rows * kb; e += blockDim.x) {
            const int r = e % rows, c = e / rows;
            P[r * LDP + c] = (r >= c) ? *A.at(k0 + r, k0 + c) : T(0);
        }
        if (tid == 0) *s_fail = -1;
        __syncthreads();
        // 2. unblocked right-looking Cholesky of the rows x kb panel
        for (int c = 0; c < kb; ++c) {
            if (tid == 0) {
                const T d = P[c * LDP + c];
                if (!(d > T(0))) *s_fail = c;
                else P[c * LDP + c] = sqrt(d);
            }
            __syncthreads();
            if (*s_fail >= 0) return (int)(k0 + *s_fail + 1);
            const T dc = P[c * LDP + c];
            for (int r = c + 1 + tid; r < rows; r += blockDim.x) P[r * LDP + c] /= dc;
            __syncthreads();
            const int rem = kb - c - 1;
            for (int e = tid; e < (rows - c - 1) * rem; e += blockDim.x) {
                const int r = c + 1 + e / rem, q = c + 1 + e % rem;
                if (q <= r) P[r * LDP + q] -= P[r * LDP + c] * P[q * LDP + c];
            }
            __syncthreads();
        }
        // 3a. panel back to the matrix
        for (int e = tid; e < rows * kb; e += blockDim.x) {
            const int r = e % rows, c = e / rows;
            if (r >= c) *A.at(k0 + r, k0 + c) = P[r * LDP + c];
        }
        // 3b. trailing update of the lower triangle rows/cols >= k0 + kb, 4 x 4 tiles
        const int m = rows - kb;
        if (m > 0) {
            const int tm = (m + 3) / 4;
            const int ntiles = tm * (tm + 1) / 2;
            for (int t = tid; t < ntiles; t += blockDim.x) {
                int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
                while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
                while (ti * (ti + 1) / 2 > t) --ti;
                const int tj = t - ti * (ti + 1) / 2;
                T acc[4][4] = {};
                for (int c = 0; c < kb; ++c) {
                    T a[4], b[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int ri = kb + 4 * ti + u, rj = kb + 4 * tj + u;
                        a[u] = ri < rows ? P[ri * LDP + c] : T(0);
                        b[u] = rj < rows ? P[rj * LDP + c] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
                }
                T cin[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int i = 4 * ti + u, j = 4 * tj + v;
                        cin[u][v] = (i < m && j <= i) ? *A.at(k0 + kb + i, k0 + kb + j) : T(0);
                    }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int i = 4 * ti + u, j = 4 * tj + v;
                        if (i < m && j <= i) *A.at(k0 + kb + i, k0 + kb + j) = cin[u][v] - acc[u][v];
                    }
            }
        }
        __syncthreads();
    }
    return 0;
}

// L L^T X = B in place for nrhs <= 8 columns (B column-major, ldb), blocked by NB.
template <typename T, int NB>
__device__ void solve_one(const Mat<T> &A, int64_t n, T *Bm, int64_t ldb, int nrhs,
                          T *D /* smem NB x (NB + 1) */)
{
    constexpr int LDD = NB + 1;
    const int tid = threadIdx.x;
    // forward: L y = b
    for (int64_t k0 = 0; k0 < n; k0 += NB) {
        const int kb = (int)(n - k0 < NB ? n - k0 : NB);
        for (int e = tid; e < kb * kb; e += blockDim.x) {
            const int r = e % kb, c = e / kb;
            D[r * LDD + c] = (r >= c) ? *A.at(k0 + r, k0 + c) : T(0);
        }
        // b(block) -= L(block, 0:k0) y(0:k0): one thread per (row, rhs)
        for (int e = tid; e < kb * nrhs; e += blockDim.x) {
            const int r = e % kb, q = e / kb;
            T s = Bm[k0 + r + q * ldb];
            for (int64_t p = 0; p < k0; ++p) s -= *A.at(k0 + r, p) * Bm[p + q * ldb];
            Bm[k0 + r + q * ldb] = s;
        }
        __syncthreads();
        for (int q = tid; q < nrhs; q += blockDim.x)       // triangle solve, one thread per rhs
            for (int r = 0; r < kb; ++r) {
                T s = Bm[k0 + r + q * ldb];
                for (int p = 0; p < r; ++p) s -= D[r * LDD + p] * Bm[k0 + p + q * ldb];
                Bm[k0 + r + q * ldb] = s / D[r * LDD + r];
            }
        __syncthreads();
    }
    // backward: L^T x = y
    const int64_t nblk = (n + NB - 1) / NB;
    for (int64_t bk = nblk - 1; bk >= 0; --bk) {
        const int64_t k0 = bk * NB;
        const int kb = (int)(n - k0 < NB ? n - k0 : NB);
        for (int e = tid; e < kb * kb; e += blockDim.x) {
            const int r = e % kb, c = e / kb;
            D[r * LDD + c] = (r >= c) ? *A.at(k0 + r, k0 + c) : T(0);
        }
        // b(block) -= L(k0+kb:n, block)^T x(k0+kb:n)
        for (int e = tid; e < kb * nrhs; e += blockDim.x) {
            const int r = e % kb, q = e / kb;
            T s = Bm[k0 + r + q * ldb];
            for (int64_t p = k0 + kb; p < n; ++p) s -= *A.at(p, k0 + r) * Bm[p + q * ldb];
            Bm[k0 + r + q * ldb] = s;
        }
        __syncthreads();
        for (int q = tid; q < nrhs; q += blockDim.x)
            for (int r = kb - 1; r >= 0; --r) {
                T s = Bm[k0 + r + q * ldb];
                for (int p = r + 1; p < kb; ++p) s -= D[p * LDD + r] * Bm[k0 + p + q * ldb];
                Bm[k0 + r + q * ldb] = s / D[r * LDD + r];
            }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kBatchThreads) batched_kernel(PlanHeader *hdr,
                                                                const PlanEntry *table,
                                                                int64_t batch, T *arf, T *B,
                                                                int32_t *info)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *P = reinterpret_cast<T *>(smem_raw);                       // kBatchMaxN x 33
    T *D = P + kBatchMaxN * 33;                                   // 32 x 33
    __shared__ int s_idx, s_fail;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(&hdr->counter, 1);
        __syncthreads();
        const int64_t idx = s_idx;
        __syncthreads();
        if (idx >= batch) return;
        const PlanEntry e = table[idx];
        Mat<T> A{bview(arf + e.arf, e.t1, e.ld), bview(arf + e.arf, e.s, e.ld),
                 bview(arf + e.arf, e.t2, e.ld), e.n1};
        const int fail = e.nb == 16 ? factor_one<T, 16>(A, e.n, P, &s_fail)
                                    : factor_one<T, 32>(A, e.n, P, &s_fail);
        if (threadIdx.x == 0) info[e.index] = fail;
        __syncthreads();
        if (fail == 0 && e.nrhs > 0) {
            if (e.nb == 16) solve_one<T, 16>(A, e.n, B + e.b, e.ldb, e.nrhs, D);
            else solve_one<T, 32>(A, e.n, B + e.b, e.ldb, e.nrhs, D);
        }
        __syncthreads();
    }
}

int g_batch_ctas_cache[64][2] = {};

template <typename T>
int resident_ctas(int smem)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const int e = sizeof(T) == 8 ? 0 : 1;
    if (dev >= 0 && dev < 64 && g_batch_ctas_cache[dev][e]) return g_batch_ctas_cache[dev][e];
    int per_sm = 1;
    cudaFuncSetAttribute(batched_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<T>, kBatchThreads, smem);
    const int ctas = std::max(1, per_sm) * device_sm_count();
    if (dev >= 0 && dev < 64) g_batch_ctas_cache[dev][e] = ctas;
    return ctas;
}

}  // namespace

size_t batch_plan_bytes(int64_t batch)
{
    return sizeof(PlanHeader) + (size_t)std::max<int64_t>(batch, 0) * sizeof(PlanEntry);
}

// Validate, order largest first, and upload.  Returns 0, -2 (entry invalid:
// *bad = its index) or a CUDA error code + 1000.
int batch_plan(int64_t batch, const rfp_batch_entry_t *h, int64_t arf_len, int64_t b_len,
               void *d_plan, cudaStream_t st, int64_t *bad)
{
    std::vector<PlanEntry> rows((size_t)batch);
    for (int64_t k = 0; k < batch; ++k) {
        const rfp_batch_entry_t &e = h[k];
        const bool tr_ok = e.transr == 'N' || e.transr == 'n' || e.transr == 'T' || e.transr == 't';
        const bool up_ok = e.uplo == 'L' || e.uplo == 'l' || e.uplo == 'U' || e.uplo == 'u';
        const int64_t nt = e.n * (e.n + 1) / 2;
        bool ok = tr_ok && up_ok && e.n >= 0 && e.n <= kBatchMaxN && e.arf >= 0 &&
                  e.arf + nt <= arf_len && (e.nb == 0 || e.nb == 16 || e.nb == 32) && e.nrhs >= 0 &&
                  e.nrhs <= 8;
        if (ok && e.nrhs > 0)   // an order-0 matrix reads no right-hand side
            ok = e.ldb >= std::max<int64_t>(1, e.n) &&
                 (e.n == 0 || (e.b >= 0 && e.b + (int64_t)(e.nrhs - 1) * e.ldb + e.n <= b_len));
        if (!ok) {
            *bad = k;
            return -2;
        }
        Layout L;
        make_layout(e.transr, e.uplo, e.n, &L);
        PlanEntry &r = rows[(size_t)k];
        r.n = e.n; r.arf = e.arf; r.b = e.b; r.nrhs = e.nrhs; r.ldb = e.ldb;
        r.nb = e.nb == 0 ? 32 : e.nb; r.index = (int32_t)k;
        r.t1 = L.t1; r.s = L.s; r.t2 = L.t2; r.n1 = L.n1; r.ld = L.ld;
    }
    std::stable_sort(rows.begin(), rows.end(),
                     [](const PlanEntry &a, const PlanEntry &b) { return a.n > b.n; });
    PlanHeader hdr;
    std::memset(&hdr, 0, sizeof hdr);
    cudaError_t err = cudaMemcpyAsync(d_plan, &hdr, sizeof hdr, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess && batch > 0)
        err = cudaMemcpyAsync(static_cast<char *>(d_plan) + sizeof hdr, rows.data(),
                              rows.size() * sizeof(PlanEntry), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);   // host staging is released below
    return err == cudaSuccess ? 0 : 1000 + (int)err;
}

template <typename T>
cudaError_t batched_run(int64_t batch, const void *d_plan, T *arf, T *B, int32_t *info,
                        cudaStream_t st)
{
    if (batch <= 0) return cudaSuccess;
    PlanHeader *hdr = static_cast<PlanHeader *>(const_cast<void *>(d_plan));
    const PlanEntry *table = reinterpret_cast<const PlanEntry *>(static_cast<const char *>(d_plan) +
                                                                 sizeof(PlanHeader));
    const int smem = (kBatchMaxN * 33 + 32 * 33) * (int)sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(batched_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&hdr->counter, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(batch, resident_ctas<T>(smem));
    batched_kernel<T><<<(unsigned)grid, kBatchThreads, smem, st>>>(hdr, table, batch, arf, B, info);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t batched_run<double>(int64_t, const void *, double *, double *, int32_t *,
                                         cudaStream_t);
template cudaError_t batched_run<float>(int64_t, const void *, float *, float *, int32_t *,
                                        cudaStream_t);

}  // namespace rfp
