// Batched PFTRF + PFTRS over many independent SPD matrices of uneven order,
// each in its own RFPF layout: one persistent launch.
//
// Every CTA takes matrices from a device work counter (largest first, as
// ordered by rfp_batch_plan) and runs, on that matrix alone, the blocked
// right-looking Cholesky of Section 3 on the logical lower factor held in the
// RFP blocks T1 / S / T2, followed by the forward and back substitutions of
// Section 4 for its right-hand sides.  Per NB-wide panel (NB = 16, 24 or 32,
// the entry's autotuned choice):
//   1. the panel (rows k0..n-1, NB columns) is read into shared memory,
//      column-major,
//   2. it is factored there column by column (pivot and its reciprocal by
//      one thread, then per row: scale, rank-1 update of the remaining panel
//      columns): this is both the diagonal POTRF and the panel TRSM,
//   3. it is written back and the trailing lower triangle receives
//      A(i, j) -= P(i, :) P(j, :)^T in 4 x 4 register tiles, whose operands
//      are four consecutive rows of a panel column.
// Orders up to 512 (the panel then takes 129 KB of shared memory in FP64).
// A failing pivot stores the global 1-based index in info[entry] and skips
// that matrix's solve.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "../../include/rfp.h"
#include "rfp_internal.cuh"

namespace rfp {

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchMaxN = 512;
constexpr int kBatchMaxRhs = 32;   // right-hand sides per matrix (solved 8 per pass)

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

// Shared-memory layout of one CTA: the panel P (kMaxNb columns of kPanelLd
// rows, column-major: a column's rows are contiguous), then the solve's
// diagonal block D (32 x 33), its block of solutions Y (32 x 8), the
// reciprocals of D's diagonal and the current pivot's reciprocal.
// A launch is sized for the widest panel among its plan's entries (16, 24
// or 32 columns): in FP64 a 24-column panel leaves room for two CTAs per SM.
constexpr int kPanelLd = kBatchMaxN + 4;     // rows padded to a multiple of 4
constexpr int kSolveNb = 32, kSolveLd = kSolveNb + 1, kMaxRhs = 8;
constexpr int smem_elems(int maxnb)
{
    return maxnb * kPanelLd + kSolveNb * kSolveLd + kSolveNb * kMaxRhs + kSolveNb + 2;
}

// Four consecutive elements from shared memory (16-byte aligned).
__device__ __forceinline__ void ld4(const double *p, double (&v)[4])
{
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4(const float *p, float (&v)[4])
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

// The FP32 panel in registers: the kb x kb diagonal block by warp 0 (lane r
// holds row r; each column's entries reach the other lanes by shuffles, so
// the block takes no barrier), then every row below it by one thread, solved
// against the block right-looking (l_rc = a_rc / l_cc, then a_rq -= l_rc l_qc
// for q > c).  Each element sees the same operations in the same order as in
// the column loop of factor_one; only the barriers between columns go.
// Returns the failing column or -1 (the panel is then left as it was read).
template <typename T, int NB>
__device__ __forceinline__ int panel_in_registers(T *P, int kb, int rows, T *rinv, int *s_fail)
{
    constexpr int LDC = kPanelLd;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        T d[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) d[q] = (q < kb && lane < kb && q <= lane) ? P[q * LDC + lane] : T(0);
        int fail = -1;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            if (c < kb && fail < 0) {   // uniform across the warp
                const T piv = __shfl_sync(0xffffffffu, d[c], c);
                if (!(piv > T(0))) {
                    fail = c;
                } else {
                    const T sq = sqrt(piv), ri = T(1) / sq;
                    d[c] = lane == c ? sq : d[c] * ri;
                    if (lane == 0) rinv[c] = ri;
#pragma unroll
                    for (int q = 1; q < NB; ++q) {   // constant trip count: d stays in registers
                        if (q > c) {
                            const T lqc = __shfl_sync(0xffffffffu, d[c], q);
                            if (q < kb && lane >= q) d[q] -= d[c] * lqc;
                        }
                    }
                }
            }
        }
        if (fail < 0)
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < kb && lane < kb && q <= lane) P[q * LDC + lane] = d[q];
        if (lane == 0) *s_fail = fail;
    }
    __syncthreads();
    const int fail = *s_fail;
    if (fail >= 0) return fail;
    for (int r = kb + tid; r < rows; r += blockDim.x) {
        T a[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) a[q] = q < kb ? P[q * LDC + r] : T(0);
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            if (c < kb) {
                a[c] *= rinv[c];
#pragma unroll
                for (int q = c + 1; q < NB; ++q)
                    if (q < kb) a[q] -= a[c] * P[c * LDC + q];
            }
        }
#pragma unroll
        for (int q = 0; q < NB; ++q)
            if (q < kb) P[q * LDC + r] = a[q];
    }
    __syncthreads();
    return -1;
}

// Factor one matrix in place; returns 0 or the 1-based failing index.
template <typename T, int NB>
__device__ int factor_one(const Mat<T> &A, int64_t n, T *P, T *s_rinv, int *s_fail, T *rbuf)
{
    constexpr int LDC = kPanelLd;
    const int tid = threadIdx.x;
    for (int64_t k0 = 0; k0 < n; k0 += NB) {
        const int kb = (int)(n - k0 < NB ? n - k0 : NB);
        const int rows = (int)(n - k0);
        const int rpad = (rows + 3) & ~3;
        // 1. panel -> shared memory; zero above the diagonal and in the row
        // padding.  A thread's loads of one row go out eight at a time (one
        // L2 latency per eight elements instead of one per element).
        for (int r = tid; r < rpad; r += blockDim.x)
            for (int c0 = 0; c0 < kb; c0 += 8) {
                T v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int c = c0 + u;
                    v[u] = (c < kb && r >= c && r < rows) ? *A.at(k0 + r, k0 + c) : T(0);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (c0 + u < kb) P[(c0 + u) * LDC + r] = v[u];
            }
        if (tid == 0) *s_fail = -1;
        __syncthreads();
        // 2. right-looking Cholesky of the rows x kb panel: in registers in
        // FP32, whose pipe outruns the column loop's barriers; column by
        // column in FP64, whose pipe the column loop keeps busy
        if constexpr (sizeof(T) == 4) {
            const int f = panel_in_registers<T, NB>(P, kb, rows, rbuf, s_fail);
            if (f >= 0) return (int)(k0 + f + 1);
        } else
        for (int c = 0; c < kb; ++c) {
            if (tid == 0) {   // pivot; scale the panel's own rows c+1 .. kb-1 of column c
                const T d = P[c * LDC + c];
                if (!(d > T(0))) {
                    *s_fail = c;
                } else {
                    T sq, ri;
                    if constexpr (sizeof(T) == 8) {   // see rsqrt_newton
                        ri = rsqrt_newton(d);
                        sq = d * ri;
                    } else {
                        sq = sqrt(d);
                        ri = T(1) / sq;
                    }
                    P[c * LDC + c] = sq;
                    *s_rinv = ri;
                    for (int q = c + 1; q < kb; ++q) P[c * LDC + q] *= ri;
                }
            }
            __syncthreads();
            if (*s_fail >= 0) return (int)(k0 + *s_fail + 1);
            const T ri = *s_rinv;
            // row r: l_rc = a_rc / l_cc, then a_rq -= l_rc l_qc for c < q <= min(r, kb-1)
            for (int r = c + 1 + tid; r < rows; r += blockDim.x) {
                T lr = P[c * LDC + r];
                if (r >= kb) {
                    lr *= ri;
                    P[c * LDC + r] = lr;
                }
                const int qmax = r < kb - 1 ? r : kb - 1;
                for (int q = c + 1; q <= qmax; ++q) P[q * LDC + r] -= lr * P[c * LDC + q];
            }
            __syncthreads();
        }
        // 3a. panel back to the matrix
        for (int c = 0; c < kb; ++c)
            for (int r = c + tid; r < rows; r += blockDim.x) *A.at(k0 + r, k0 + c) = P[c * LDC + r];
        // 3b. trailing update of the lower triangle rows/cols >= k0 + kb, 4 x 4 tiles
        const int m = rows - kb;
        if (m > 0) {
            const int tm = (m + 3) / 4;
            const int ntiles = tm * (tm + 1) / 2;
            // Consecutive threads take consecutive tiles along the unit stride
            // of the block holding most of the trailing matrix (S, or T2 once
            // the panel is past T1): down a tile column when its columns are
            // contiguous, along a tile row otherwise.  Column order of the
            // lower tiles is the reverse of the row order of the same
            // triangle reflected about its anti-diagonal.
            const bool colfast = (k0 + kb >= A.n1 ? A.t2.rs : A.s.rs) == 1;
            for (int t = tid; t < ntiles; t += blockDim.x) {
                const int u = colfast ? ntiles - 1 - t : t;
                int ui = (int)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
                while ((ui + 1) * (ui + 2) / 2 <= u) ++ui;
                while (ui * (ui + 1) / 2 > u) --ui;
                const int uj = u - ui * (ui + 1) / 2;
                const int ti = colfast ? tm - 1 - uj : ui, tj = colfast ? tm - 1 - ui : uj;
                const T *pa = P + kb + 4 * ti, *pb = P + kb + 4 * tj;   // zero beyond `rows`
                // the tile's current values first: their load latency overlaps
                // the multiply-adds below (nothing in the loop writes them).
                // FP32: a tile inside one RFP block (all but those straddling
                // row or column n1) is addressed from that block's base with
                // 32-bit offsets, the FP32 pipe otherwise waiting on the address
                // arithmetic; FP64 goes through A.at, its pipe hiding that
                // arithmetic (and held addresses would cost it registers).
                const int64_t gi0 = k0 + kb + 4 * ti, gj0 = k0 + kb + 4 * tj;
                T *tb = nullptr;
                int trs = 0, tcs = 0;
                if constexpr (sizeof(T) == 4) {
                    const View<T> *blk = nullptr;
                    int64_t bi = gi0, bj = gj0;
                    if (gj0 >= A.n1) { blk = &A.t2; bi -= A.n1; bj -= A.n1; }
                    else if (gj0 + 3 < A.n1 && gi0 + 3 < A.n1) blk = &A.t1;
                    else if (gj0 + 3 < A.n1 && gi0 >= A.n1) { blk = &A.s; bi -= A.n1; }
                    if (blk) {
                        tb = blk->p + bi * blk->rs + bj * blk->cs;
                        trs = (int)blk->rs;
                        tcs = (int)blk->cs;
                    }
                }
                T cin[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int i = 4 * ti + u, j = 4 * tj + v;
                        const bool in = i < m && j <= i;
                        if constexpr (sizeof(T) == 4)
                            cin[u][v] = in ? (tb ? tb[u * trs + v * tcs] : *A.at(gi0 + u, gj0 + v)) : T(0);
                        else
                            cin[u][v] = in ? *A.at(k0 + kb + i, k0 + kb + j) : T(0);
                    }
                T acc[4][4] = {};
                for (int c = 0; c < kb; ++c) {
                    T a[4], b[4];
                    ld4(pa + c * LDC, a);
                    ld4(pb + c * LDC, b);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int i = 4 * ti + u, j = 4 * tj + v;
                        if (!(i < m && j <= i)) continue;
                        if constexpr (sizeof(T) == 4) {
                            T *q = tb ? tb + (u * trs + v * tcs) : A.at(gi0 + u, gj0 + v);
                            *q = cin[u][v] - acc[u][v];
                        } else {
                            *A.at(k0 + kb + i, k0 + kb + j) = cin[u][v] - acc[u][v];
                        }
                    }
            }
        }
        __syncthreads();
    }
    return 0;
}

// The solve's right-looking update after diagonal block [k0, k0 + kb):
// FWD: rows i >= k0 + kb get b_i -= L(i, block) y_block;
// !FWD: rows i < k0 get y_i -= L(block, i)^T x_block.
// One thread per row, R right-hand sides in registers.
template <typename T, bool FWD, int R>
__device__ __forceinline__ void rows_update_r(const Mat<T> &A, int64_t n, int64_t k0, int kb,
                                              T *Bm, int64_t ldb, const T *Y)
{
    const int64_t lo = FWD ? k0 + kb : 0, hi = FWD ? n : k0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        T acc[R] = {};
        // eight loads of the row of L issued together, then their products
        for (int c0 = 0; c0 < kb; c0 += 8) {
            T l[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + u;
                l[u] = c < kb ? (FWD ? *A.at(i, k0 + c) : *A.at(k0 + c, i)) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (c0 + u < kb)
#pragma unroll
                    for (int q = 0; q < R; ++q) acc[q] = fma(l[u], Y[(c0 + u) * kMaxRhs + q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) Bm[i + q * ldb] -= acc[q];
    }
}

template <typename T, bool FWD>
__device__ void rows_update(const Mat<T> &A, int64_t n, int64_t k0, int kb, T *Bm, int64_t ldb,
                            int nrhs, const T *Y)
{
    switch (nrhs) {
    case 1: rows_update_r<T, FWD, 1>(A, n, k0, kb, Bm, ldb, Y); break;
    case 2: rows_update_r<T, FWD, 2>(A, n, k0, kb, Bm, ldb, Y); break;
    case 3: rows_update_r<T, FWD, 3>(A, n, k0, kb, Bm, ldb, Y); break;
    case 4: rows_update_r<T, FWD, 4>(A, n, k0, kb, Bm, ldb, Y); break;
    case 5: rows_update_r<T, FWD, 5>(A, n, k0, kb, Bm, ldb, Y); break;
    case 6: rows_update_r<T, FWD, 6>(A, n, k0, kb, Bm, ldb, Y); break;
    case 7: rows_update_r<T, FWD, 7>(A, n, k0, kb, Bm, ldb, Y); break;
    default: rows_update_r<T, FWD, 8>(A, n, k0, kb, Bm, ldb, Y); break;
    }
}

// L L^T X = B in place for nrhs <= 8 columns (B column-major, ldb), by
// 32-row blocks.  Each diagonal block is solved by one warp per right-hand
// side (lane r holds row r; the finished value of row c is broadcast with a
// shuffle); the block's contribution to the remaining rows is then
// subtracted with one thread per row (right-looking).
template <typename T>
__device__ void solve_one(const Mat<T> &A, int64_t n, T *Bm, int64_t ldb, int nrhs, T *D, T *Y,
                          T *rdiag)
{
    constexpr int SB = kSolveNb, LDD = kSolveLd;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t nblk = (n + SB - 1) / SB;
    for (int e = tid; e < SB * kMaxRhs; e += blockDim.x) Y[e] = T(0);
    auto stage_diag = [&](int64_t k0, int kb) {
        // the block's (at most) 4 elements per thread loaded together
        constexpr int Q = (SB * SB + kBatchThreads - 1) / kBatchThreads;
        T v[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int e = tid + q * kBatchThreads, r = e % SB, c = e / SB;
            v[q] = (r < kb && c < kb && r >= c) ? *A.at(k0 + r, k0 + c) : T(0);
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int e = tid + q * kBatchThreads, r = e % SB, c = e / SB;
            if (r < kb && c < kb) D[r * LDD + c] = v[q];
        }
        __syncthreads();
        if (tid < kb) rdiag[tid] = T(1) / D[tid * LDD + tid];
        __syncthreads();
    };
    // forward: L y = b
    for (int64_t bk = 0; bk < nblk; ++bk) {
        const int64_t k0 = bk * SB;
        const int kb = (int)(n - k0 < SB ? n - k0 : SB);
        stage_diag(k0, kb);
        if (warp < nrhs) {
            T y = lane < kb ? Bm[k0 + lane + warp * ldb] : T(0);
            for (int c = 0; c < kb; ++c) {
                if (lane == c) y *= rdiag[c];
                const T yc = __shfl_sync(0xffffffffu, y, c);
                if (lane > c && lane < kb) y -= D[lane * LDD + c] * yc;
            }
            if (lane < kb) {
                Bm[k0 + lane + warp * ldb] = y;
                Y[lane * kMaxRhs + warp] = y;
            }
        }
        __syncthreads();
        rows_update<T, true>(A, n, k0, kb, Bm, ldb, nrhs, Y);   // b_i -= L(i, block) y_block
        __syncthreads();
    }
    // backward: L^T x = y
    for (int64_t bk = nblk - 1; bk >= 0; --bk) {
        const int64_t k0 = bk * SB;
        const int kb = (int)(n - k0 < SB ? n - k0 : SB);
        stage_diag(k0, kb);
        if (warp < nrhs) {
            T y = lane < kb ? Bm[k0 + lane + warp * ldb] : T(0);
            for (int c = kb - 1; c >= 0; --c) {
                if (lane == c) y *= rdiag[c];
                const T xc = __shfl_sync(0xffffffffu, y, c);
                if (lane < c) y -= D[c * LDD + lane] * xc;
            }
            if (lane < kb) {
                Bm[k0 + lane + warp * ldb] = y;
                Y[lane * kMaxRhs + warp] = y;
            }
        }
        __syncthreads();
        rows_update<T, false>(A, n, k0, kb, Bm, ldb, nrhs, Y);  // y_i -= L(block, i)^T x_block
        __syncthreads();
    }
}

template <typename T, int MAXNB>
__global__ void __launch_bounds__(kBatchThreads) batched_kernel(PlanHeader *hdr,
                                                                const PlanEntry *table,
                                                                int64_t batch, T *arf, T *B,
                                                                int32_t *info)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *P = reinterpret_cast<T *>(smem_raw);
    T *D = P + MAXNB * kPanelLd;
    T *Y = D + kSolveNb * kSolveLd;
    T *rdiag = Y + kSolveNb * kMaxRhs;
    T *s_rinv = rdiag + kSolveNb;
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
        const int nb = e.nb < MAXNB ? e.nb : MAXNB;
        int fail;
        if (nb == 16) fail = factor_one<T, 16>(A, e.n, P, s_rinv, &s_fail, rdiag);
        else if (MAXNB >= 24 && nb == 24)
            fail = factor_one<T, (MAXNB >= 24 ? 24 : 16)>(A, e.n, P, s_rinv, &s_fail, rdiag);
        else fail = factor_one<T, MAXNB>(A, e.n, P, s_rinv, &s_fail, rdiag);
        if (threadIdx.x == 0) info[e.index] = fail;
        __syncthreads();
        // up to kMaxRhs right-hand sides per pass; the factor (n <= 512) stays in L2
        for (int g = 0; fail == 0 && g < e.nrhs; g += kMaxRhs) {
            solve_one<T>(A, e.n, B + e.b + (int64_t)g * e.ldb, e.ldb,
                         e.nrhs - g < kMaxRhs ? e.nrhs - g : kMaxRhs, D, Y, rdiag);
            __syncthreads();
        }
        __syncthreads();
    }
}

// Resident CTAs of batched_kernel<T, MAXNB> on the current device (cached).
std::mutex g_ctas_mutex;
std::map<std::tuple<int, int, int>, int> g_ctas_cache;

template <typename T, int MAXNB>
int resident_ctas(int smem)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, (int)sizeof(T), MAXNB);
    {
        std::lock_guard<std::mutex> lock(g_ctas_mutex);
        auto it = g_ctas_cache.find(key);
        if (it != g_ctas_cache.end()) return it->second;
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<T, MAXNB>, kBatchThreads,
                                                  smem);
    const int ctas = std::max(1, per_sm) * device_sm_count();
    std::lock_guard<std::mutex> lock(g_ctas_mutex);
    g_ctas_cache[key] = ctas;
    return ctas;
}

// Widest panel of the plan last written at each d_plan address by this
// process; a launch is sized for it (32 when the address is unknown).
std::mutex g_plan_mutex;
std::map<const void *, int> g_plan_maxnb;

int plan_maxnb(const void *d_plan)
{
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    auto it = g_plan_maxnb.find(d_plan);
    return it == g_plan_maxnb.end() ? 32 : it->second;
}

template <typename T, int MAXNB>
cudaError_t launch_batched(int64_t batch, PlanHeader *hdr, const PlanEntry *table, T *arf, T *B,
                           int32_t *info, cudaStream_t st)
{
    const int smem = smem_elems(MAXNB) * (int)sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(batched_kernel<T, MAXNB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(batch, resident_ctas<T, MAXNB>(smem));
    batched_kernel<T, MAXNB><<<(unsigned)grid, kBatchThreads, smem, st>>>(hdr, table, batch, arf,
                                                                         B, info);
    return cudaSuccess;
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
                  e.arf + nt <= arf_len && (e.nb == 0 || e.nb == 16 || e.nb == 24 || e.nb == 32) &&
                  e.nrhs >= 0 &&
                  e.nrhs <= kBatchMaxRhs;
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
    int maxnb = 16;
    for (const PlanEntry &r : rows) maxnb = std::max(maxnb, (int)r.nb);
    std::stable_sort(rows.begin(), rows.end(),
                     [](const PlanEntry &a, const PlanEntry &b) { return a.n > b.n; });
    PlanHeader hdr;
    std::memset(&hdr, 0, sizeof hdr);
    cudaError_t err = cudaMemcpyAsync(d_plan, &hdr, sizeof hdr, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess && batch > 0)
        err = cudaMemcpyAsync(static_cast<char *>(d_plan) + sizeof hdr, rows.data(),
                              rows.size() * sizeof(PlanEntry), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);   // host staging is released below
    if (err == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_plan_mutex);
        g_plan_maxnb[d_plan] = maxnb;
    }
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
    cudaError_t e = cudaMemsetAsync(&hdr->counter, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const int maxnb = plan_maxnb(d_plan);
    if (maxnb <= 16) e = launch_batched<T, 16>(batch, hdr, table, arf, B, info, st);
    else if (maxnb <= 24) e = launch_batched<T, 24>(batch, hdr, table, arf, B, info, st);
    else e = launch_batched<T, 32>(batch, hdr, table, arf, B, info, st);
    if (e != cudaSuccess) return e;
    note_launch();
    return cudaGetLastError();
}

template cudaError_t batched_run<double>(int64_t, const void *, double *, double *, int32_t *,
                                         cudaStream_t);
template cudaError_t batched_run<float>(int64_t, const void *, float *, float *, int32_t *,
                                        cudaStream_t);

}  // namespace rfp
