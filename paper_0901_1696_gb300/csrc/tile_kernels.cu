// Tile kernels shared by PFTRF, PFTRS and PFTRI.
//
// The paper's four-step algorithms (Section 3: POTRF, TRSM, SYRK, POTRF;
// Section 4: TRSM, GEMM, TRSM; Section 5: TRTRI, TRMM, LAUUM, SYRK) are built
// here from five kernels:
//   gemm_nt_kernel    C = alpha A B^T + beta C on strided views, with optional
//                     triangle masks: the update, SYRK, GEMM and TRMM steps
//   trsm_right_kernel X op(L) = alpha X for a strip of rows, by substitution
//   potrf/trtri/lauum_tile_kernel   the diagonal-tile LAPACK steps
// In FP64 these kernels are bound by the FP64 pipe (sm_103a has no FP64
// tensor-core MMA), so the GEMM keeps 4x4 register tiles and double-buffered
// shared memory, which keeps one DFMA in flight per thread per cycle of
// shared-memory traffic; memory traffic is far below the HBM roofline.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <climits>

#include "rfp_internal.cuh"

namespace rfp {

// Tile configurations: BM x BN C tile, TM x TN per thread, BK-deep K steps.
template <typename T, int BM_, int BN_, int TM_, int TN_>
struct GemmCfg {
    static constexpr int BM = BM_, BN = BN_, BK = 16, TM = TM_, TN = TN_;
    static constexpr int TX = BN / TN, NT = (BM / TM) * (BN / TN);
    static constexpr int PAD = 16 / (int)sizeof(T);
    static_assert(NT % BM == 0 && NT % BN == 0 && NT % BK == 0, "loader mapping");
};
// FP64: 256 threads in every shape, so that a CTA alone on an SM keeps all
// four of its schedulers issuing to the FP64 pipe (small grids are common
// on the latency-bound chains); 2 x 2 per thread is enough reuse at FP64's
// arithmetic rate.  The strips are the in-place shapes (gemm_tile_choice).
template <typename T> struct GemmBig;
template <typename T> struct GemmSmall;
template <> struct GemmBig<double> { using C = GemmCfg<double, 64, 64, 4, 4>; };
template <> struct GemmSmall<double> { using C = GemmCfg<double, 32, 32, 2, 2>; };
using GemmColStrip = GemmCfg<double, 64, 16, 2, 2>;
using GemmRowStrip = GemmCfg<double, 16, 64, 2, 2>;
template <> struct GemmBig<float> { using C = GemmCfg<float, 128, 128, 8, 8>; };
template <> struct GemmSmall<float> { using C = GemmCfg<float, 64, 64, 4, 4>; };

template <typename T>
struct GemmArgs {
    View<T> C, A, B;
    int64_t M, N, K;
    T alpha, beta;
    int cmode, amask, bmask;
    const int32_t *abort;
    int64_t kchunk = 0;     // split-K: blockIdx.z covers K range [z kchunk, (z+1) kchunk)
    int64_t zstride = 0;    //          and writes C + z * zstride
};

template <typename T>
__device__ __forceinline__ void load_vec(T *dst, const T *src, int n)
{
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (i < n) dst[i] = src[i];
}

constexpr int64_t kGemmGroup = 16;   // row tiles per band of the grouped tile order

template <typename T, typename Cfg>
__global__ void __launch_bounds__(Cfg::NT) gemm_nt_kernel(GemmArgs<T> g)
{
    constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, TM = Cfg::TM, TN = Cfg::TN;
    constexpr int kGemmThreads = Cfg::NT;
    constexpr int LDA_S = BM + Cfg::PAD, LDB_S = BN + Cfg::PAD;
    constexpr int A_PER = BM * BK / kGemmThreads, B_PER = BN * BK / kGemmThreads;
    __shared__ __align__(16) T As[2][BK][LDA_S];
    __shared__ __align__(16) T Bs[2][BK][LDB_S];

    if (g.abort && *g.abort) return;
    // Grouped tile order: consecutive CTAs sweep the columns under a band of
    // kGemmGroup row tiles (column by column), so the CTAs resident at one
    // time share a few A and B strips and find them in L2.  A bijection of the
    // grid: every tile is still computed exactly once, by the same arithmetic.
    int64_t by = blockIdx.y, bx = blockIdx.x;
    if (gridDim.y > kGemmGroup) {
        const int64_t gx = gridDim.x, id = (int64_t)blockIdx.y * gx + blockIdx.x;
        const int64_t first = id / (kGemmGroup * gx) * kGemmGroup;
        const int64_t rows = gridDim.y - first < kGemmGroup ? gridDim.y - first : kGemmGroup;
        const int64_t r = id - first * gx;
        by = first + r % rows;
        bx = r / rows;
    }
    const int64_t m0 = by * BM, n0 = bx * BN;
    if (g.cmode == MASK_LOWER && m0 + BM - 1 < n0) return;   // tile strictly above diagonal

    // K range that can hold non-zero products for this tile.
    int64_t kbeg = 0, kend = g.K;
    if (g.kchunk > 0) {
        kbeg = (int64_t)blockIdx.z * g.kchunk;
        kend = min(kend, kbeg + g.kchunk);
        g.C.p += (int64_t)blockIdx.z * g.zstride;
    }
    if (g.amask == MASK_LOWER || g.amask == MASK_STRICT_LOWER) kend = min(kend, m0 + BM);
    if (g.amask == MASK_UPPER || g.amask == MASK_STRICT_UPPER) kbeg = max(kbeg, m0);
    if (g.bmask == MASK_LOWER || g.bmask == MASK_STRICT_LOWER) kend = min(kend, n0 + BN);
    if (g.bmask == MASK_UPPER || g.bmask == MASK_STRICT_UPPER) kbeg = max(kbeg, n0);
    const int64_t ntiles = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;

    const int tid = threadIdx.x, tx = tid % Cfg::TX, ty = tid / Cfg::TX;
    const bool a_mfast = (g.A.rs == 1), b_nfast = (g.B.rs == 1);

    T acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = T(0);

    T ra[A_PER], rb[B_PER];
    auto a_coord = [&](int q, int &mm, int &kk) {
        if (a_mfast) { mm = tid % BM; kk = tid / BM + q * (kGemmThreads / BM); }
        else { kk = tid % BK; mm = tid / BK + q * (kGemmThreads / BK); }
    };
    auto b_coord = [&](int q, int &nn, int &kk) {
        if (b_nfast) { nn = tid % BN; kk = tid / BN + q * (kGemmThreads / BN); }
        else { kk = tid % BK; nn = tid / BK + q * (kGemmThreads / BK); }
    };
    auto load_regs = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < A_PER; ++q) {
            int mm, kk;
            a_coord(q, mm, kk);
            const int64_t gm = m0 + mm, gk = k0 + kk;
            const bool ok = gm < g.M && gk < kend && mask_keeps(g.amask, gm, gk);
            ra[q] = ok ? g.A.p[gm * g.A.rs + gk * g.A.cs] : T(0);
        }
#pragma unroll
        for (int q = 0; q < B_PER; ++q) {
            int nn, kk;
            b_coord(q, nn, kk);
            const int64_t gn = n0 + nn, gk = k0 + kk;
            const bool ok = gn < g.N && gk < kend && mask_keeps(g.bmask, gn, gk);
            rb[q] = ok ? g.B.p[gn * g.B.rs + gk * g.B.cs] : T(0);
        }
    };
    auto store_smem = [&](int buf) {
#pragma unroll
        for (int q = 0; q < A_PER; ++q) {
            int mm, kk;
            a_coord(q, mm, kk);
            As[buf][kk][mm] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < B_PER; ++q) {
            int nn, kk;
            b_coord(q, nn, kk);
            Bs[buf][kk][nn] = rb[q];
        }
    };

    if (ntiles > 0) {
        load_regs(kbeg);
        store_smem(0);
        __syncthreads();
        for (int64_t t = 0; t < ntiles; ++t) {
            const int buf = (int)(t & 1);
            if (t + 1 < ntiles) load_regs(kbeg + (t + 1) * BK);
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                T a[TM], b[TN];
                load_vec(a, &As[buf][kk][ty * TM], TM);
                load_vec(b, &Bs[buf][kk][tx * TN], TN);
#pragma unroll
                for (int r = 0; r < TM; ++r)
#pragma unroll
                    for (int c = 0; c < TN; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
            }
            if (t + 1 < ntiles) store_smem(buf ^ 1);
            __syncthreads();
        }
    }

    // Epilogue: every C load is issued before the first store (stores may
    // alias the loads as far as the compiler can tell), then C is written.
    T cin[TM][TN];
    if (g.beta != T(0)) {
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                const int64_t i = m0 + ty * TM + r, j = n0 + tx * TN + c;
                const bool ok = i < g.M && j < g.N && !(g.cmode == MASK_LOWER && j > i);
                cin[r][c] = ok ? g.C.p[i * g.C.rs + j * g.C.cs] : T(0);
            }
    }
#pragma unroll
    for (int r = 0; r < TM; ++r) {
        const int64_t i = m0 + ty * TM + r;
        if (i >= g.M) continue;
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int64_t j = n0 + tx * TN + c;
            if (j >= g.N) continue;
            if (g.cmode == MASK_LOWER && j > i) continue;
            T v = g.alpha * acc[r][c];
            if (g.beta != T(0)) v = fma(g.beta, cin[r][c], v);
            g.C.p[i * g.C.rs + j * g.C.cs] = v;
        }
    }
}

template <typename T, typename Cfg>
static void launch_gemm(cudaStream_t st, const GemmArgs<T> &g, unsigned splits = 1)
{
    dim3 grid((unsigned)((g.N + Cfg::BN - 1) / Cfg::BN), (unsigned)((g.M + Cfg::BM - 1) / Cfg::BM),
              splits);
    gemm_nt_kernel<T, Cfg><<<grid, Cfg::NT, 0, st>>>(g);
}

// C = beta C + alpha sum_z W_z, W_z dense column-major M x N slices, summed in
// increasing z (the same order on every run).
template <typename T>
__global__ void splitk_reduce_kernel(View<T> C, const T *W, int64_t M, int64_t N, int splits,
                                     T alpha, T beta, int cmode, const int32_t *abort)
{
    if (abort && *abort) return;
    const int64_t total = M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % M, j = e / M;
        if (cmode == MASK_LOWER && j > i) continue;
        T s = T(0);
        for (int z = 0; z < splits; ++z) s += W[(int64_t)z * total + e];
        T v = alpha * s;
        if (beta != T(0)) v = fma(beta, C(i, j), v);
        C(i, j) = v;
    }
}

template <typename T>
cudaError_t gemm_nt_splitk(cudaStream_t st, View<T> C, View<T> A, View<T> B, int64_t M, int64_t N,
                           int64_t K, T alpha, T beta, int cmode, int amask, int bmask,
                           const int32_t *abort, int splits, T *work)
{
    if (splits <= 1 || !work) return gemm_nt(st, C, A, B, M, N, K, alpha, beta, cmode, amask, bmask, abort);
    if (M <= 0 || N <= 0) return cudaSuccess;
    GemmArgs<T> g{View<T>{work, 1, M}, A, B, M, N, K, T(1), T(0), cmode, amask, bmask, abort};
    g.kchunk = (K + splits - 1) / splits;
    g.zstride = M * N;
    int occ_big = 1, occ_small = 1;
    gemm_occupancy((int)sizeof(T), &occ_big, &occ_small);
    const GemmTileChoice tc = gemm_tile_choice(M, N, cmode, GEMM_INPLACE_NONE, (int)sizeof(T),
                                               device_sm_count(), occ_big, occ_small, splits);
    if (tc.kind == GEMM_TILE_SMALL) launch_gemm<T, typename GemmSmall<T>::C>(st, g, (unsigned)splits);
    else launch_gemm<T, typename GemmBig<T>::C>(st, g, (unsigned)splits);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>((M * N + 255) / 256, 4096);
    splitk_reduce_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(C, work, M, N, splits, alpha, beta,
                                                            cmode, abort);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t gemm_nt(cudaStream_t st, View<T> C, View<T> A, View<T> B, int64_t M, int64_t N,
                    int64_t K, T alpha, T beta, int cmode, int amask, int bmask,
                    const int32_t *abort, int inplace)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K <= 0 && beta == T(1)) return cudaSuccess;
    GemmArgs<T> g{C, A, B, M, N, K, alpha, beta, cmode, amask, bmask, abort};
    int occ_big = 1, occ_small = 1;
    gemm_occupancy((int)sizeof(T), &occ_big, &occ_small);
    const GemmTileChoice tc = gemm_tile_choice(M, N, cmode, inplace, (int)sizeof(T),
                                               device_sm_count(), occ_big, occ_small);
    if (tc.kind == GEMM_TILE_SMALL) launch_gemm<T, typename GemmSmall<T>::C>(st, g);
    else if constexpr (sizeof(T) == 8) {
        if (tc.kind == GEMM_TILE_COLSTRIP) launch_gemm<T, GemmColStrip>(st, g);
        else if (tc.kind == GEMM_TILE_ROWSTRIP) launch_gemm<T, GemmRowStrip>(st, g);
        else launch_gemm<T, typename GemmBig<T>::C>(st, g);
    } else launch_gemm<T, typename GemmBig<T>::C>(st, g);
    note_launch();
    return cudaGetLastError();
}

// Per-device caches of launch properties.  Several host threads may fill one
// at the same time (the serving loop's scheduler and a caller's own thread):
// they compute the same values; the small-tile figure is published before the
// large-tile one, whose release store marks the entry complete.
void gemm_occupancy(int elem_size, int *occ_big, int *occ_small)
{
    static std::atomic<int> cache[64][2][2] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    const int e = elem_size == 8 ? 0 : 1;
    if (!cache[dev][e][0].load(std::memory_order_acquire)) {
        int b = 1, sm = 1;
        if (elem_size == 8) {
            using Cb = GemmBig<double>::C;
            using Cs = GemmSmall<double>::C;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gemm_nt_kernel<double, Cb>, Cb::NT, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sm, gemm_nt_kernel<double, Cs>, Cs::NT, 0);
        } else {
            using Cb = GemmBig<float>::C;
            using Cs = GemmSmall<float>::C;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gemm_nt_kernel<float, Cb>, Cb::NT, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sm, gemm_nt_kernel<float, Cs>, Cs::NT, 0);
        }
        cache[dev][e][1].store(sm > 0 ? sm : 1, std::memory_order_relaxed);
        cache[dev][e][0].store(b > 0 ? b : 1, std::memory_order_release);
    }
    *occ_big = cache[dev][e][0].load(std::memory_order_acquire);
    *occ_small = cache[dev][e][1].load(std::memory_order_relaxed);
}

int device_sm_count()
{
    static std::atomic<int> cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int sms = cache[dev].load(std::memory_order_relaxed);
    if (!sms) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            return 152;
        cache[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

// ---------------------------------------------------------------------------
// Strip triangular solve: X op(L) = alpha X, 64 rows per CTA, w <= 64.

constexpr int kTileMax = 64, kTileLd = 65, kStripRows = 64;
constexpr int kTileThreads = 256;

// Tile loaders with a compile-time trip count: every thread issues all its
// global loads before its first shared-memory store, so a 64 x 64 tile costs
// one load latency rather than one per loop iteration.  Element (i, j) of the
// 64 x 64 index space is read when (i, j) is inside the w x w (or rows x w)
// block and keep(i, j) holds; the shared tile gets `fill(i, j)` elsewhere.
template <int NT, typename T, typename Keep, typename Fill>
__device__ __forceinline__ void load_tile64(T *S, View<T> A, int rows, int w, Keep keep, Fill fill,
                                            T scale = T(1))
{
    constexpr int IT = kTileMax * kTileMax / NT;
    const bool rowfast = A.rs == 1;
    T v[IT];
#pragma unroll
    for (int q = 0; q < IT; ++q) {
        const int e = threadIdx.x + q * NT, a = e % kTileMax, b = e / kTileMax;
        const int i = rowfast ? a : b, j = rowfast ? b : a;
        v[q] = (i < rows && j < w && keep(i, j)) ? scale * A(i, j) : T(0);
    }
#pragma unroll
    for (int q = 0; q < IT; ++q) {
        const int e = threadIdx.x + q * NT, a = e % kTileMax, b = e / kTileMax;
        const int i = rowfast ? a : b, j = rowfast ? b : a;
        S[i * kTileLd + j] = (i < rows && j < w && keep(i, j)) ? v[q] : fill(i, j);
    }
}

template <typename T>
struct TrsmArgs {
    View<T> X, L;
    int64_t M;
    int w, transL;
    T alpha;
    const int32_t *abort;
    int unit;   // unit diagonal: the triangle's diagonal is taken as 1 and never read
};

template <typename T>
__global__ void __launch_bounds__(256) trsm_right_kernel(TrsmArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ls = reinterpret_cast<T *>(smem_raw);
    T *Xs = Ls + kTileMax * kTileLd;
    if (a.abort && *a.abort) return;
    const int tid = threadIdx.x, w = a.w;
    const int64_t r0 = (int64_t)blockIdx.x * kStripRows;

    const int unit = a.unit;
    load_tile64<kTileThreads>(Ls, a.L, w, w, [unit](int i, int j) { return unit ? i > j : i >= j; },
                              [unit](int i, int j) { return (unit && i == j) ? T(1) : T(0); });
    const int64_t rows_left = a.M - r0;
    const int rows = (int)(rows_left < kStripRows ? rows_left : kStripRows);
    View<T> Xv = a.X.sub(r0, 0);
    const T alpha = a.alpha;
    load_tile64<kTileThreads>(Xs, Xv, rows, w, [](int, int) { return true; },
                              [](int, int) { return T(0); }, alpha);
    __syncthreads();

    const int row = tid % kStripRows, grp = tid / kStripRows;   // 4 column groups
    T *xr = Xs + row * kTileLd;
    // Reciprocals of the pivots, formed once (row tid of the diagonal): a
    // division per row per step would dominate on GB300's narrow FP64 pipe.
    T *rinv = Xs + kTileMax * kTileLd;
    if (tid < w) rinv[tid] = T(1) / Ls[tid * kTileLd + tid];
    __syncthreads();
    if (a.transL) {                  // X L^T = B: columns in increasing order
        for (int j = 0; j < w; ++j) {
            if (grp == 0) xr[j] = xr[j] * rinv[j];
            __syncthreads();
            const T xj = xr[j];
            for (int c = j + 1 + grp; c < w; c += 4) xr[c] -= xj * Ls[c * kTileLd + j];
            __syncthreads();
        }
    } else {                         // X L = B: columns in decreasing order
        for (int j = w - 1; j >= 0; --j) {
            if (grp == 0) xr[j] = xr[j] * rinv[j];
            __syncthreads();
            const T xj = xr[j];
            for (int c = grp; c < j; c += 4) xr[c] -= xj * Ls[j * kTileLd + c];
            __syncthreads();
        }
    }

    {
        constexpr int IT = kTileMax * kTileMax / kTileThreads;
        const bool xrow = (a.X.rs == 1);
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int e = tid + q * kTileThreads, p1 = e % kTileMax, p2 = e / kTileMax;
            const int rr = xrow ? p1 : p2, cc = xrow ? p2 : p1;
            if (rr < rows && cc < w) Xv(rr, cc) = Xs[rr * kTileLd + cc];
        }
    }
}

// FP32 variant: one thread solves one row of X entirely in registers against
// the 64 x 64 triangle in shared memory (padded with the identity when w < 64),
// with no barrier inside the substitution.  In FP32 the per-column barriers
// of trsm_right_kernel, not the arithmetic, bound a diagonal-block solve;
// FP64 keeps trsm_right_kernel, whose four threads per row spread the FP64
// work over more of the SM's pipes.
constexpr int kRowsPerCta = 128;

template <int TRANSL>
__global__ void __launch_bounds__(kRowsPerCta) trsm_rows_f32_kernel(TrsmArgs<float> a)
{
    __shared__ float Ls[kTileMax][kTileMax + 1];
    if (a.abort && *a.abort) return;
    const int w = a.w;
    const int unit = a.unit;
    load_tile64<kRowsPerCta>(&Ls[0][0], a.L, w, w,
                             [unit](int i, int j) { return unit ? i > j : i >= j; },
                             [w, unit](int i, int j) { return (i == j && (unit || i >= w)) ? 1.f : 0.f; });
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * kRowsPerCta + threadIdx.x;
    if (r >= a.M) return;
    float x[kTileMax];
#pragma unroll
    for (int c = 0; c < kTileMax; ++c) x[c] = (c < w) ? a.alpha * a.X(r, c) : 0.f;
    // Right-looking order: once x_j is final, its contribution is removed
    // from every later x_c at once, so each step issues up to 63 independent
    // FMAs (the per-element summation order is the same ascending order as
    // the dot-product form).
    if (TRANSL) {            // X L^T = B: x_j = (b_j - sum_{k<j} L(j,k) x_k) / L(j,j)
#pragma unroll
        for (int j = 0; j < kTileMax; ++j) {
            x[j] = x[j] / Ls[j][j];
#pragma unroll
            for (int c = j + 1; c < kTileMax; ++c) x[c] -= Ls[c][j] * x[j];
        }
    } else {                 // X L = B: x_j = (b_j - sum_{k>j} L(k,j) x_k) / L(j,j)
#pragma unroll
        for (int j = kTileMax - 1; j >= 0; --j) {
            x[j] = x[j] / Ls[j][j];
#pragma unroll
            for (int c = 0; c < j; ++c) x[c] -= Ls[j][c] * x[j];
        }
    }
#pragma unroll
    for (int c = 0; c < kTileMax; ++c)
        if (c < w) a.X(r, c) = x[c];
}

template <typename T>
static cudaError_t set_smem_once(const void *fn, int bytes)
{
    // The opt-in above 48 KB is a per-function, per-device attribute; setting
    // it again is harmless, so no cache is kept.
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename T>
cudaError_t trsm_strip(cudaStream_t st, View<T> X, View<T> Ltri, int64_t M, int w, int transL,
                       T alpha, const int32_t *abort, bool unit)
{
    if (M <= 0 || w <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        TrsmArgs<float> a{X, Ltri, M, w, transL, alpha, abort, unit ? 1 : 0};
        const unsigned grid = (unsigned)((M + kRowsPerCta - 1) / kRowsPerCta);
        if (transL) trsm_rows_f32_kernel<1><<<grid, kRowsPerCta, 0, st>>>(a);
        else trsm_rows_f32_kernel<0><<<grid, kRowsPerCta, 0, st>>>(a);
        note_launch();
        return cudaGetLastError();
    }
    const int smem = (2 * kTileMax * kTileLd + kTileMax) * (int)sizeof(T);
    cudaError_t e = set_smem_once<T>((const void *)trsm_right_kernel<T>, smem);
    if (e != cudaSuccess) return e;
    TrsmArgs<T> a{X, Ltri, M, w, transL, alpha, abort, unit ? 1 : 0};
    const unsigned grid = (unsigned)((M + kStripRows - 1) / kStripRows);
    trsm_right_kernel<T><<<grid, 256, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagonal tiles (one CTA each).

template <typename T>
__device__ __forceinline__ void load_lower_tile(T *S, View<T> A, int w)
{
    load_tile64<kTileThreads>(S, A, w, w, [](int i, int j) { return i >= j; },
                              [](int, int) { return T(0); });
}

template <typename T>
__device__ __forceinline__ void store_lower_tile(View<T> A, const T *S, int w)
{
    constexpr int IT = kTileMax * kTileMax / kTileThreads;
    const bool rowfast = A.rs == 1;
#pragma unroll
    for (int q = 0; q < IT; ++q) {
        const int e = threadIdx.x + q * kTileThreads, p1 = e % kTileMax, p2 = e / kTileMax;
        const int i = rowfast ? p1 : p2, j = rowfast ? p2 : p1;
        if (i < w && j < w && i >= j) A(i, j) = S[i * kTileLd + j];
    }
}

// Unblocked right-looking Cholesky of one tile, l_ij = a_ij * (1 / sqrt(pivot))
// (LAPACK's unblocked Cholesky also scales a column by the reciprocal of its
// diagonal).
// FP64: at step j one thread forms the pivot's reciprocal square root y
// (Newton-Raphson, rsqrt_newton) and l_jj = d y (on GB300's narrow FP64
// pipe a square root and a division per step, let alone per thread, would
// cost more than the step's multiply-adds), the column is scaled in
// place, and the trailing triangle is updated by a 16 x 16 grid of threads
// (one DFMA per element); three barriers per column.
// FP32: one barrier per column; each thread forms the pivot's reciprocal and
// the scaled values it needs, and the columns are scaled on write-back.
template <typename T>
__global__ void __launch_bounds__(256) potrf_tile_kernel(View<T> A, int w, int32_t *info,
                                                         int64_t base)
{
    __shared__ __align__(16) T S[kTileMax * kTileLd];
    __shared__ T rinv[kTileMax], sq[kTileMax];
    __shared__ int s_fail;
    if (*info != 0) return;
    load_lower_tile(S, A, w);
    __syncthreads();
    int fail = -1;
    if constexpr (sizeof(T) == 8) {
        const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
        for (int j = 0; j < w; ++j) {
            if (threadIdx.x == 0) {
                const T d = S[j * kTileLd + j];
                s_fail = (d > T(0)) ? -1 : j;              // pivot <= 0 or NaN fails
                const T y = rsqrt_newton(d);
                sq[j] = d * y;
                rinv[j] = y;
            }
            __syncthreads();
            if (s_fail >= 0) { fail = s_fail; break; }
            const T ri = rinv[j];
            for (int i = j + 1 + threadIdx.x; i < w; i += blockDim.x) S[i * kTileLd + j] *= ri;
            __syncthreads();
            for (int i = j + 1 + ty; i < w; i += 16) {
                const T lij = S[i * kTileLd + j];
                for (int k = j + 1 + tx; k <= i; k += 16) S[i * kTileLd + k] -= lij * S[k * kTileLd + j];
            }
            __syncthreads();
        }
    } else {
        for (int j = 0; j < w; ++j) {
            const T d = S[j * kTileLd + j];
            if (!(d > T(0))) { fail = j; break; }      // every thread sees the same d
            const T r = sqrt(d), ri = T(1) / r;
            if (threadIdx.x == 0) { sq[j] = r; rinv[j] = ri; }
            const int rem = w - j - 1;
            for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
                const int i = j + 1 + e / rem, k = j + 1 + e % rem;
                if (k <= i) S[i * kTileLd + k] -= (S[i * kTileLd + j] * ri) * (S[k * kTileLd + j] * ri);
            }
            __syncthreads();
        }
    }
    if (fail >= 0) {
        if (threadIdx.x == 0) *info = (int32_t)(base + fail + 1);
        return;
    }
    constexpr int IT = kTileMax * kTileMax / kTileThreads;
    const bool rowfast = A.rs == 1;
#pragma unroll
    for (int q = 0; q < IT; ++q) {
        const int e = threadIdx.x + q * kTileThreads, p1 = e % kTileMax, p2 = e / kTileMax;
        const int i = rowfast ? p1 : p2, j = rowfast ? p2 : p1;
        if (i >= w || j >= w || i < j) continue;
        if (i > j) A(i, j) = sizeof(T) == 8 ? S[i * kTileLd + j] : S[i * kTileLd + j] * rinv[j];
        else A(i, j) = sq[j];
    }
}

template <typename T>
cudaError_t potrf_tile(cudaStream_t st, View<T> A, int w, int32_t *info, int64_t base)
{
    if (w <= 0) return cudaSuccess;
    potrf_tile_kernel<T><<<1, 256, 0, st>>>(A, w, info, base);
    note_launch();
    return cudaGetLastError();
}

// Inverse of one lower-triangular tile: column c of W = L^{-1} by forward
// substitution, W(c, c) = 1 / L(c, c) and, for i > c,
//   W(i, c) = -(sum_{p = c}^{i-1} L(i, p) W(p, c)) / L(i, i).
// Four lanes of one warp share a column: each sums every fourth term, the
// partial sums are combined by shuffles inside the group of four, and the
// group's first lane writes W(i, c).  The diagonal's reciprocals are formed
// once, in parallel (a division per element would dominate on GB300's narrow
// FP64 pipe).
template <typename T>
__global__ void __launch_bounds__(256) trtri_tile_kernel(View<T> A, int w, const int32_t *abort)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ls = reinterpret_cast<T *>(smem_raw);
    T *Ws = Ls + kTileMax * kTileLd;
    T *rinv = Ws + kTileMax * kTileLd;
    if (abort && *abort) return;
    load_lower_tile(Ls, A, w);
    __syncthreads();
    if ((int)threadIdx.x < w) rinv[threadIdx.x] = T(1) / Ls[threadIdx.x * kTileLd + threadIdx.x];
    __syncthreads();
    const int c = threadIdx.x / 4, part = threadIdx.x % 4;
    const int lane = threadIdx.x % 32;
    const unsigned group = 0xFu << (lane & ~3);   // this column's four lanes
    if (c < w) {
        if (part == 0) Ws[c * kTileLd + c] = rinv[c];
        __syncwarp(group);
        for (int i = c + 1; i < w; ++i) {
            T s = T(0);
            for (int p = c + part; p < i; p += 4) s += Ls[i * kTileLd + p] * Ws[p * kTileLd + c];
            s += __shfl_xor_sync(group, s, 1);
            s += __shfl_xor_sync(group, s, 2);
            if (part == 0) Ws[i * kTileLd + c] = -s * rinv[i];
            __syncwarp(group);   // W(i, c) visible to the group's next sums
        }
    }
    __syncthreads();
    store_lower_tile(A, Ws, w);
}

template <typename T>
cudaError_t trtri_tile(cudaStream_t st, View<T> A, int w, const int32_t *abort)
{
    if (w <= 0) return cudaSuccess;
    const int smem = (2 * kTileMax * kTileLd + kTileMax) * (int)sizeof(T);
    cudaError_t e = set_smem_once<T>((const void *)trtri_tile_kernel<T>, smem);
    if (e != cudaSuccess) return e;
    trtri_tile_kernel<T><<<1, 256, smem, st>>>(A, w, abort);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Inverses of the kInvBlock-wide diagonal blocks of an FP32 lower triangle,
// one CTA per block.  Thread c forms column c of W = L_bb^{-1} by forward
// substitution on L_bb e_c, i.e. W(c, c) = 1 / L(c, c) and, for i > c,
//   W(i, c) = -(sum_{p = c}^{i-1} L(i, p) W(p, c)) / L(i, i).
// Both triangles sit in shared memory (2 x 128 x 129 floats).

constexpr int kInvThreads = (int)kInvBlock, kInvLd = (int)kInvBlock + 1;

__global__ void __launch_bounds__(kInvThreads) inv_diag_kernel(View<float> V, int64_t m,
                                                                float *Inv, const int32_t *abort)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *Ls = reinterpret_cast<float *>(smem_raw);
    float *Ws = Ls + kInvBlock * kInvLd;
    if (abort && *abort) return;
    const int64_t k0 = (int64_t)blockIdx.x * kInvBlock;
    const int w = (int)(m - k0 < kInvBlock ? m - k0 : kInvBlock);
    const int t = threadIdx.x;
    const bool rowfast = V.rs == 1;
    View<float> Vb = V.sub(k0, k0);
    for (int q = 0; q < (int)kInvBlock; ++q) {     // coalesced along V's unit-stride index
        const int i = rowfast ? t : q, j = rowfast ? q : t;
        Ls[i * kInvLd + j] = (i < w && j <= i) ? Vb(i, j) : 0.f;
    }
    __syncthreads();
    const int c = t;
    for (int i = 0; i < (int)kInvBlock; ++i) Ws[i * kInvLd + c] = 0.f;
    if (c < w) {
        Ws[c * kInvLd + c] = 1.f / Ls[c * kInvLd + c];
        for (int i = c + 1; i < w; ++i) {
            float s = 0.f;
            for (int p = c; p < i; ++p) s += Ls[i * kInvLd + p] * Ws[p * kInvLd + c];
            Ws[i * kInvLd + c] = -s / Ls[i * kInvLd + i];
        }
    }
    __syncthreads();
    float *out = Inv + (int64_t)blockIdx.x * kInvBlock * kInvBlock;   // column-major, ld kInvBlock
    for (int j = 0; j < (int)kInvBlock; ++j) out[(int64_t)j * kInvBlock + t] = Ws[t * kInvLd + j];
}

cudaError_t inv_diag_blocks(cudaStream_t st, View<float> V, int64_t m, float *Inv,
                            const int32_t *abort)
{
    if (m <= 0) return cudaSuccess;
    const int smem = 2 * (int)kInvBlock * kInvLd * (int)sizeof(float);
    cudaError_t e = set_smem_once<float>((const void *)inv_diag_kernel, smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((m + kInvBlock - 1) / kInvBlock);
    inv_diag_kernel<<<grid, kInvThreads, smem, st>>>(V, m, Inv, abort);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) lauum_tile_kernel(View<T> A, int w, const int32_t *abort)
{
    __shared__ __align__(16) T Ws[kTileMax * kTileLd];
    if (abort && *abort) return;
    load_lower_tile(Ws, A, w);
    __syncthreads();
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        int i, j;
        if (A.rs == 1) { i = e % w; j = e / w; } else { j = e % w; i = e / w; }
        if (i < j) continue;
        T s = T(0);
        for (int k = i; k < w; ++k) s += Ws[k * kTileLd + i] * Ws[k * kTileLd + j];
        A(i, j) = s;
    }
}

template <typename T>
cudaError_t lauum_tile(cudaStream_t st, View<T> A, int w, const int32_t *abort)
{
    if (w <= 0) return cudaSuccess;
    lauum_tile_kernel<T><<<1, 256, 0, st>>>(A, w, abort);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(1024) check_diag_kernel(View<T> t1, int64_t n1, View<T> t2,
                                                          int64_t n2, int32_t *info)
{
    __shared__ unsigned long long best;
    if (threadIdx.x == 0) best = ULLONG_MAX;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
        const T d = i < n1 ? t1(i, i) : t2(i - n1, i - n1);
        if (d == T(0)) {
            atomicMin(&best, (unsigned long long)i);
            break;   // later indices of this thread are larger
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *info = best == ULLONG_MAX ? 0 : (int32_t)(best + 1);
}

template <typename T>
cudaError_t check_diag(cudaStream_t st, View<T> t1, int64_t n1, View<T> t2, int64_t n2,
                       int32_t *info)
{
    check_diag_kernel<T><<<1, 1024, 0, st>>>(t1, n1, t2, n2, info);
    note_launch();
    return cudaGetLastError();
}

// dst = I (mode 0) or dst(i, j) = src(i, j) for j <= i (mode 1), m x m; one
// thread per element along dst's unit stride, grid-stride.
__global__ void tri_fill_kernel(View<double> dst, View<double> src, int64_t m, int mode,
                                const int32_t *abort)
{
    if (abort && *abort) return;
    const bool rowfast = dst.rs == 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = e % m, v = e / m;
        const int64_t i = rowfast ? u : v, j = rowfast ? v : u;
        if (mode == 0) dst(i, j) = i == j ? 1.0 : 0.0;
        else if (j <= i) dst(i, j) = src(i, j);
    }
}

static cudaError_t tri_fill(cudaStream_t st, View<double> dst, View<double> src, int64_t m, int mode,
                            const int32_t *abort)
{
    if (m <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((m * m + 255) / 256, 8 * (int64_t)device_sm_count());
    tri_fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(dst, src, m, mode, abort);
    note_launch();
    return cudaGetLastError();
}

cudaError_t identity_fill(cudaStream_t st, View<double> W, int64_t m, const int32_t *abort)
{
    return tri_fill(st, W, W, m, 0, abort);
}

cudaError_t lower_copy(cudaStream_t st, View<double> dst, View<double> src, int64_t m,
                       const int32_t *abort)
{
    return tri_fill(st, dst, src, m, 1, abort);
}

#define RFP_INSTANTIATE(T)                                                                    \
    template cudaError_t gemm_nt<T>(cudaStream_t, View<T>, View<T>, View<T>, int64_t, int64_t, \
                                    int64_t, T, T, int, int, int, const int32_t *, int);      \
    template cudaError_t gemm_nt_splitk<T>(cudaStream_t, View<T>, View<T>, View<T>, int64_t,   \
                                           int64_t, int64_t, T, T, int, int, int,             \
                                           const int32_t *, int, T *);                        \
    template cudaError_t trsm_strip<T>(cudaStream_t, View<T>, View<T>, int64_t, int, int, T,  \
                                       const int32_t *, bool);                                \
    template cudaError_t potrf_tile<T>(cudaStream_t, View<T>, int, int32_t *, int64_t);       \
    template cudaError_t trtri_tile<T>(cudaStream_t, View<T>, int, const int32_t *);          \
    template cudaError_t lauum_tile<T>(cudaStream_t, View<T>, int, const int32_t *);          \
    template cudaError_t check_diag<T>(cudaStream_t, View<T>, int64_t, View<T>, int64_t,      \
                                       int32_t *);
RFP_INSTANTIATE(double)
RFP_INSTANTIATE(float)
#undef RFP_INSTANTIATE

}  // namespace rfp
