// TRTTF / TFTTR (Table "lapack"): full <-> RFPF copies.
//
// Pure data movement, bound by HBM bandwidth: each element of the stored
// triangle is read once and written once (8 n(n+1) bytes per FP64 call).
// The three blocks T1, S and T2 are cut into 64 x 64 tiles; each CTA copies
// one tile through shared memory so that both the read and the write walk
// their array's unit-stride direction (a transposed block such as T2 = L22^T
// under TRANSR='N' is a shared-memory transpose).  Tiles on the diagonal of
// T1 / T2 copy only i >= j, so the other triangle of A is never read (pack)
// nor written (unpack), and the copy is bit-exact.
#include "rfp_internal.cuh"

namespace rfp {

constexpr int kPackTile = 64, kPackThreads = 256;
constexpr int kPackPer = kPackTile * kPackTile / kPackThreads;   // 16 elements per thread

template <typename T>
struct PackArgs {
    T *A;
    int64_t lda;
    int lowerA;             // 1: A's lower triangle is stored (UPLO='L')
    T *arf;
    int64_t ld;
    int64_t n1, n2;
    Block t1, s, t2;
    int64_t nt1, nt2, ntri1, nrect;
    int unpack;
};

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

// Row/column of the t-th tile of a lower-triangular tile grid (row-major).
__device__ __forceinline__ void tri_tile(int64_t t, int64_t &ti, int64_t &tj)
{
    // single-precision guess (the FP64 pipe is narrow), corrected below
    int64_t r = (int64_t)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    ti = r;
    tj = t - r * (r + 1) / 2;
}

template <typename T>
__global__ void __launch_bounds__(kPackThreads, 3) pack_kernel(PackArgs<T> a)
{
    __shared__ T tile[kPackTile][kPackTile + 1];
    const int64_t t = blockIdx.x;
    int64_t ti, tj, rows, cols, roff, coff;
    Block b;
    bool tri;
    if (t < a.ntri1) {
        tri_tile(t, ti, tj);
        rows = cols = a.n1; roff = coff = 0; b = a.t1; tri = true;
    } else if (t < a.ntri1 + a.nrect) {
        const int64_t u = t - a.ntri1;
        ti = u / a.nt1; tj = u % a.nt1;
        rows = a.n2; cols = a.n1; roff = a.n1; coff = 0; b = a.s; tri = false;
    } else {
        tri_tile(t - a.ntri1 - a.nrect, ti, tj);
        rows = cols = a.n2; roff = coff = a.n1; b = a.t2; tri = true;
    }
    const int64_t bi0 = ti * kPackTile, bj0 = tj * kPackTile;
    const int h = (int)(rows - bi0 < kPackTile ? rows - bi0 : kPackTile);
    const int wd = (int)(cols - bj0 < kPackTile ? cols - bj0 : kPackTile);

    // Logical block element (bi, bj) is A(roff+bi, coff+bj) of the stored
    // triangle (A(j, i) for UPLO='U') and X(bi, bj) of RFP block b.
    View<T> vA = a.lowerA ? View<T>{a.A + (roff + bi0) + (coff + bj0) * a.lda, 1, a.lda}
                          : View<T>{a.A + (coff + bj0) + (roff + bi0) * a.lda, a.lda, 1};
    View<T> vR = b.trans ? View<T>{a.arf + b.off + bj0 + bi0 * a.ld, a.ld, 1}
                         : View<T>{a.arf + b.off + bi0 + bj0 * a.ld, 1, a.ld};
    const View<T> src = a.unpack ? vR : vA;
    const View<T> dst = a.unpack ? vA : vR;

    // Thread (fast, slow): `fast` runs along the array's unit-stride index.
    const int fast = threadIdx.x % kPackTile, slow0 = threadIdx.x / kPackTile;
    constexpr int kSlowStep = kPackThreads / kPackTile;
    const bool src_rows = (src.rs == 1), dst_rows = (dst.rs == 1);

    // Valid elements: bi < h, bj < wd and, on a diagonal tile, bi0+bi >= bj0+bj.
    // For a thread whose fast index is bi (rows) or bj (columns) this is a
    // range [lo, hi) of its slow index.
    auto slow_range = [&](bool rows_fast, int &lo, int &hi) {
        const int f = fast;
        const int64_t d = bi0 - bj0;   // diagonal offset of the tile
        if (rows_fast) {               // bi = f, bj = slow
            hi = (f < h) ? wd : 0;
            if (tri) hi = (int)imin64(hi, imax64(0, d + f + 1));
            lo = 0;
        } else {                       // bj = f, bi = slow
            hi = (f < wd) ? h : 0;
            lo = tri ? (int)imax64(0, imin64(h, f - d)) : 0;
        }
    };
    int slo, shi;
    slow_range(src_rows, slo, shi);
    const int64_t sstride = src_rows ? src.cs : src.rs;
    const T *sp = src.p + fast + (int64_t)slow0 * sstride;

    T v[kPackPer];
#pragma unroll
    for (int q = 0; q < kPackPer; ++q) {
        const int sl = slow0 + q * kSlowStep;
        if (sl >= slo && sl < shi) v[q] = sp[(int64_t)q * kSlowStep * sstride];
    }
    if (src_rows == dst_rows) {
        // Both arrays are contiguous along the same index: store straight
        // from registers (same (fast, slow) ownership, same validity).
        const int64_t dstride = dst_rows ? dst.cs : dst.rs;
        T *dp = dst.p + fast + (int64_t)slow0 * dstride;
#pragma unroll
        for (int q = 0; q < kPackPer; ++q) {
            const int sl = slow0 + q * kSlowStep;
            if (sl >= slo && sl < shi) dp[(int64_t)q * kSlowStep * dstride] = v[q];
        }
        return;
    }
    // Transposed block: through shared memory, tile[bi][bj].
#pragma unroll
    for (int q = 0; q < kPackPer; ++q) {
        const int sl = slow0 + q * kSlowStep;
        if (sl >= slo && sl < shi) {
            if (src_rows) tile[fast][sl] = v[q];
            else tile[sl][fast] = v[q];
        }
    }
    __syncthreads();
    int dlo, dhi;
    slow_range(dst_rows, dlo, dhi);
    const int64_t dstride = dst_rows ? dst.cs : dst.rs;
    T *dp = dst.p + fast + (int64_t)slow0 * dstride;
#pragma unroll
    for (int q = 0; q < kPackPer; ++q) {
        const int sl = slow0 + q * kSlowStep;
        if (sl >= dlo && sl < dhi)
            dp[(int64_t)q * kSlowStep * dstride] = dst_rows ? tile[fast][sl] : tile[sl][fast];
    }
}

template <typename T>
cudaError_t pack_copy(cudaStream_t st, const Layout &L, bool lowerA, T *A, int64_t lda, T *arf,
                      bool unpack)
{
    PackArgs<T> a;
    a.A = A; a.lda = lda; a.lowerA = lowerA ? 1 : 0; a.arf = arf; a.ld = L.ld;
    a.n1 = L.n1; a.n2 = L.n2; a.t1 = L.t1; a.s = L.s; a.t2 = L.t2;
    a.nt1 = (L.n1 + kPackTile - 1) / kPackTile;
    a.nt2 = (L.n2 + kPackTile - 1) / kPackTile;
    a.ntri1 = a.nt1 * (a.nt1 + 1) / 2;
    a.nrect = a.nt2 * a.nt1;
    a.unpack = unpack ? 1 : 0;
    const int64_t ntiles = a.ntri1 + a.nrect + a.nt2 * (a.nt2 + 1) / 2;
    if (ntiles <= 0) return cudaSuccess;
    pack_kernel<T><<<(unsigned)ntiles, kPackThreads, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t pack_copy<double>(cudaStream_t, const Layout &, bool, double *, int64_t,
                                       double *, bool);
template cudaError_t pack_copy<float>(cudaStream_t, const Layout &, bool, float *, int64_t,
                                      float *, bool);

}  // namespace rfp
