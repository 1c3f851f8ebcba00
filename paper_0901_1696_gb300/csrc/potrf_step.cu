// FP64 Cholesky of one RFP triangle (PFTRF steps 1 and 4, Section 3) with a
// one-panel lookahead, one launch per panel step.
//
// Right-looking blocked Cholesky of the m x m lower triangle V with panels
// of width PW (32 for small triangles, 64 beyond): after panel k (columns
// [k0, k1)) is factored, the trailing matrix A(k1:m, k1:m) receives
// -= L(:, k0:k1) L(:, k0:k1)^T, and panel k+1 (columns [k1, k2)) is then
// factored: POTRF of its diagonal tile, and the rows below solved against
// that tile (TRSM).  Launch k does all of this:
//   ticket 0             the diagonal tile of panel k+1: its update, then
//                        POTRF in shared memory; writes L and raises a flag;
//   tickets 1 .. P       32- or 64-row strips of panel k+1 below the diagonal: the
//                        update, then (once the flag is up) the solve
//                        X L_D^T = strip with the new diagonal tile;
//   the other tickets    lower tiles of A(k2:m, k2:m), 64 x 64 or (when those
//                        are too few to fill the device) 32 x 32: the update.
// The strips wait only on ticket 0, which is running whenever they hold a
// ticket, so every wait ends; each wait is also bounded in time (2 s).  The
// diagonal chain of the factorization (tile POTRF, strip solve) thus runs
// beside the bulk of the trailing update instead of between launches.  No
// element is written by one CTA and read by another except the diagonal
// tile, which is read only after its flag.
//
// The chain's length is set by one SM's FP64 pipe: a PW x PW x PW update,
// a PW-column POTRF and a PW-column solve, one after another.  Halving PW
// cuts that chain about four-fold per step for twice the steps, which pays
// while the chain, not the bulk update, bounds a step (small triangles).
#include "rfp_internal.cuh"

namespace rfp {

namespace {

constexpr int kT = 64;              // bulk tile width; the widest panel
// Panel width: 32 for triangles up to kNarrowPanels, 64 beyond.
constexpr int64_t kNarrowPanels = 4096;
// Rows of a panel strip task: 32 for triangles up to kSmallStrips (their
// factorization is bound by the diagonal chain, which shorter strips
// shorten), 64 beyond (fewer, more efficient tasks beside the bulk update).
constexpr int64_t kSmallStrips = 2048;
constexpr int kTh = 256;            // threads per CTA
constexpr int kBk = 16;             // K step of the tile update
constexpr int kSLd = kT + 2;        // staging rows (doubles; 16-byte aligned)
constexpr int kTLd = kT + 1;        // factor / solve tiles
constexpr uint64_t kStepWaitNs = 2000000000ull;

struct StepArgs {
    View<double> V;                 // the m x m lower triangle
    int64_t m, k0, k1, k2;          // panel k = [k0, k1), panel k+1 = [k1, k2)
    int nstrip;                     // strips of panel k+1 in rows [k2, m)
    int bt;                         // bulk tile width (32 or 64)
    int64_t nbulk;                  // lower bt x bt tiles of A(k2:m, k2:m)
    int32_t *info;                  // failure index (1-based, global); also the abort word
    int64_t base;                   // global index of V's first row
    int32_t *sync;                  // [0] ticket counter, [1] diagonal flag (1 ok, 2 failed)
};

struct Smem {
    double As[2][kBk][kSLd];        // staged panel rows of the C tile
    double Bs[2][kBk][kSLd];        // staged panel rows of the C tile's columns
    double T[kT][kTLd];             // updated tile (diagonal / strip)
    double Ld[kT][kTLd];            // new diagonal factor tile (strips)
    double rinv[kT], sq[kT];
    int ticket, flag;
};

__device__ __forceinline__ uint64_t step_globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The block of the C tile a thread owns: TM rows x CW columns at row block
// ry, column block cx.  The usual map is cx = tid % 16, ry = tid / 16 (a
// 16 TM x 16 CW tile); for the 64-wide diagonal tile (`lower`, TM = CW = 4)
// threads 0 .. 135 take the 136 blocks with ry >= cx in order and the others
// own none, so warps 5 .. 7 issue no multiply-adds on the factorization's
// critical path.
template <int TM, int CW>
struct Owner {
    int ry, cx;
    bool active;
    __device__ __forceinline__ Owner(bool lower)
    {
        const int tid = threadIdx.x;
        if (!lower) {
            cx = tid % 16;
            ry = tid / 16;
            active = true;
        } else {
            int r = (int)((sqrtf(8.f * (float)tid + 1.f) - 1.f) * 0.5f);
            while ((r + 1) * (r + 2) / 2 <= tid) ++r;
            while (r * (r + 1) / 2 > tid) --r;
            ry = r;
            cx = tid - r * (r + 1) / 2;
            active = tid < 136;
        }
    }
};

// acc(16 TM x 16 CW: TM x CW per thread) = P_rows(16 TM x w) P_cols(16 CW x w)^T
// with P_rows(i, k) = V(r0 + i, k0 + k) for i < nr (zero beyond), likewise
// P_cols with c0 / nc.  w <= 64.  Register-staged, double-buffered K steps
// of 16 read along V's unit stride.
template <int TM, int CW>
__device__ __forceinline__ void panel_product(const StepArgs &a, Smem &sm, int64_t r0, int nr,
                                              int64_t c0, int nc, int w, const Owner<TM, CW> &o,
                                              double (&acc)[TM][CW])
{
    constexpr int ROWS = 16 * TM, COLS = 16 * CW;
    const int tid = threadIdx.x;
    const bool rowfast = a.V.rs == 1;
    const View<double> Pr = a.V.sub(r0, a.k0), Pc = a.V.sub(c0, a.k0);
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < CW; ++j) acc[i][j] = 0.0;
    double ra[TM], rb[CW];
    // element q of this thread's share of a (R rows x 16 k) block: consecutive
    // threads along V's unit stride
    auto at = [&](int R, int q, int &i, int &k) {
        if (rowfast) { i = tid % R; k = tid / R + (kTh / R) * q; }
        else { k = tid % kBk; i = tid / kBk + 16 * q; }
    };
    auto load = [&](int kb) {
#pragma unroll
        for (int q = 0; q < TM; ++q) {
            int i, k;
            at(ROWS, q, i, k);
            ra[q] = (i < nr && kb + k < w) ? Pr(i, kb + k) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < CW; ++q) {
            int i, k;
            at(COLS, q, i, k);
            rb[q] = (i < nc && kb + k < w) ? Pc(i, kb + k) : 0.0;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < TM; ++q) {
            int i, k;
            at(ROWS, q, i, k);
            sm.As[buf][k][i] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < CW; ++q) {
            int i, k;
            at(COLS, q, i, k);
            sm.Bs[buf][k][i] = rb[q];
        }
    };
    const int nsteps = (w + kBk - 1) / kBk;
    load(0);
    for (int s = 0; s < nsteps; ++s) {
        const int buf = s & 1;
        store(buf);
        __syncthreads();
        if (s + 1 < nsteps) load((s + 1) * kBk);
        if (o.active) {
#pragma unroll
            for (int kk = 0; kk < kBk; ++kk) {
                double av[TM], bv[CW];
#pragma unroll
                for (int i = 0; i < TM; i += 2) {
                    const double2 t2 = *reinterpret_cast<const double2 *>(&sm.As[buf][kk][o.ry * TM + i]);
                    av[i] = t2.x;
                    av[i + 1] = t2.y;
                }
#pragma unroll
                for (int j = 0; j < CW; j += 2) {
                    const double2 t2 = *reinterpret_cast<const double2 *>(&sm.Bs[buf][kk][o.cx * CW + j]);
                    bv[j] = t2.x;
                    bv[j + 1] = t2.y;
                }
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < CW; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
            }
        }
    }
    __syncthreads();   // staging buffers free for the next product
}

// T = V(r0.., c0..) - acc for the owned blocks of the nr x nc tile (lower
// part only when `lower`), into shared memory; entries outside are zero.
template <int TM, int CW>
__device__ __forceinline__ void updated_tile_to_smem(const StepArgs &a, Smem &sm, int64_t r0, int nr,
                                                     int64_t c0, int nc, bool lower,
                                                     const Owner<TM, CW> &o,
                                                     const double (&acc)[TM][CW])
{
    if (!o.active) return;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            const int r = o.ry * TM + i, c = o.cx * CW + j;
            const bool in = r < nr && c < nc && (!lower || c <= r);
            sm.T[r][c] = in ? a.V(r0 + r, c0 + c) - acc[i][j] : 0.0;
        }
}

// Bulk task: lower tile (ti, tj) of A(k2:m, k2:m) in BT x BT tiles (BT = 16 TM)
// receives -= P_rows P_cols^T over panel k.
template <int TM>
__device__ __forceinline__ void bulk_tile(const StepArgs &a, Smem &sm, int64_t ti, int64_t tj)
{
    constexpr int BT = 16 * TM;
    const int64_t r0 = a.k2 + ti * BT, c0 = a.k2 + tj * BT;
    const int nr = (int)(a.m - r0 < BT ? a.m - r0 : BT), nc = (int)(a.m - c0 < BT ? a.m - c0 : BT);
    const Owner<TM, TM> o(false);
    double acc[TM][TM];
    panel_product<TM, TM>(a, sm, r0, nr, c0, nc, (int)(a.k1 - a.k0), o, acc);
    double cin[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) {
            const int r = o.ry * TM + i, c = o.cx * TM + j;
            const bool in = r < nr && c < nc && (ti != tj || c <= r);
            cin[i][j] = in ? a.V(r0 + r, c0 + c) : 0.0;
        }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) {
            const int r = o.ry * TM + i, c = o.cx * TM + j;
            if (r < nr && c < nc && (ti != tj || c <= r)) a.V(r0 + r, c0 + c) = cin[i][j] - acc[i][j];
        }
}

// Element e of a rows x cols block written or read along V's unit stride.
__device__ __forceinline__ void block_elem(const View<double> &V, int e, int rows, int cols, int &i,
                                           int &j)
{
    if (V.rs == 1) { i = e % rows; j = e / rows; }
    else { j = e % cols; i = e / cols; }
}

template <int PW, int STRIP>
__global__ void __launch_bounds__(kTh) potrf_step_kernel(StepArgs a)
{
    static_assert(PW == 32 || PW == 64, "panel width");
    constexpr int CW = PW / 16;       // columns per thread in a panel tile's update
    constexpr int STM = STRIP / 16;   // rows per thread in a strip's update
    extern __shared__ __align__(16) unsigned char step_smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(step_smem_raw);
    if (*a.info != 0) return;   // an earlier panel failed (written before this launch)
    const int tid = threadIdx.x;
    if (tid == 0) sm.ticket = atomicAdd(a.sync, 1);
    __syncthreads();
    const int64_t t = sm.ticket;
    const int w = (int)(a.k1 - a.k0);            // panel k width
    const int wn = (int)(a.k2 - a.k1);           // panel k+1 width
    int32_t *flag = a.sync + 1;

    if (t == 0) {
        // ---- diagonal tile of panel k+1: update (its lower blocks only when
        // 64 wide; a 32-wide tile spreads over all warps), then unblocked
        // Cholesky
        constexpr int DM = PW == 64 ? 4 : 2;
        const Owner<DM, CW> o(PW == 64);
        double acc[DM][CW];
        panel_product<DM, CW>(a, sm, a.k1, wn, a.k1, wn, w, o, acc);
        updated_tile_to_smem<DM, CW>(a, sm, a.k1, wn, a.k1, wn, true, o, acc);
        __syncthreads();
        const int tx = tid % 16, ty = tid / 16;
        int fail = -1;
        for (int j = 0; j < wn; ++j) {
            if (tid == 0) {
                const double d = sm.T[j][j];
                sm.flag = (d > 0.0) ? -1 : j;            // pivot <= 0 or NaN fails
                const double y = rsqrt_newton(d);        // 1 / sqrt(d), a few ulp
                sm.sq[j] = d * y;
                sm.rinv[j] = y;
            }
            __syncthreads();
            if (sm.flag >= 0) { fail = sm.flag; break; }
            const double ri = sm.rinv[j];
            for (int i = j + 1 + tid; i < wn; i += kTh) sm.T[i][j] *= ri;
            __syncthreads();
            for (int i = j + 1 + ty; i < wn; i += 16) {
                const double lij = sm.T[i][j];
                for (int k = j + 1 + tx; k <= i; k += 16) sm.T[i][k] -= lij * sm.T[k][j];
            }
            __syncthreads();
        }
        if (fail >= 0) {
            if (tid == 0) {
                atomicCAS(a.info, 0, (int32_t)(a.base + a.k1 + fail + 1));
                __threadfence();
                atomicExch(flag, 2);
            }
            return;
        }
        for (int e = tid; e < PW * PW; e += kTh) {
            int i, j;
            block_elem(a.V, e, PW, PW, i, j);
            if (i < wn && j <= i) a.V(a.k1 + i, a.k1 + j) = (i == j) ? sm.sq[j] : sm.T[i][j];
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicExch(flag, 1);
        return;
    }

    if (t <= a.nstrip) {
        // ---- a STRIP-row strip of panel k+1: update, wait for the diagonal tile, solve
        const int64_t r0 = a.k2 + (t - 1) * STRIP;
        const int nr = (int)(a.m - r0 < STRIP ? a.m - r0 : STRIP);
        const Owner<STM, CW> o(false);
        double acc[STM][CW];
        panel_product<STM, CW>(a, sm, r0, nr, a.k1, wn, w, o, acc);
        updated_tile_to_smem<STM, CW>(a, sm, r0, nr, a.k1, wn, false, o, acc);
        if (tid == 0) {
            const uint64_t t0 = step_globaltimer();
            int f = 0;
            for (uint32_t it = 0;; ++it) {
                f = *(volatile int32_t *)flag;
                if (f != 0) break;
                __nanosleep(64);
                if ((it & 63) == 63 && step_globaltimer() - t0 > kStepWaitNs) break;
            }
            __threadfence();
            sm.flag = f;
        }
        __syncthreads();
        if (sm.flag != 1) {
            // The diagonal tile failed (info is set) or never came: the strip is
            // left as NaN so that the failure cannot pass unnoticed.
            if (sm.flag == 0)
                for (int e = tid; e < STRIP * PW; e += kTh) {
                    int i, j;
                    block_elem(a.V, e, STRIP, PW, i, j);
                    if (i < nr && j < wn) a.V(r0 + i, a.k1 + j) = __longlong_as_double(0x7ff8000000000000ll);
                }
            return;
        }
        // the new diagonal factor tile, from L2 (another SM wrote it in this
        // launch); unrolled so that each thread's loads are in flight together
#pragma unroll
        for (int q = 0; q < PW * PW / kTh; ++q) {
            int i, j;
            block_elem(a.V, tid + q * kTh, PW, PW, i, j);
            if (i < wn && j <= i) sm.Ld[i][j] = __ldcg(&a.V(a.k1 + i, a.k1 + j));
        }
        __syncthreads();
        if (tid < wn) sm.rinv[tid] = 1.0 / sm.Ld[tid][tid];
        __syncthreads();
        // X L_D^T = T, columns in increasing order; rows are independent.
        // G = 256 / STRIP consecutive lanes share a row, lane g holding its
        // columns g + G i in registers: column j is scaled by its owner lane
        // and handed to the row's other lanes by a shuffle, so the solve takes
        // no block barrier, and registers whose columns are all finished drop
        // out of the step at compile time.
        {
            constexpr int G = kTh / STRIP, NC = PW / G;
            const int row = tid / G, grp = tid % G;
            double x[NC];
#pragma unroll
            for (int i = 0; i < NC; ++i) x[i] = sm.T[row][grp + G * i];
#pragma unroll
            for (int j = 0; j < PW; ++j) {
                if (j < wn) {   // uniform
                    const int oi = j / G, og = j % G;
                    const double xj = __shfl_sync(0xffffffffu, x[oi] * sm.rinv[j], og, G);
                    if (grp == og) x[oi] = xj;
#pragma unroll
                    for (int i = 0; i < NC; ++i) {
                        if (i < oi) continue;
                        const int c = grp + G * i;
                        if (c > j && c < wn) x[i] = fma(-sm.Ld[c][j], xj, x[i]);
                    }
                }
            }
            __syncthreads();   // every thread has read its row of T
#pragma unroll
            for (int i = 0; i < NC; ++i) sm.T[row][grp + G * i] = x[i];
            __syncthreads();
        }
        for (int e = tid; e < STRIP * PW; e += kTh) {
            int i, j;
            block_elem(a.V, e, STRIP, PW, i, j);
            if (i < nr && j < wn) a.V(r0 + i, a.k1 + j) = sm.T[i][j];
        }
        return;
    }

    // ---- a lower bt x bt tile of A(k2:m, k2:m): the update only
    const int64_t b = t - 1 - a.nstrip;
    // single-precision guess (the FP64 pipe is narrow), corrected below
    int64_t ti = (int64_t)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= b) ++ti;
    while (ti * (ti + 1) / 2 > b) --ti;
    const int64_t tj = b - ti * (ti + 1) / 2;
    if (a.bt == 32) bulk_tile<2>(a, sm, ti, tj);
    else bulk_tile<4>(a, sm, ti, tj);
}

}  // namespace

int potrf_step_width(int64_t m)
{
    return m <= kNarrowPanels ? 32 : kT;
}

size_t potrf_step_sync_words(int64_t m)
{
    const int64_t pw = potrf_step_width(m), np = (m + pw - 1) / pw;
    return (size_t)(2 * (np > 1 ? np - 1 : 1));
}

template <int PW, int STRIP>
static cudaError_t launch_step(cudaStream_t st, const StepArgs &a, int64_t grid)
{
    const int smem = (int)sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(potrf_step_kernel<PW, STRIP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    potrf_step_kernel<PW, STRIP><<<(unsigned)grid, kTh, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t potrf_step(cudaStream_t st, View<double> V, int64_t m, int64_t k0, int32_t *info,
                       int64_t base, int32_t *sync)
{
    const int64_t pw = potrf_step_width(m);
    const int64_t k1 = k0 + pw < m ? k0 + pw : m;
    if (k1 >= m) return cudaSuccess;                  // no next panel
    const int64_t k2 = k1 + pw < m ? k1 + pw : m;
    const int64_t strip = m <= kSmallStrips ? 32 : 64;
    const int64_t strips = (m - k2 + strip - 1) / strip;
    const int bt = potrf_step_bulk_tile(m - k2, 2 * (int64_t)device_sm_count());   // 2 CTAs per SM
    const int64_t rest = (m - k2 + bt - 1) / bt;      // row tiles of A(k2:m, k2:m)
    StepArgs a{V, m, k0, k1, k2, (int)strips, bt, rest * (rest + 1) / 2, info, base, sync};
    const int64_t grid = 1 + a.nstrip + a.nbulk;
    if (grid > INT32_MAX) return cudaErrorInvalidValue;
    if (pw == 32) return strip == 32 ? launch_step<32, 32>(st, a, grid) : launch_step<32, 64>(st, a, grid);
    return strip == 32 ? launch_step<64, 32>(st, a, grid) : launch_step<64, 64>(st, a, grid);
}

}  // namespace rfp
