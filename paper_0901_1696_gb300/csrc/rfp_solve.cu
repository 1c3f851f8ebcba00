// One-launch FP64 triangular solves with the whole RFP factor (PFTRS).
//
// Section 4 solves A X = B with the factor L = [L11 0; L21 L22] held in the
// RFP array's three blocks, as three steps each way (Fig. 4, "solve"):
//   forward:  L11 Y1 = B1;  B2 -= L21 Y1;  L22 Y2 = B2
//   backward: L22^T X2 = Y2;  Y1 -= L21^T X2;  L11^T X1 = Y1.
// Both directions are block substitutions on the n x n lower triangle L,
// whose R-row blocks are cut separately in T1 (rows [0, n1)) and T2 (rows
// [n1, n)), so every block of L lies inside one of T1, S or T2:
//   forward, block row b:   X_b = L_bb^{-1} (B_b - sum_{j<b} L_bj X_j)
//   backward, block row b:  X_b = L_bb^{-T} (Y_b - sum_{j>b} L_jb^T X_j).
// One launch per direction computes all of it.  A task is (block row b,
// group g of G right-hand-side columns, G = 8 or 16).  Tasks take tickets from a device
// counter in solve order (block rows in solve order, then column groups).
// For each group, blocks complete in solve order (block b needs every
// earlier one), so one progress word per group says how many of its blocks
// are final; a task reads X_j only once that count has passed j.  A CTA
// waits only on lower tickets, held by CTAs that are already running and
// that wait only on lower tickets in turn, so every wait ends.  Each wait is
// also bounded in time: on expiry the CTA raises the error word, every task
// that sees it gives up, and each task that gives up writes NaN into its own
// block of X, so an incomplete solve cannot pass for a result.
//
// Per task: 128 threads, each owning R/16 rows x 2 columns of the R x 16
// block in registers (R = 32 or 64 rows).  Blocks of L are streamed through
// shared memory in R x 16 chunks (register-staged, double-buffered); X_j is
// read from L2 (ld.global.cg: other SMs wrote it during this launch).  The
// diagonal block is then solved by substitution, one warp per 4 columns,
// each lane holding one column of R/8 rows, the solved values handed out by
// shuffles.
#include <cmath>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "rfp_internal.cuh"

namespace rfp {

namespace {

// Right-hand sides per task (G): 16, or 8 when there are at most 16 of them
// (two chains of half the work each instead of one).
constexpr int kKc = 16;             // K chunk staged in shared memory
constexpr int kThreads = 128;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kErrWait = 4;
// Block rows: 64 for large orders (fewer, larger tasks), 32 up to
// kSmallSolve rows, where the diagonal chain bounds the solve: on GB300 a
// 64-row block's update and substitution keep one SM's FP64 pipe busy about
// four times longer than a 32-row block's.
constexpr int64_t kSmallSolve = 4096;

struct SolveArgs {
    View<double> t1, s, t2;
    int64_t n1, n2;
    int nb1, nb;                    // row blocks in T1, in total
    View<double> X;                 // n x nrhs, any strides
    int64_t nrhs;
    int ng;
    int32_t *counter, *prog, *err;
    const int32_t *abort;           // if set (non-zero) at launch, nothing is done
    double alpha;                   // the right-hand side is alpha X
    int lower_rhs;                  // X lower triangular (forward, one triangle): see rfp_solve
};

__device__ __forceinline__ uint64_t rs_globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// First row (global) and row count of block b (R-row blocks).
template <int R>
__device__ __forceinline__ void block_rows(const SolveArgs &a, int b, int64_t &r0, int &rows)
{
    if (b < a.nb1) {
        r0 = (int64_t)b * R;
        rows = (int)(a.n1 - r0 < R ? a.n1 - r0 : R);
    } else {
        const int64_t lr = (int64_t)(b - a.nb1) * R;
        r0 = a.n1 + lr;
        rows = (int)(a.n2 - lr < R ? a.n2 - lr : R);
    }
}

// View of block (bi, bj) of L, bi >= bj, at the block's first element.
template <int R>
__device__ __forceinline__ View<double> lblock(const SolveArgs &a, int bi, int bj)
{
    const int64_t ri = bi < a.nb1 ? (int64_t)bi * R : (int64_t)(bi - a.nb1) * R;
    const int64_t cj = bj < a.nb1 ? (int64_t)bj * R : (int64_t)(bj - a.nb1) * R;
    if (bi < a.nb1) return a.t1.sub(ri, cj);
    if (bj < a.nb1) return a.s.sub(ri, cj);
    return a.t2.sub(ri, cj);
}

// Thread 0 waits until *prog >= need; false if the error word is (or becomes) set.
__device__ __forceinline__ bool wait_progress(const int32_t *prog, int need, int32_t *err)
{
    const uint64_t t0 = rs_globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (*(volatile const int32_t *)prog >= need) return true;
        if (*(volatile int32_t *)err != 0) return false;
        __nanosleep(32);
        if ((it & 63) == 63 && rs_globaltimer() - t0 > kWaitNs) {
            atomicCAS(err, 0, kErrWait);
            return false;
        }
    }
}

// Staging of one R x 16 chunk of op(L_jb) (rows r < rv of the task's block,
// k in [k0, k0 + 16) < kv) and of the matching 16 x G chunk of X_j.
// A(r, k) = V(r, k) for a view V; both loaders read along their view's unit
// stride (X's rows for a right-hand-side block, its columns for a
// transposed RFP block).
template <int R, int G>
struct ChunkRegs {
    static constexpr int AQ = R * kKc / kThreads, ALd = R + 2, XQ = kKc * G / kThreads, XLd = G + 2;
    double a[AQ];
    double x[XQ];

    __device__ __forceinline__ void load(View<double> V, int rv, int k0, int kv, View<double> Xj,
                                         int cols)
    {
        const int tid = threadIdx.x;
        if (V.rs == 1) {      // rows contiguous
#pragma unroll
            for (int q = 0; q < AQ; ++q) {
                const int r = tid % R, k = k0 + tid / R + (kThreads / R) * q;
                a[q] = (r < rv && k < kv) ? __ldg(&V.p[r + (int64_t)k * V.cs]) : 0.0;
            }
        } else {              // k contiguous
#pragma unroll
            for (int q = 0; q < AQ; ++q) {
                const int k = k0 + tid % kKc, r = tid / kKc + 8 * q;
                a[q] = (r < rv && k < kv) ? __ldg(&V.p[(int64_t)r * V.rs + k * V.cs]) : 0.0;
            }
        }
        if (Xj.rs == 1) {     // X rows contiguous
#pragma unroll
            for (int q = 0; q < XQ; ++q) {
                const int k = k0 + tid % kKc, c = tid / kKc + (kThreads / kKc) * q;
                x[q] = (k < kv && c < cols) ? __ldcg(&Xj(k, c)) : 0.0;
            }
        } else {              // X columns contiguous
#pragma unroll
            for (int q = 0; q < XQ; ++q) {
                const int c = tid % G, k = k0 + tid / G + (kThreads / G) * q;
                x[q] = (k < kv && c < cols) ? __ldcg(&Xj(k, c)) : 0.0;
            }
        }
    }
    __device__ __forceinline__ void store(const View<double> &V, bool xrowfast, double (*As)[ALd],
                                          double (*Xs)[XLd]) const
    {
        const int tid = threadIdx.x;
        if (V.rs == 1) {
#pragma unroll
            for (int q = 0; q < AQ; ++q) As[tid / R + (kThreads / R) * q][tid % R] = a[q];
        } else {
#pragma unroll
            for (int q = 0; q < AQ; ++q) As[tid % kKc][tid / kKc + 8 * q] = a[q];
        }
        if (xrowfast) {
#pragma unroll
            for (int q = 0; q < XQ; ++q) Xs[tid % kKc][tid / kKc + (kThreads / kKc) * q] = x[q];
        } else {
#pragma unroll
            for (int q = 0; q < XQ; ++q) Xs[tid / G + (kThreads / G) * q][tid % G] = x[q];
        }
    }
};

template <int R, int G>
struct UpdateSmem {
    double As[2][kKc][R + 2];
    double Xs[2][kKc][G + 2];
};
template <int R, int G>
struct DiagSmem {
    double Ld[R][R + 1];        // lower triangle of L_bb
    double Bs[R][G + 1];        // the block's right-hand side, redistributed
    double rinv[R];             // 1 / L_bb(j, j)
};
// 64-row blocks share one region between the update's staging and the
// diagonal block; 32-row blocks keep both (26 KB), so that the diagonal
// block is loaded before the task's first wait, off the critical path.
template <int R, int G>
union SolveSmemShared {
    UpdateSmem<R, G> u;
    DiagSmem<R, G> d;
};
template <int R, int G>
struct SolveSmemSplit {
    UpdateSmem<R, G> u;
    DiagSmem<R, G> d;
};
template <int R, int G>
using SolveSmem = std::conditional_t<R == 32, SolveSmemSplit<R, G>, SolveSmemShared<R, G>>;

template <bool TRANS, int R, int G>
__global__ void __launch_bounds__(kThreads) rfp_solve_kernel(SolveArgs a)
{
    constexpr int CP = G / 2;                 // column pairs of the update
    constexpr int RM = R * CP / kThreads;     // rows per thread in the update
    static_assert(RM >= 1 && R * CP == RM * kThreads, "update layout");
    __shared__ __align__(16) SolveSmem<R, G> sm;
    __shared__ int s_ticket, s_ok;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // The abort word is written before this launch and not during it, so
    // every CTA sees the same value and none is left waiting.
    if (a.abort && *a.abort) return;
    if (tid == 0) s_ticket = atomicAdd(a.counter, 1);
    __syncthreads();
    const int ticket = s_ticket;
    const int g = ticket % a.ng, p = ticket / a.ng;          // p: position in solve order
    const int b = TRANS ? a.nb - 1 - p : p;
    const int64_t c0 = (int64_t)g * G;
    // A lower-triangular right-hand side (forward): the group's columns are
    // zero above row c0 in B and in the solution, so blocks above c0's block
    // are left as they are, publish nothing, and are not read below.
    const int jf = a.lower_rhs ? (int)(c0 / R) : 0;
    if (b < jf) return;
    int64_t r0;
    int rows;
    block_rows<R>(a, b, r0, rows);
    const int cols = (int)(a.nrhs - c0 < G ? a.nrhs - c0 : G);
    const View<double> Xb = a.X.sub(r0, c0);
    int32_t *prog = a.prog + g;

    const int tx = tid % CP, ty = tid / CP;                  // 2 columns x RM rows each
    double acc[RM][2];
#pragma unroll
    for (int m = 0; m < RM; ++m)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int r = ty * RM + m, cc = tx * 2 + c;
            acc[m][c] = (r < rows && cc < cols) ? a.alpha * __ldcg(&Xb(r, cc)) : 0.0;
        }

    // The lower triangle of L_bb and the reciprocals of its pivots into
    // shared memory.
    auto load_diag = [&]() {
        const View<double> D = lblock<R>(a, b, b);
        const bool rowfast = D.rs == 1;
        // unrolled by 8: eight loads per thread in flight at a time
#pragma unroll 8
        for (int q = 0; q < R * R / kThreads; ++q) {
            const int e = tid + q * kThreads, u = e % R, v = e / R;
            const int i = rowfast ? u : v, jj = rowfast ? v : u;
            if (i < rows && jj <= i) sm.d.Ld[i][jj] = D(i, jj);
        }
        // Reciprocals of the pivots, formed once in parallel: on GB300's
        // narrow FP64 pipe a division per lane per step would cost more
        // than the substitution's multiply-adds.
        if (tid < rows) sm.d.rinv[tid] = 1.0 / D(tid, tid);
    };
    constexpr bool kEarlyDiag = R == 32;
    if (kEarlyDiag) load_diag();   // ordered before its use by the barriers below

    bool ok = true;
    // Off-diagonal blocks in solve order: forward j = jf .. b-1, backward j = nb-1 .. b+1.
    const int nblk = p;
    for (int q = jf; q < nblk && ok; ++q) {
        const int j = TRANS ? a.nb - 1 - q : q;
        if (tid == 0) {
            s_ok = wait_progress(prog, q + 1, a.err) ? 1 : 0;
            __threadfence();
        }
        __syncthreads();
        if (!s_ok) {
            ok = false;
            break;
        }
        int64_t j0;
        int kv;
        block_rows<R>(a, j, j0, kv);
        // op(L) for this task: forward A = L_bj (rows b, k over j);
        // backward A = L_jb^T (rows b, k over j).
        const View<double> V = TRANS ? lblock<R>(a, j, b).t() : lblock<R>(a, b, j);
        const View<double> Xj = a.X.sub(j0, c0);
        const int nch = (kv + kKc - 1) / kKc;
        ChunkRegs<R, G> st;
        st.load(V, rows, 0, kv, Xj, cols);
        for (int ch = 0; ch < nch; ++ch) {
            const int buf = ch & 1;
            st.store(V, Xj.rs == 1, sm.u.As[buf], sm.u.Xs[buf]);
            __syncthreads();
            if (ch + 1 < nch) st.load(V, rows, (ch + 1) * kKc, kv, Xj, cols);
#pragma unroll
            for (int kk = 0; kk < kKc; ++kk) {
                double av[RM];
                if constexpr (RM % 2 == 0) {
#pragma unroll
                    for (int m = 0; m < RM; m += 2) {
                        const double2 t2 = *reinterpret_cast<const double2 *>(&sm.u.As[buf][kk][ty * RM + m]);
                        av[m] = t2.x;
                        av[m + 1] = t2.y;
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < RM; ++m) av[m] = sm.u.As[buf][kk][ty * RM + m];
                }
                const double2 x = *reinterpret_cast<const double2 *>(&sm.u.Xs[buf][kk][tx * 2]);
#pragma unroll
                for (int m = 0; m < RM; ++m) {
                    acc[m][0] = fma(-av[m], x.x, acc[m][0]);
                    acc[m][1] = fma(-av[m], x.y, acc[m][1]);
                }
            }
            // the next store overwrites the other buffer, last read two chunks ago
        }
        __syncthreads();   // all reads of this block's buffers done before the next block
    }

    if (!ok) {             // a wait gave up: mark this block of X as not computed
#pragma unroll
        for (int m = 0; m < RM; ++m)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int r = ty * RM + m, cc = tx * 2 + c;
                if (r < rows && cc < cols) Xb(r, cc) = __longlong_as_double(0x7ff8000000000000ll);
            }
        return;
    }

    // Diagonal block (64-row blocks: loaded now, into the staging region),
    // the right-hand side from the accumulators, then substitution.
    if (!kEarlyDiag) load_diag();
#pragma unroll
    for (int m = 0; m < RM; ++m)
#pragma unroll
        for (int c = 0; c < 2; ++c) sm.d.Bs[ty * RM + m][tx * 2 + c] = acc[m][c];
    __syncthreads();

    // Substitution.  Warp w takes columns CW w .. CW w + CW - 1 (CW = G / 4);
    // lane (lr, lc) = (lane / CW, lane % CW) holds column CW w + lc of rows
    // lr + RG k, k < R / RG (RG = 32 / CW row groups).  Step j: the CW lanes
    // holding row j scale it by the pivot's reciprocal (one instruction for
    // the warp's columns), a shuffle hands each lane its column's x_j, and
    // every lane removes x_j from its later (forward) or earlier (backward)
    // rows; registers whose rows are all finished drop out of the step at
    // compile time.  On GB300's FP64 pipe, where a warp instruction costs
    // the same whatever its active lanes, this is about 3.5 instructions a
    // step for 32-row blocks of 16 columns (2.5 for 8) against 8 with one
    // lane per row.
    constexpr int CW = G / 4, RG = 32 / CW, K = R / RG;
    const int lr = lane / CW, lc = lane % CW, col = warp * CW + lc;
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = sm.d.Bs[lr + RG * k][col];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int j = TRANS ? R - 1 - q : q;
        if (j < rows) {    // uniform
            const int kj = j / RG, oj = j % RG;
            const double xj = __shfl_sync(0xffffffffu, v[kj] * sm.d.rinv[j], oj * CW + lc);
            if (lr == oj) v[kj] = xj;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (TRANS ? k > kj : k < kj) continue;
                const int r = lr + RG * k;
                if (TRANS ? r < j : (r > j && r < rows)) {
                    const double l = TRANS ? sm.d.Ld[j][r] : sm.d.Ld[r][j];
                    v[k] = fma(-l, xj, v[k]);
                }
            }
        }
    }
    // out through shared memory, along X's unit stride
    __syncthreads();   // every lane is done reading Bs
#pragma unroll
    for (int k = 0; k < K; ++k) sm.d.Bs[lr + RG * k][col] = v[k];
    __syncthreads();
    if (Xb.rs == 1) {      // X's rows contiguous
#pragma unroll
        for (int q = 0; q < R * G / kThreads; ++q) {
            const int r = tid % R, cc = tid / R + (kThreads / R) * q;
            if (r < rows && cc < cols) Xb(r, cc) = sm.d.Bs[r][cc];
        }
    } else {               // X's columns contiguous
#pragma unroll
        for (int q = 0; q < R * G / kThreads; ++q) {
            const int cc = tid % G, r = tid / G + (kThreads / G) * q;
            if (r < rows && cc < cols) Xb(r, cc) = sm.d.Bs[r][cc];
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicExch(prog, p + 1);
}

}  // namespace

// Dynamic shared memory that leaves room for one CTA of `fn` per SM (0 if
// the device attributes cannot be read or set), cached per device and kernel.
// A wide solve of a small triangle (many column groups, little work each)
// is bound by its diagonal chain; with several resident tasks per SM the
// tasks on that chain share their SM's FP64 pipe with tasks that are only
// accumulating earlier blocks.  One per SM: n = 1001's 500-column solves
// went from about 316 to 254 us (two per SM: 266 us).
static int one_cta_per_sm_smem(const void *fn)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find({dev, fn});
        if (it != cache.end()) return it->second;
    }
    int dyn = 0, per_sm = 0, per_block = 0;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess &&
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess) {
        dyn = per_sm / 2 + 1 - (int)fa.sharedSizeBytes;   // two such CTAs exceed the SM
        if (dyn < 0 || dyn + (int)fa.sharedSizeBytes > per_block ||
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
            dyn = 0;
    }
    (void)cudaGetLastError();   // a failed query is not the caller's error
    std::lock_guard<std::mutex> lock(mu);
    cache[{dev, fn}] = dyn;
    return dyn;
}

// Right-hand sides per task: 8 when there are at most 16 (two chains, each
// with half the update per block and a shorter substitution), else 16.
static int64_t group_width(int64_t nrhs) { return nrhs <= 16 ? 8 : 16; }

size_t rfp_solve_sync_words(int64_t nrhs)
{
    const int64_t G = group_width(nrhs);
    return (size_t)(2 + (nrhs + G - 1) / G);
}

cudaError_t rfp_solve(cudaStream_t st, View<double> t1, View<double> s, View<double> t2, int64_t n1,
                      int64_t n2, View<double> X, int64_t nrhs, bool trans, int32_t *sync,
                      const int32_t *abort, double alpha, bool lower_rhs)
{
    const int64_t n = n1 + n2;
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    if (lower_rhs && (trans || n2 != 0)) return cudaErrorInvalidValue;
    const int64_t R = n <= kSmallSolve ? 32 : 64;
    const int64_t G = group_width(nrhs);
    const int64_t nb1 = (n1 + R - 1) / R, nb2 = (n2 + R - 1) / R, ng = (nrhs + G - 1) / G;
    const int64_t tasks = (nb1 + nb2) * ng;
    if (tasks > INT32_MAX) return cudaErrorInvalidValue;
    // sync: [0] ticket counter, [1] error word, [2 .. 2 + ng) progress per
    // column group; all start at zero.
    cudaError_t e = cudaMemsetAsync(sync, 0, rfp_solve_sync_words(nrhs) * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    SolveArgs a{t1, s, t2, n1, n2, (int)nb1, (int)(nb1 + nb2), X, nrhs, (int)ng,
                sync, sync + 2, sync + 1, abort, alpha, lower_rhs ? 1 : 0};
    const unsigned grid = (unsigned)tasks;
    if (R == 32 && G == 8) {
        if (trans) rfp_solve_kernel<true, 32, 8><<<grid, kThreads, 0, st>>>(a);
        else rfp_solve_kernel<false, 32, 8><<<grid, kThreads, 0, st>>>(a);
    } else if (R == 32) {
        // wide and small: one task per SM (see one_cta_per_sm_smem)
        const bool cap = ng >= 8 && n * nrhs <= (int64_t(1) << 19);
        const void *fn = trans ? (const void *)rfp_solve_kernel<true, 32, 16>
                               : (const void *)rfp_solve_kernel<false, 32, 16>;
        const int dyn = cap ? one_cta_per_sm_smem(fn) : 0;
        if (trans) rfp_solve_kernel<true, 32, 16><<<grid, kThreads, dyn, st>>>(a);
        else rfp_solve_kernel<false, 32, 16><<<grid, kThreads, dyn, st>>>(a);
    } else if (G == 8) {
        if (trans) rfp_solve_kernel<true, 64, 8><<<grid, kThreads, 0, st>>>(a);
        else rfp_solve_kernel<false, 64, 8><<<grid, kThreads, 0, st>>>(a);
    } else {
        if (trans) rfp_solve_kernel<true, 64, 16><<<grid, kThreads, 0, st>>>(a);
        else rfp_solve_kernel<false, 64, 16><<<grid, kThreads, 0, st>>>(a);
    }
    note_launch();
    return cudaGetLastError();
}

// ---- stream-ordered scratch for the sync words ------------------------------
//
// A library-private memory pool per device (created on first use, never
// destroyed) from which each solve takes its few sync words with
// cudaMallocFromPoolAsync and returns them with cudaFreeAsync on the same
// stream, so concurrent solves on different streams never share them.  The
// pool keeps up to 128 MiB between calls instead of returning it to the
// driver (PFTRI of a small triangle takes up to 9 m^2 doubles, m <= 1024).
// Under stream capture the caller does not use it (it runs the multi-launch
// form instead).

namespace {
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[64] = {};
}  // namespace

cudaError_t solve_scratch_acquire(cudaStream_t st, size_t words, int32_t **out)
{
    *out = nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return e;
    if (cap != cudaStreamCaptureStatusNone) return cudaErrorNotSupported;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorNotSupported;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mutex);
        if (!g_pool[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t p;
            e = cudaMemPoolCreate(&p, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = 128ull << 20;
            e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(p);
                return e;
            }
            g_pool[dev] = p;
        }
        pool = g_pool[dev];
    }
    void *ptr = nullptr;
    e = cudaMallocFromPoolAsync(&ptr, words * sizeof(int32_t), pool, st);
    if (e != cudaSuccess) return e;
    *out = static_cast<int32_t *>(ptr);
    return cudaSuccess;
}

cudaError_t solve_scratch_release(cudaStream_t st, int32_t *p)
{
    return p ? cudaFreeAsync(p, st) : cudaSuccess;
}

}  // namespace rfp
