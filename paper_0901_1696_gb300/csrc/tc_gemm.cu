// Tensor-core (tcgen05) low-precision GEMM update for the mixed-precision
// factorization: C (FP32, strided view) = alpha * A * B^T + beta * C, with A
// (M x K) and B (N x K) stored K-contiguous in BF16 (kind::f16) or FP32 read
// as TF32 (kind::tf32), accumulated in FP32 in tensor memory.
//
// This is the SYRK / GEMM of the paper's step 3 (Fig. 4, T2 <- T2 - S S^T)
// and of the trailing updates inside the Cholesky of a triangle, run on the
// 5th-generation tensor cores.  The kernel is persistent: one CTA per SM
// walks the list of 128 x 128 output tiles (lower-triangular tiles only for
// a SYRK), tiles b, b + grid, b + 2 grid, ...
//   * warp 4 issues TMA loads (cp.async.bulk.tensor.2d, 128-byte swizzle) of
//     128-byte K slices of A and B into a 4-stage shared-memory ring that
//     runs on across tile boundaries,
//   * warp 5 (one thread) issues tcgen05.mma (K = 32 bytes per instruction)
//     into one of two TMEM accumulators (2 x 128 FP32 columns), alternating
//     between consecutive tiles, and tcgen05.commit to release each stage
//     and to hand each finished accumulator to the epilogue,
//   * warps 0-3 read an accumulator with tcgen05.ld (one TMEM lane per
//     thread = one C row), hand it back, and apply the masked epilogue to C;
//     meanwhile the MMAs of the next tile fill the other accumulator.  When
//     the C view allows it, the C tile is staged in shared memory by TMA in
//     two halves of 64 columns (two 128 x 32 FP32 boxes each); half h of the
//     next tile is loaded as soon as half h of the current one has been read,
//     so the epilogue does not wait on scattered C loads.
// Every mbarrier wait is bounded by time; on expiry the kernel records an
// error code in *err and every role stops issuing work; the producer then
// waits (bounded) for its copies in flight, the MMA issuer for its MMAs, and
// the CTA frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "rfp_internal.cuh"

namespace rfp {

namespace tc {

constexpr int kBM = 128, kBN = 128, kStages = 4;
constexpr int kRowBytes = 128;                    // one K slice per row (swizzle span)
constexpr int kTileBytes = kBM * kRowBytes;       // 16 KB per operand per stage
constexpr int kThreads = 192;                     // 4 epilogue warps + TMA warp + MMA warp
constexpr uint64_t kWaitNs = 2000000000ull;       // 2 s bound on any single wait
constexpr int kCBox = 32;                         // C columns per TMA box (128 rows x 32 FP32 = 16 KB)
constexpr int kCBytes = kBM * kBN * 4;            // one C tile staged in shared memory (64 KB)
constexpr int kSmemBytes = 1024 /*align*/ + 2 * kStages * kTileBytes + kCBytes + 256;   // + barriers, TMEM slot

struct Args {
    float *C;
    int64_t crs, ccs;       // C element (i, j) at C[i*crs + j*ccs]
    int64_t M, N, K;        // K in elements
    int a_row0, b_row0;     // first row of A / B inside their tensor maps
    float alpha, beta;
    int cmode;              // MASK_LOWER: write only i >= j (C-local)
    int tiles_n;            // column tiles
    int lower_tiles;        // 1: the tile list is the lower-triangular tile set
    int64_t num_tiles;      // tiles in the list
    int c_tma;              // 1: C tiles are staged in shared memory by TMA (tmC)
    int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on phase `parity` of an mbarrier; false (and *err set) on
// expiry or when another role already failed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, int code)
{
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255) {
            if (*(volatile int *)err != 0) return false;
            if (globaltimer() - t0 > kWaitNs) {
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}

// Wait bounded by time only (not by the error word): used to let work
// already issued finish before the CTA tears down.
__device__ __forceinline__ bool mbar_wait_quiet(uint64_t *bar, uint32_t parity)
{
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && globaltimer() - t0 > kWaitNs) return false;
    }
}

// AND of `p` over the 128 threads of the four epilogue warps (named
// barrier 1); every one of them must reach it.
__device__ __forceinline__ bool epilogue_all(bool p)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.and.pred po, 1, 128, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
    d |= (uint64_t)(16u >> 4) << 16;                   // leading byte offset (unused, SW128 K-major)
    d |= (uint64_t)(1024u >> 4) << 32;                 // stride byte offset: 8-row group pitch
    d |= (uint64_t)1 << 46;                            // fixed field 0b001
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format, both K-major, N, M.
template <int KIND>
__host__ __device__ constexpr uint32_t instr_desc()
{
    return (1u << 4)                                    // D = F32
           | ((KIND == 0 ? 1u : 2u) << 7)               // A = BF16 (f16 kind) / TF32
           | ((KIND == 0 ? 1u : 2u) << 10)              // B = BF16 / TF32
           | ((uint32_t)(kBN >> 3) << 17)               // N / 8
           | ((uint32_t)(kBM >> 4) << 24);              // M / 16
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                    uint32_t accumulate)
{
    constexpr uint32_t idesc = instr_desc<KIND>();
    if (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Tile t of the launch's tile list: (row tile, column tile).
__device__ __forceinline__ void tile_coords(const Args &a, int64_t t, int64_t &tm, int64_t &tn)
{
    if (a.lower_tiles) {   // row-major lower-triangular tile list
        // single-precision guess (the FP64 pipe is narrow), corrected below
        int64_t r = (int64_t)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
        while ((r + 1) * (r + 2) / 2 <= t) ++r;
        while (r * (r + 1) / 2 > t) --r;
        tm = r;
        tn = t - r * (r + 1) / 2;
    } else {
        tm = t / a.tiles_n;
        tn = t % a.tiles_n;
    }
}

// Persistent: CTA b computes tiles b, b + gridDim.x, ... of the tile list.
// Two accumulators of kBN TMEM columns alternate between consecutive tiles
// of a CTA, so the epilogue of one tile overlaps the loads and MMAs of the
// next; the shared-memory ring runs on across tile boundaries.
template <int KIND>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, Args a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sB = base + kStages * kTileBytes;
    float *sC = reinterpret_cast<float *>(sB + kStages * kTileBytes);   // [kBN][kBM], rows fastest
    uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(sC) + kCBytes);
    uint64_t *empty = full + kStages;
    uint64_t *accf = empty + kStages;     // [2] accumulator ready (MMA commit)
    uint64_t *acce = accf + 2;            // [2] accumulator drained (4 epilogue warps)
    uint64_t *drain = acce + 2;           // every MMA of this CTA completed
    uint64_t *cfull = drain + 1;          // [2] a staged half of the C tile has landed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(cfull + 2);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int bk = kRowBytes / (KIND == 0 ? 2 : 4);                 // K elements per stage
    const int nk = (int)((a.K + bk - 1) / bk);

    if (warp == 0) {   // one warp allocates both accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(2 * kBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(drain, 1);
        mbar_init(&cfull[0], 1);
        mbar_init(&cfull[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t ntiles = a.num_tiles;

    if (warp == 4 && lane == 0) {
        // ---- TMA producer: stage it of the ring holds K slice kt of a tile
        int64_t it = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            int64_t tm, tn;
            tile_coords(a, t, tm, tn);
            for (int kt = 0; kt < nk; ++kt, ++it) {
                const int s = (int)(it % kStages);
                const int64_t r = it / kStages;
                if (r > 0 && !mbar_wait(&empty[s], (uint32_t)((r - 1) & 1), a.err, 1)) { ok = false; break; }
                mbar_expect_tx(&full[s], 2 * kTileBytes);
                tma_load_2d(sA + s * kTileBytes, &tmA, &full[s], kt * bk, a.a_row0 + (int)(tm * kBM));
                tma_load_2d(sB + s * kTileBytes, &tmB, &full[s], kt * bk, a.b_row0 + (int)(tn * kBN));
            }
        }
        // On failure, let the copies still in flight land before the CTA exits
        // (the last kStages stages issued, each waited on its own phase).
        if (!ok)
            for (int64_t q = (it > kStages ? it - kStages : 0); q < it; ++q)
                mbar_wait_quiet(&full[q % kStages], (uint32_t)((q / kStages) & 1));
    } else if (warp == 5 && lane == 0) {
        // ---- MMA issuer
        int64_t it = 0, lt = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
            const int buf = (int)(lt & 1);
            const int64_t u = lt >> 1;
            if (u > 0 && !mbar_wait(&acce[buf], (uint32_t)((u - 1) & 1), a.err, 2)) { ok = false; break; }
            fence_after();
            const uint32_t acc = tmem + (uint32_t)(buf * kBN);
            for (int kt = 0; kt < nk; ++kt, ++it) {
                const int s = (int)(it % kStages);
                if (!mbar_wait(&full[s], (uint32_t)((it / kStages) & 1), a.err, 2)) { ok = false; break; }
                fence_after();
                const uint32_t a0 = smem_u32(sA + s * kTileBytes), b0 = smem_u32(sB + s * kTileBytes);
#pragma unroll
                for (int kk = 0; kk < kRowBytes / 32; ++kk)
                    mma<KIND>(acc, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32),
                              (kt | kk) != 0 ? 1u : 0u);
                mma_commit(&empty[s]);
            }
            if (ok) mma_commit(&accf[buf]);
        }
        // Every MMA issued above completes before the CTA tears down.
        mma_commit(drain);
        mbar_wait_quiet(drain, 0);
    } else if (warp < 4) {
        // ---- epilogue: lane = row of the tile.  With c_tma, the C tile is
        // staged in shared memory in two halves of 64 columns; thread 0 loads
        // half h of the CTA's next tile by TMA as soon as every epilogue
        // thread has read half h of the current one, so each load overlaps
        // the processing of the other half.
        const int etid = threadIdx.x;   // 0 .. 127
        int64_t lt = 0, issued0 = 0, issued1 = 0;   // C-half loads issued (thread 0)
        auto issue_half = [&](int64_t t, int h) {
            int64_t tm, tn;
            tile_coords(a, t, tm, tn);
            mbar_expect_tx(&cfull[h], kCBytes / 2);
#pragma unroll
            for (int b = 2 * h; b < 2 * h + 2; ++b)
                tma_load_2d(sC + b * kCBox * kBM, &tmC, &cfull[h], (int)(tm * kBM), (int)(tn * kBN) + b * kCBox);
            if (h) ++issued1;
            else ++issued0;
        };
        if (a.c_tma && etid == 0 && blockIdx.x < ntiles) {
            issue_half(blockIdx.x, 0);
            issue_half(blockIdx.x, 1);
        }
        bool stop = false;
        for (int64_t t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++lt) {
            const int buf = (int)(lt & 1);
            const int64_t u = lt >> 1;
            int64_t tm, tn;
            tile_coords(a, t, tm, tn);
            const int64_t m0 = tm * kBM, n0 = tn * kBN;
            const bool acc_ok = nk == 0 || mbar_wait(&accf[buf], (uint32_t)(u & 1), a.err, 3);
            const bool have = nk > 0;   // uniform: tcgen05.ld is a .sync.aligned warp instruction
            const int64_t i = m0 + warp * 32 + lane;
            const bool row_ok = i < a.M;
            const uint32_t acc = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * kBN);
            const float *crow = sC + warp * 32 + lane;   // sC[j][row]
            for (int h = 0; h < 2; ++h) {
                // Both waits are bounded; whether to go on is then decided for
                // all four epilogue warps at once (a barrier reduction they all
                // reach), so that none is left at the named barrier below.
                const bool c_ok = !a.c_tma || mbar_wait(&cfull[h], (uint32_t)(lt & 1), a.err, 3);
                if (!epilogue_all(acc_ok && c_ok)) {
                    stop = true;
                    break;
                }
                fence_after();
#pragma unroll 1
                for (int c0 = 64 * h; c0 < 64 * h + 64; c0 += 32) {
                    float v[32];
                    if (have) tmem_ld32(acc + (uint32_t)c0, v);
                    else {
#pragma unroll
                        for (int q = 0; q < 32; ++q) v[q] = 0.f;
                    }
                    if (!row_ok) continue;
                    float cv[32];
                    float *prow = a.C + i * a.crs + (n0 + c0) * a.ccs;
                    const int64_t jmax = (a.cmode == MASK_LOWER && i < a.N - 1) ? i : a.N - 1;
                    const int cnt = (int)(jmax - (n0 + c0) + 1 < 32 ? jmax - (n0 + c0) + 1 : 32);
                    if (a.beta != 0.f) {
                        if (a.c_tma) {
#pragma unroll
                            for (int q = 0; q < 32; ++q) cv[q] = crow[(c0 + q) * kBM];
                        } else {
                            // All loads of the chunk are issued before any store (the
                            // stores could alias the loads as far as the compiler knows).
#pragma unroll
                            for (int q = 0; q < 32; ++q) cv[q] = q < cnt ? prow[q * a.ccs] : 0.f;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        if (q >= cnt) continue;
                        float out = a.alpha * v[q];
                        if (a.beta != 0.f) out = fmaf(a.beta, cv[q], out);
                        prow[q * a.ccs] = out;
                    }
                }
                if (a.c_tma) {
                    // every epilogue thread is done with half h of the staged tile
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    if (etid == 0 && t + gridDim.x < ntiles) issue_half(t + gridDim.x, h);
                }
            }
            if (stop) break;
            // this warp's lanes of the accumulator are read: hand it back
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[buf]);
        }
        // the last load of each half lands before teardown (a wait above may
        // have given up with it still in flight; a completed one returns at once)
        if (a.c_tma && etid == 0) {
            if (issued0 > 0) mbar_wait_quiet(&cfull[0], (uint32_t)((issued0 - 1) & 1));
            if (issued1 > 0) mbar_wait_quiet(&cfull[1], (uint32_t)((issued1 - 1) & 1));
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kBN)
                     : "memory");
    }
}

// ---- host side --------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D tensor map over a K-contiguous matrix: `rows` rows of `cols` elements,
// `pitch_bytes` apart (multiple of 16), box = 128 rows x 128 bytes, 128-byte
// swizzle, zero fill outside the matrix.
cudaError_t make_map(CUtensorMap *map, const void *ptr, int kind, int64_t rows, int64_t cols,
                     int64_t pitch_bytes)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const int esz = kind == 0 ? 2 : 4;
    if ((reinterpret_cast<uintptr_t>(ptr) % 16) || (pitch_bytes % 16)) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)kBM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 2-D tensor map over the FP32 C view (rows contiguous): M x N, columns
// `ld_elems` apart, box = 128 rows x kCBox columns, no swizzle, zero fill.
// Returns false (and the caller keeps C in registers) when the view does not
// meet TMA's rules: unit row stride, 16-byte aligned base and column stride.
bool make_c_map(CUtensorMap *map, const float *C, int64_t rs, int64_t ld_elems, int64_t M, int64_t N)
{
    auto fn = encode_fn();
    if (!fn || rs != 1 || (reinterpret_cast<uintptr_t>(C) % 16) || ((ld_elems * 4) % 16) || M <= 0 ||
        N <= 0 || ld_elems < M)
        return false;
    cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)(ld_elems * 4)};
    cuuint32_t box[2] = {(cuuint32_t)kBM, (cuuint32_t)kCBox};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(C), dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace tc

cudaError_t tc_gemm_nt(cudaStream_t st, int kind, const void *A, int64_t a_rows, int64_t a_pitch_elems,
                       int a_row0, const void *B, int64_t b_rows, int64_t b_pitch_elems, int b_row0,
                       View<float> C, int64_t M, int64_t N, int64_t K, float alpha, float beta,
                       int cmode, int *err)
{
    using namespace tc;
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int esz = kind == 0 ? 2 : 4;
    CUtensorMap ma, mb;
    cudaError_t e = make_map(&ma, A, kind, a_rows, K, a_pitch_elems * esz);
    if (e != cudaSuccess) return e;
    e = make_map(&mb, B, kind, b_rows, K, b_pitch_elems * esz);
    if (e != cudaSuccess) return e;
    Args args;
    args.C = C.p; args.crs = C.rs; args.ccs = C.cs;
    args.M = M; args.N = N; args.K = K;
    args.a_row0 = a_row0; args.b_row0 = b_row0;
    args.alpha = alpha; args.beta = beta; args.cmode = cmode;
    const int64_t tiles_m = (M + kBM - 1) / kBM, tiles_n = (N + kBN - 1) / kBN;
    args.tiles_n = (int)tiles_n;
    args.lower_tiles = (cmode == MASK_LOWER && M == N) ? 1 : 0;
    args.err = err;
    CUtensorMap mc = ma;   // unused unless C is staged by TMA
    args.c_tma = (beta != 0.f && make_c_map(&mc, C.p, C.rs, C.cs, M, N)) ? 1 : 0;
    args.num_tiles = args.lower_tiles ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
    // one CTA per SM (shared memory and TMEM fit one), never more than tiles
    const int64_t sms = device_sm_count();
    const int64_t grid = args.num_tiles < sms ? args.num_tiles : sms;
    if (kind == 0) {
        e = cudaFuncSetAttribute(tc_gemm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        tc_gemm_kernel<0><<<(unsigned)grid, kThreads, kSmemBytes, st>>>(ma, mb, mc, args);
    } else {
        e = cudaFuncSetAttribute(tc_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        tc_gemm_kernel<1><<<(unsigned)grid, kThreads, kSmemBytes, st>>>(ma, mb, mc, args);
    }
    note_launch();
    return cudaGetLastError();
}

}  // namespace rfp
