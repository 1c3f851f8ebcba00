// One-launch FP32 triangular solves with many 128-row blocks and few
// right-hand sides: L X = B or L^T X = B in place, L lower (the FP32 factor
// of the mixed-precision solve), with the inverses W_ii of L's 128 x 128
// diagonal blocks formed beforehand (inv_diag_blocks).
//
// The block forward substitution of Section 4 (Fig. 4, "solve"), written per
// block row i:
//   L X = B:    X_i = W_ii (B_i - sum_{j<i} L_ij X_j)
//   L^T X = B:  X_i = W_ii^T (B_i - sum_{j>i} L_ji^T X_j)
// A task is (block row i, group of 16 right-hand-side columns).  Tasks take
// tickets from a device counter in dependency order (block rows in solve
// order, then column groups); a task reads X_j only after the task that
// wrote it has raised its ready flag.  A CTA waits only on tasks with lower
// tickets, which were taken by CTAs that are already running and that wait
// only on lower tickets in turn, so every wait ends.  Each wait is also
// bounded in time: on expiry the CTA records an error code, and every other
// waiter gives up as soon as it sees a non-zero error word.
//
// Per task: 128 threads; each owns 8 rows x 2 columns of the 128 x 16 block
// in registers.  L is streamed through shared memory in 128 x 32 chunks
// (register-staged, double-buffered); X_j comes from L2 (ld.global.cg).
#include "rfp_internal.cuh"

namespace rfp {

namespace {

constexpr int kB = (int)kInvBlock;   // block rows (128)
constexpr int kG = 16;               // right-hand sides per task
constexpr int kKc = 32;              // K chunk staged in shared memory
constexpr int kThreads = 128;
constexpr int kLsLd = kB + 4;        // floats; rows stay 16-byte aligned
constexpr int kXsLd = kG + 2;        // floats; 2-way bank spread, 8-byte aligned pairs
constexpr uint64_t kWaitNs = 2000000000ull;

struct WfArgs {
    const float *L;
    int64_t ldl;
    const float *Inv;
    float *X;
    int64_t ldx, n, nrhs;
    int nb, ng;
    int32_t *counter, *flags, *err;
    const int32_t *stop;
};

__device__ __forceinline__ uint64_t wf_globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 waits until flag != 0; false if the error word is (or becomes) set.
__device__ __forceinline__ bool wait_flag(const int32_t *flag, int32_t *err)
{
    const uint64_t t0 = wf_globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (*(volatile const int32_t *)flag != 0) return true;
        if (*(volatile int32_t *)err != 0) return false;
        __nanosleep(64);
        if ((it & 63) == 63 && wf_globaltimer() - t0 > kWaitNs) {
            atomicCAS(err, 0, 4);
            return false;
        }
    }
}

// Chunk loader: op(A)(r, k) for r < 128, k in [k0, k0 + 32), into Ls[k - k0][r].
// TRANS = false: op(A)(r, k) = base[k * ld + r]  (A column-major)
// TRANS = true:  op(A)(r, k) = base[r * ld + k]  (A^T of a column-major A)
// Entries with r >= rv or k >= kv read as zero.  base and ld keep every
// float4 below 16-byte aligned (ld a multiple of 4, offsets multiples of 4).
template <bool TRANS>
struct ChunkLoader {
    float4 v[8];
    __device__ __forceinline__ void load(const float *base, int64_t ld, int k0, int rv, int kv)
    {
        const int tid = threadIdx.x;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (!TRANS) {
                const int kk = (tid >> 5) + 4 * q, r4 = (tid & 31) * 4, k = k0 + kk;
                const float *p = base + (int64_t)k * ld + r4;
                if (k < kv && r4 + 3 < rv) {
                    v[q] = *reinterpret_cast<const float4 *>(p);
                } else {
                    v[q].x = (k < kv && r4 + 0 < rv) ? p[0] : 0.f;
                    v[q].y = (k < kv && r4 + 1 < rv) ? p[1] : 0.f;
                    v[q].z = (k < kv && r4 + 2 < rv) ? p[2] : 0.f;
                    v[q].w = (k < kv && r4 + 3 < rv) ? p[3] : 0.f;
                }
            } else {
                const int r = tid, k = k0 + 4 * q;
                const float *p = base + (int64_t)r * ld + k;
                if (r < rv && k + 3 < kv) {
                    v[q] = *reinterpret_cast<const float4 *>(p);
                } else {
                    v[q].x = (r < rv && k + 0 < kv) ? p[0] : 0.f;
                    v[q].y = (r < rv && k + 1 < kv) ? p[1] : 0.f;
                    v[q].z = (r < rv && k + 2 < kv) ? p[2] : 0.f;
                    v[q].w = (r < rv && k + 3 < kv) ? p[3] : 0.f;
                }
            }
        }
    }
    __device__ __forceinline__ void store(float (*Ls)[kLsLd]) const
    {
        const int tid = threadIdx.x;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (!TRANS) {
                const int kk = (tid >> 5) + 4 * q, r4 = (tid & 31) * 4;
                *reinterpret_cast<float4 *>(&Ls[kk][r4]) = v[q];
            } else {
                const int r = tid, kk = 4 * q;
                Ls[kk + 0][r] = v[q].x;
                Ls[kk + 1][r] = v[q].y;
                Ls[kk + 2][r] = v[q].z;
                Ls[kk + 3][r] = v[q].w;
            }
        }
    }
};

// acc[m][c] += sign * sum_kk Ls[kk][row0 + m] * Xs[xk0 + kk][col0 + c]
template <bool SUB>
__device__ __forceinline__ void mma_chunk(float (&acc)[8][2], const float (*Ls)[kLsLd],
                                          const float (*Xs)[kXsLd], int xk0, int row0, int col0)
{
#pragma unroll 8
    for (int kk = 0; kk < kKc; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4 *>(&Ls[kk][row0]);
        const float4 a1 = *reinterpret_cast<const float4 *>(&Ls[kk][row0 + 4]);
        const float2 x = *reinterpret_cast<const float2 *>(&Xs[xk0 + kk][col0]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            acc[m][0] = SUB ? fmaf(-a[m], x.x, acc[m][0]) : fmaf(a[m], x.x, acc[m][0]);
            acc[m][1] = SUB ? fmaf(-a[m], x.y, acc[m][1]) : fmaf(a[m], x.y, acc[m][1]);
        }
    }
}

template <bool TRANS>
__global__ void __launch_bounds__(kThreads) trsm_wavefront_kernel(WfArgs a)
{
    __shared__ __align__(16) float Ls[2][kKc][kLsLd];
    __shared__ __align__(16) float Xs[kB][kXsLd];
    __shared__ int s_ticket, s_ok;

    if (a.stop && *a.stop) return;
    const int tid = threadIdx.x;
    if (tid == 0) s_ticket = atomicAdd(a.counter, 1);
    __syncthreads();
    const int ticket = s_ticket;
    const int g = ticket % a.ng, step = ticket / a.ng;
    const int i = TRANS ? a.nb - 1 - step : step;
    const int64_t r0 = (int64_t)i * kB;
    const int rows = (int)(a.n - r0 < kB ? a.n - r0 : kB);
    const int64_t c0 = (int64_t)g * kG;
    const int cols = (int)(a.nrhs - c0 < kG ? a.nrhs - c0 : kG);

    const int lane = tid & 31, warp = tid >> 5;
    const int row0 = warp * 32 + (lane >> 3) * 8;   // 8 rows
    const int col0 = (lane & 7) * 2;                 // 2 columns

    // acc = B_i (this task's own rows: nobody else writes them)
    float acc[8][2];
#pragma unroll
    for (int m = 0; m < 8; ++m)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int r = row0 + m, cc = col0 + c;
            acc[m][c] = (r < rows && cc < cols) ? a.X[(c0 + cc) * a.ldx + r0 + r] : 0.f;
        }

    // Off-diagonal blocks in solve order: forward j = 0 .. i-1, backward j = nb-1 .. i+1.
    const int nblk = TRANS ? a.nb - 1 - i : i;
    const int nq = nblk * (kB / kKc);
    auto blk = [&](int q) { return TRANS ? a.nb - 1 - q / (kB / kKc) : q / (kB / kKc); };
    auto chunk_base = [&](int j) -> const float * {
        return TRANS ? a.L + r0 * a.ldl + (int64_t)j * kB : a.L + (int64_t)j * kB * a.ldl + r0;
    };
    auto kvalid = [&](int j) { return (int)(a.n - (int64_t)j * kB < kB ? a.n - (int64_t)j * kB : kB); };

    ChunkLoader<TRANS> ld;
    if (nq > 0) {
        const int j = blk(0);
        ld.load(chunk_base(j), a.ldl, 0, rows, kvalid(j));
    }
    for (int q = 0; q < nq; ++q) {
        const int j = blk(q), s = q % (kB / kKc);
        if (s == 0) {   // X_j must be final: wait for its task's flag, then stage it
            if (tid == 0) {
                s_ok = wait_flag(a.flags + (int64_t)j * a.ng + g, a.err) ? 1 : 0;
                __threadfence();
            }
            __syncthreads();
            if (!s_ok) return;
            const int kv = kvalid(j);
            const float *xj = a.X + (int64_t)j * kB;
#pragma unroll 4
            for (int c = 0; c < kG; ++c)
                Xs[tid][c] = (tid < kv && c < cols) ? __ldcg(xj + (c0 + c) * a.ldx + tid) : 0.f;
        }
        ld.store(Ls[q & 1]);
        __syncthreads();
        if (q + 1 < nq) {
            const int jn = blk(q + 1);
            ld.load(chunk_base(jn), a.ldl, ((q + 1) % (kB / kKc)) * kKc, rows, kvalid(jn));
        }
        mma_chunk<true>(acc, Ls[q & 1], Xs, s * kKc, row0, col0);
        __syncthreads();
    }

    // Diagonal block: X_i = op(W_ii) acc.
#pragma unroll
    for (int m = 0; m < 8; ++m)
#pragma unroll
        for (int c = 0; c < 2; ++c) Xs[row0 + m][col0 + c] = acc[m][c];
    float out[8][2] = {};
    const float *W = a.Inv + (int64_t)i * kB * kB;
    ld.load(W, kB, 0, rows, rows);
    for (int s = 0; s < kB / kKc; ++s) {
        ld.store(Ls[s & 1]);
        __syncthreads();
        if (s + 1 < kB / kKc) ld.load(W, kB, (s + 1) * kKc, rows, rows);
        mma_chunk<false>(out, Ls[s & 1], Xs, s * kKc, row0, col0);
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < 8; ++m)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int r = row0 + m, cc = col0 + c;
            if (r < rows && cc < cols) a.X[(c0 + cc) * a.ldx + r0 + r] = out[m][c];
        }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicExch(a.flags + (int64_t)i * a.ng + g, 1);
}

}  // namespace

size_t wavefront_sync_words(int64_t n, int64_t nrhs)
{
    const int64_t nb = (n + kB - 1) / kB, ng = (nrhs + kG - 1) / kG;
    return (size_t)(1 + nb * ng);
}

cudaError_t trsm_wavefront(cudaStream_t st, View<float> Lv, int64_t n, const float *Inv, float *X,
                           int64_t ldx, int64_t nrhs, bool trans, int32_t *sync, int32_t *err,
                           const int32_t *stop)
{
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    if (Lv.rs != 1 || Lv.cs % 4 != 0 || reinterpret_cast<uintptr_t>(Lv.p) % 16 != 0 ||
        reinterpret_cast<uintptr_t>(Inv) % 16 != 0)
        return cudaErrorInvalidValue;   // the chunk loader's float4 alignment
    const int64_t nb = (n + kB - 1) / kB, ng = (nrhs + kG - 1) / kG;
    cudaError_t e = cudaMemsetAsync(sync, 0, wavefront_sync_words(n, nrhs) * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    WfArgs a{Lv.p, Lv.cs, Inv, X, ldx, n, nrhs, (int)nb, (int)ng, sync, sync + 1, err, stop};
    const unsigned grid = (unsigned)(nb * ng);
    if (trans) trsm_wavefront_kernel<true><<<grid, kThreads, 0, st>>>(a);
    else trsm_wavefront_kernel<false><<<grid, kThreads, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace rfp
