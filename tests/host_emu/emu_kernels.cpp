// CPU emulation of the library's kernel launchers (tile_kernels.cu, pack.cu),
// used ONLY by tests/test_host_orchestration.py to check the host-side
// orchestration (chol.cu, api.cu) without a GPU.
//
// Each launcher is emulated with the same CTA decomposition as its kernel.
// Within one launch every CTA computes from the memory state before the
// launch and its writes are applied afterwards; every address a CTA touches is
// recorded, and a launch fails (illegal-address / race error) if
//   - any access falls outside the buffers registered with emu_register, or
//   - an element written by one CTA is read or written by another CTA.
// A launch free of such conflicts gives the same result in any CTA order, so
// the emulated result equals the GPU result up to floating-point rounding.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <unordered_map>
#include <vector>

#include "../../paper_0901_1696_gb300/csrc/mixed_internal.cuh"
#include "../../paper_0901_1696_gb300/csrc/rfp_internal.cuh"

namespace {

struct Region { uintptr_t lo, hi; };
std::vector<Region> g_regions;
int g_violations = 0;
char g_msg[512] = "";
long g_launches = 0;

bool in_bounds(const void *p, size_t sz)
{
    uintptr_t a = (uintptr_t)p;
    for (auto &r : g_regions)
        if (a >= r.lo && a + sz <= r.hi) return true;
    return false;
}

void violation(const char *what, const void *p)
{
    if (g_violations++ == 0) snprintf(g_msg, sizeof g_msg, "%s at %p", what, p);
}

// Access log of one launch: address -> (first CTA id, written?)
struct Launch {
    std::unordered_map<uintptr_t, int> writer;               // addr -> cta
    std::unordered_map<uintptr_t, std::vector<int>> readers;  // addr -> ctas
    std::vector<std::pair<void *, double>> pend_d;
    std::vector<std::pair<void *, float>> pend_f;
    std::vector<std::pair<void *, uint16_t>> pend_b;
    int cta = 0;
    // Ordered launches (CTAs that hand results to each other through ready
    // flags) run their CTAs in ticket order with writes applied at once;
    // only bounds are checked.
    bool ordered = false;
    template <typename T>
    T rd(const T *p)
    {
        if (!in_bounds(p, sizeof(T))) { violation("out-of-bounds read", p); return T(0); }
        if (ordered) return *p;
        auto &v = readers[(uintptr_t)p];
        if (v.empty() || v.back() != cta) v.push_back(cta);
        return *p;
    }
    void wr(double *p, double x)
    {
        if (ordered) { if (in_bounds(p, 8)) *p = x; else violation("out-of-bounds write", p); return; }
        wr_any(p, sizeof(double)); pend_d.push_back({p, x});
    }
    void wr(float *p, float x)
    {
        if (ordered) { if (in_bounds(p, 4)) *p = x; else violation("out-of-bounds write", p); return; }
        wr_any(p, sizeof(float)); pend_f.push_back({p, x});
    }
    void wr(int32_t *p, int32_t x)
    {
        if (!in_bounds(p, 4)) { violation("out-of-bounds write", p); return; }
        if (!ordered) violation("int write outside an ordered launch", p);
        *p = x;
    }
    void wr_any(void *p, size_t sz)
    {
        if (!in_bounds(p, sz)) { violation("out-of-bounds write", p); return; }
        auto it = writer.find((uintptr_t)p);
        if (it != writer.end() && it->second != cta) violation("two CTAs write one element", p);
        writer[(uintptr_t)p] = cta;
    }
    cudaError_t commit()
    {
        ++g_launches;
        for (auto &kv : writer) {
            auto it = readers.find(kv.first);
            if (it == readers.end()) continue;
            for (int c : it->second)
                if (c != kv.second) { violation("element written by one CTA and read by another", (void *)kv.first); break; }
        }
        for (auto &w : pend_d) *(double *)w.first = w.second;
        for (auto &w : pend_f) *(float *)w.first = w.second;
        for (auto &w : pend_b) *(uint16_t *)w.first = w.second;
        return g_violations ? cudaErrorIllegalAddress : cudaSuccess;
    }
};


bool aborted(Launch &L, const int32_t *abort) { return abort && L.rd(abort) != 0; }

}  // namespace

extern "C" {
void emu_reset() { g_regions.clear(); g_violations = 0; g_msg[0] = 0; g_launches = 0; }
void emu_register(void *p, size_t bytes) { g_regions.push_back({(uintptr_t)p, (uintptr_t)p + bytes}); }
int emu_violations() { return g_violations; }
const char *emu_message() { return g_msg; }
long emu_launches() { return g_launches; }
void emu_set_sms(int);
}

cudaError_t cudaMemsetAsync(void *p, int v, size_t n, cudaStream_t)
{
    if (!in_bounds(p, n)) { violation("out-of-bounds memset", p); return cudaErrorIllegalAddress; }
    memset(p, v, n);
    return cudaSuccess;
}
const char *cudaGetErrorName(cudaError_t e) { return e ? "emulated error" : "cudaSuccess"; }
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
cudaError_t cudaEventCreate(cudaEvent_t *e) { *e = nullptr; return cudaSuccess; }
cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t, cudaEvent_t) { *ms = 0.f; return cudaSuccess; }

namespace rfp {

// The emulated device has the SM count given by emu_set_sms (default 152).
static int g_emu_sms = 152;
int device_sm_count() { return g_emu_sms; }

template <typename T>
cudaError_t gemm_nt(cudaStream_t, View<T> C, View<T> A, View<T> B, int64_t M, int64_t N, int64_t K,
                    T alpha, T beta, int cmode, int amask, int bmask, const int32_t *abort,
                    int inplace)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K <= 0 && beta == T(1)) return cudaSuccess;
    // resident CTAs per SM of the GB300 build (large / small): FP64 2 / 5, FP32 1 / 2
    const GemmTileChoice tc = gemm_tile_choice(M, N, cmode, inplace, (int)sizeof(T), device_sm_count(),
                                               sizeof(T) == 8 ? 2 : 1, sizeof(T) == 8 ? 5 : 2);
    const int BM = tc.bm, BN = tc.bn;
    Launch L;
    const int64_t gy = (M + BM - 1) / BM, gx = (N + BN - 1) / BN;
    for (int64_t by = 0; by < gy; ++by)
        for (int64_t bx = 0; bx < gx; ++bx) {
            L.cta = (int)(by * gx + bx);
            if (aborted(L, abort)) continue;
            const int64_t m0 = by * BM, n0 = bx * BN;
            if (cmode == MASK_LOWER && m0 + BM - 1 < n0) continue;
            int64_t kbeg = 0, kend = K;
            if (amask == MASK_LOWER || amask == MASK_STRICT_LOWER) kend = std::min(kend, m0 + BM);
            if (amask == MASK_UPPER || amask == MASK_STRICT_UPPER) kbeg = std::max(kbeg, m0);
            if (bmask == MASK_LOWER || bmask == MASK_STRICT_LOWER) kend = std::min(kend, n0 + BN);
            if (bmask == MASK_UPPER || bmask == MASK_STRICT_UPPER) kbeg = std::max(kbeg, n0);
            for (int64_t i = m0; i < std::min(M, m0 + BM); ++i)
                for (int64_t j = n0; j < std::min(N, n0 + BN); ++j) {
                    T acc = T(0);
                    for (int64_t k = kbeg; k < kend; ++k) {
                        bool aok = mask_keeps(amask, i, k);
                        bool bok = mask_keeps(bmask, j, k);
                        T a = aok ? L.rd(&A(i, k)) : T(0);
                        T b = bok ? L.rd(&B(j, k)) : T(0);
                        acc += a * b;
                    }
                    if (cmode == MASK_LOWER && j > i) continue;
                    T v = alpha * acc;
                    if (beta != T(0)) v += beta * L.rd(&C(i, j));
                    L.wr(&C(i, j), v);
                }
        }
    return L.commit();
}

// Split-K: CTA (z, tile) writes slice z of the work buffer, then the reduce
// kernel sums the slices into C (one CTA per element range).
template <typename T>
cudaError_t gemm_nt_splitk(cudaStream_t st, View<T> C, View<T> A, View<T> B, int64_t M, int64_t N,
                           int64_t K, T alpha, T beta, int cmode, int amask, int bmask,
                           const int32_t *abort, int splits, T *work)
{
    if (splits <= 1 || !work) return gemm_nt(st, C, A, B, M, N, K, alpha, beta, cmode, amask, bmask, abort);
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int64_t kc = (K + splits - 1) / splits;
    for (int z = 0; z < splits; ++z) {      // each slice's launch part, checked like a launch
        const int64_t k0 = std::min<int64_t>(K, z * kc), k1 = std::min<int64_t>(K, k0 + kc);
        View<T> Wz{work + (int64_t)z * M * N, 1, M};
        cudaError_t e;
        if (k1 > k0) {
            e = gemm_nt(st, Wz, A.sub(0, k0), B.sub(0, k0), M, N, k1 - k0, T(1), T(0), cmode,
                        MASK_NONE, MASK_NONE, abort, false);
            // masks in the full K coordinates: emulate directly when a mask is set
            if (amask != MASK_NONE || bmask != MASK_NONE) {
                Launch L;
                for (int64_t i = 0; i < M; ++i)
                    for (int64_t j = 0; j < N; ++j) {
                        T acc = T(0);
                        for (int64_t k = k0; k < k1; ++k) {
                            T a = mask_keeps(amask, i, k) ? L.rd(&A(i, k)) : T(0);
                            T b = mask_keeps(bmask, j, k) ? L.rd(&B(j, k)) : T(0);
                            acc += a * b;
                        }
                        L.wr(&Wz(i, j), acc);
                    }
                e = L.commit();
            }
        } else {
            Launch L;
            for (int64_t i = 0; i < M; ++i)
                for (int64_t j = 0; j < N; ++j) L.wr(&Wz(i, j), T(0));
            e = L.commit();
        }
        if (e != cudaSuccess) return e;
    }
    Launch L;
    if (abort && L.rd(abort)) return L.commit();
    for (int64_t j = 0; j < N; ++j)
        for (int64_t i = 0; i < M; ++i) {
            if (cmode == MASK_LOWER && j > i) continue;
            T s = T(0);
            for (int z = 0; z < splits; ++z) s += L.rd(&work[(int64_t)z * M * N + i + j * M]);
            T v = alpha * s;
            if (beta != T(0)) v += beta * L.rd(&C(i, j));
            L.wr(&C(i, j), v);
        }
    return L.commit();
}

template <typename T>
cudaError_t trsm_strip(cudaStream_t, View<T> X, View<T> Lt, int64_t M, int w, int transL, T alpha,
                       const int32_t *abort, bool unit)
{
    if (M <= 0 || w <= 0) return cudaSuccess;
    if (w > 64) { violation("trsm tile wider than 64", nullptr); return cudaErrorInvalidValue; }
    Launch L;
    for (int64_t r0 = 0, cta = 0; r0 < M; r0 += 64, ++cta) {
        L.cta = (int)cta;
        if (aborted(L, abort)) continue;
        std::vector<T> l(w * w), x;
        for (int i = 0; i < w; ++i)
            for (int j = 0; j <= i; ++j)
                l[i * w + j] = (unit && i == j) ? T(1) : L.rd(&Lt(i, j));   // unit: diagonal not read
        for (int64_t r = r0; r < std::min(M, r0 + 64); ++r) {
            x.assign(w, T(0));
            for (int c = 0; c < w; ++c) x[c] = alpha * L.rd(&X(r, c));
            if (transL) {
                for (int j = 0; j < w; ++j) {
                    x[j] /= l[j * w + j];
                    for (int c = j + 1; c < w; ++c) x[c] -= x[j] * l[c * w + j];
                }
            } else {
                for (int j = w - 1; j >= 0; --j) {
                    x[j] /= l[j * w + j];
                    for (int c = 0; c < j; ++c) x[c] -= x[j] * l[j * w + c];
                }
            }
            for (int c = 0; c < w; ++c) L.wr(&X(r, c), x[c]);
        }
    }
    return L.commit();
}

template <typename T>
cudaError_t potrf_tile(cudaStream_t, View<T> A, int w, int32_t *info, int64_t base)
{
    if (w <= 0) return cudaSuccess;
    Launch L;
    if (L.rd(info) != 0) return L.commit();
    std::vector<T> s(w * w, T(0));
    for (int i = 0; i < w; ++i)
        for (int j = 0; j <= i; ++j) s[i * w + j] = L.rd(&A(i, j));
    for (int j = 0; j < w; ++j) {
        T d = s[j * w + j];
        if (!(d > T(0))) {
            int32_t v = (int32_t)(base + j + 1);
            L.wr_any(info, 4);
            L.commit();
            *info = v;
            return g_violations ? cudaErrorIllegalAddress : cudaSuccess;
        }
        const T sqd = std::sqrt(d), ri = T(1) / sqd;   // same arithmetic as the kernel
        s[j * w + j] = sqd;
        for (int i = j + 1; i < w; ++i) s[i * w + j] *= ri;
        for (int i = j + 1; i < w; ++i)
            for (int k = j + 1; k <= i; ++k) s[i * w + k] -= s[i * w + j] * s[k * w + j];
    }
    for (int i = 0; i < w; ++i)
        for (int j = 0; j <= i; ++j) L.wr(&A(i, j), s[i * w + j]);
    return L.commit();
}

template <typename T>
cudaError_t trtri_tile(cudaStream_t, View<T> A, int w, const int32_t *abort)
{
    if (w <= 0) return cudaSuccess;
    Launch L;
    if (aborted(L, abort)) return L.commit();
    std::vector<T> l(w * w, T(0)), x(w * w, T(0));
    for (int i = 0; i < w; ++i)
        for (int j = 0; j <= i; ++j) l[i * w + j] = L.rd(&A(i, j));
    for (int c = 0; c < w; ++c) {
        x[c * w + c] = T(1) / l[c * w + c];
        for (int i = c + 1; i < w; ++i) {
            T s = T(0);
            for (int p = c; p < i; ++p) s += l[i * w + p] * x[p * w + c];
            x[i * w + c] = -s / l[i * w + i];
        }
    }
    for (int i = 0; i < w; ++i)
        for (int j = 0; j <= i; ++j) L.wr(&A(i, j), x[i * w + j]);
    return L.commit();
}

// One-launch block triangular solve: tasks (block row, 16-column group) in
// ticket order; each reads its rows of X, the blocks of L before (forward)
// or after (backward) its diagonal block, the finished X blocks of the
// earlier tasks and its inverted diagonal block, and writes its X block and
// ready flag.
size_t wavefront_sync_words(int64_t n, int64_t nrhs)
{
    const int64_t nb = (n + kInvBlock - 1) / kInvBlock, ng = (nrhs + 15) / 16;
    return (size_t)(1 + nb * ng);
}

cudaError_t trsm_wavefront(cudaStream_t, View<float> Lv, int64_t n, const float *Inv, float *X,
                           int64_t ldx, int64_t nrhs, bool trans, int32_t *sync, int32_t *err,
                           const int32_t *stop)
{
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    if (Lv.rs != 1 || Lv.cs % 4 != 0 || (uintptr_t)Lv.p % 16 || (uintptr_t)Inv % 16)
        return cudaErrorInvalidValue;
    const int64_t B = kInvBlock, nb = (n + B - 1) / B, ng = (nrhs + 15) / 16;
    Launch L;
    L.ordered = true;
    for (size_t w = 0; w < wavefront_sync_words(n, nrhs); ++w) L.wr(sync + w, 0);   // the memset
    (void)err;
    if (aborted(L, stop)) return L.commit();
    for (int64_t t = 0; t < nb * ng; ++t) {
        L.cta = (int)t;
        L.wr(sync, (int32_t)(t + 1));                       // ticket counter
        const int64_t g = t % ng, step = t / ng, i = trans ? nb - 1 - step : step;
        const int64_t r0 = i * B, rows = std::min(B, n - r0), c0 = g * 16,
                      cols = std::min<int64_t>(16, nrhs - c0);
        std::vector<float> acc(rows * cols);
        for (int64_t c = 0; c < cols; ++c)
            for (int64_t r = 0; r < rows; ++r) acc[c * rows + r] = L.rd(&X[(c0 + c) * ldx + r0 + r]);
        const int64_t jlo = trans ? i + 1 : 0, jhi = trans ? nb : i;
        for (int64_t jj = jlo; jj < jhi; ++jj) {
            const int64_t j = trans ? nb - 1 - (jj - jlo) : jj;   // solve order
            if (L.rd(sync + 1 + j * ng + g) != 1) violation("X block read before its flag", sync);
            const int64_t kv = std::min(B, n - j * B);
            for (int64_t c = 0; c < cols; ++c)
                for (int64_t r = 0; r < rows; ++r) {
                    float s = acc[c * rows + r];
                    for (int64_t k = 0; k < kv; ++k) {
                        const float a = trans ? L.rd(&Lv(j * B + k, r0 + r)) : L.rd(&Lv(r0 + r, j * B + k));
                        s -= a * L.rd(&X[(c0 + c) * ldx + j * B + k]);
                    }
                    acc[c * rows + r] = s;
                }
        }
        const float *W = Inv + i * B * B;                    // column-major, ld B
        for (int64_t c = 0; c < cols; ++c)
            for (int64_t r = 0; r < rows; ++r) {
                float s = 0.f;
                for (int64_t k = 0; k < rows; ++k)
                    s += (trans ? L.rd(&W[r * B + k]) : L.rd(&W[k * B + r])) * acc[c * rows + k];
                L.wr(&X[(c0 + c) * ldx + r0 + r], s);
            }
        L.wr(sync + 1 + i * ng + g, 1);
    }
    return L.commit();
}

// rfp_solve: one ordered launch of (block row, column group) tasks in
// ticket order (block rows in solve order, then column groups).  Each task
// reads its rows of X, the blocks of L to the left of its diagonal block
// (forward) or below it (backward), transposed for the backward solve, and the
// final X blocks of the earlier tasks of its group; it writes its X block
// and its group's progress word.  L is addressed through the three RFP block
// views exactly as the kernel addresses it.
// right-hand sides per task, as the kernel picks them
static int64_t solve_group(int64_t nrhs) { return nrhs <= 16 ? 8 : 16; }
size_t rfp_solve_sync_words(int64_t nrhs)
{
    const int64_t G = solve_group(nrhs);
    return (size_t)(2 + (nrhs + G - 1) / G);
}

cudaError_t rfp_solve(cudaStream_t, View<double> t1, View<double> s, View<double> t2, int64_t n1,
                      int64_t n2, View<double> Xv, int64_t nrhs, bool trans, int32_t *sync,
                      const int32_t *abort, double alpha, bool lower_rhs)
{
    const int64_t n = n1 + n2;
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    if (lower_rhs && (trans || n2 != 0)) return cudaErrorInvalidValue;
    const int64_t R = n <= 4096 ? 32 : 64;             // block rows, as the kernel picks them
    const int64_t G = solve_group(nrhs);
    const int64_t nb1 = (n1 + R - 1) / R, nb = nb1 + (n2 + R - 1) / R, ng = (nrhs + G - 1) / G;
    Launch L;
    L.ordered = true;
    for (size_t w = 0; w < rfp_solve_sync_words(nrhs); ++w) L.wr(sync + w, 0);   // the memset
    if (aborted(L, abort)) return L.commit();
    auto xat = [&](int64_t r, int64_t c) { return &Xv(r, c); };
    auto rows_of = [&](int64_t b, int64_t &r0, int64_t &rows) {
        if (b < nb1) { r0 = b * R; rows = std::min(R, n1 - r0); }
        else { const int64_t lr = (b - nb1) * R; r0 = n1 + lr; rows = std::min(R, n2 - lr); }
    };
    // element (i, j), i >= j, of block (bi, bj) of L
    auto lel = [&](int64_t bi, int64_t bj, int64_t i, int64_t j) -> const double * {
        const int64_t ri = (bi < nb1 ? bi * R : (bi - nb1) * R) + i;
        const int64_t cj = (bj < nb1 ? bj * R : (bj - nb1) * R) + j;
        if (bi < nb1) return &t1(ri, cj);
        if (bj < nb1) return &s(ri, cj);
        return &t2(ri, cj);
    };
    int32_t *prog = sync + 2;
    for (int64_t t = 0; t < nb * ng; ++t) {
        L.cta = (int)t;
        L.wr(sync, (int32_t)(t + 1));                       // ticket counter
        const int64_t g = t % ng, p = t / ng, b = trans ? nb - 1 - p : p;
        const int64_t c0 = g * G, cols = std::min<int64_t>(G, nrhs - c0);
        const int64_t jf = lower_rhs ? c0 / R : 0;   // blocks above stay zero, untouched
        if (b < jf) continue;
        int64_t r0, rows;
        rows_of(b, r0, rows);
        std::vector<double> acc(rows * cols);
        for (int64_t c = 0; c < cols; ++c)
            for (int64_t r = 0; r < rows; ++r) acc[c * rows + r] = alpha * L.rd(xat(r0 + r, c0 + c));
        for (int64_t q = jf; q < p; ++q) {
            const int64_t j = trans ? nb - 1 - q : q;
            if (L.rd(prog + g) < q + 1) violation("X block read before its group's progress", prog + g);
            int64_t j0, kv;
            rows_of(j, j0, kv);
            for (int64_t c = 0; c < cols; ++c)
                for (int64_t r = 0; r < rows; ++r) {
                    double sum = acc[c * rows + r];
                    for (int64_t k = 0; k < kv; ++k) {
                        const double a = trans ? L.rd(lel(j, b, k, r)) : L.rd(lel(b, j, r, k));
                        sum -= a * L.rd(xat(j0 + k, c0 + c));
                    }
                    acc[c * rows + r] = sum;
                }
        }
        for (int64_t c = 0; c < cols; ++c) {     // substitution with the diagonal block
            double *v = &acc[c * rows];
            if (!trans) {
                for (int64_t j = 0; j < rows; ++j) {
                    v[j] /= L.rd(lel(b, b, j, j));
                    for (int64_t r = j + 1; r < rows; ++r) v[r] -= L.rd(lel(b, b, r, j)) * v[j];
                }
            } else {
                for (int64_t j = rows - 1; j >= 0; --j) {
                    v[j] /= L.rd(lel(b, b, j, j));
                    for (int64_t r = 0; r < j; ++r) v[r] -= L.rd(lel(b, b, j, r)) * v[j];
                }
            }
            for (int64_t r = 0; r < rows; ++r) L.wr(xat(r0 + r, c0 + c), v[r]);
        }
        L.wr(prog + g, (int32_t)(p + 1));
    }
    return L.commit();
}

// potrf_step: one ordered launch (ticket order: the diagonal tile of panel
// k+1, its 32-row (m <= 2048) or 64-row strips, then the lower tiles of
// A(k2:m, k2:m), 32 or 64 wide by the kernel's rule) with the kernel's own
// tile decomposition; panels 32 wide for m <= 4096, 64 beyond.  Besides the bounds checks, every element one
// task writes is recorded, and a read of it by another task is a violation
// unless it is the new diagonal tile read by a strip (which the kernel does
// only after the diagonal task's flag).
// The kernel's rules (panels 32 wide up to m = 4096, strips 32 rows up to
// m = 2048); emu_set_step_rules lowers the bounds so that small orders also
// take the 64-wide panels and 64-row strips, and a bulk tile width can be
// forced.
static int64_t g_narrow_panels = 4096, g_small_strips = 2048, g_bulk_tile = 0;
extern "C" void emu_set_step_rules(long narrow_panels, long small_strips, long bulk_tile)
{
    g_narrow_panels = narrow_panels;
    g_small_strips = small_strips;
    g_bulk_tile = bulk_tile;   // 0: the kernel's rule; 32 or 64: that width
}

int potrf_step_width(int64_t m)
{
    return m <= g_narrow_panels ? 32 : 64;
}

size_t potrf_step_sync_words(int64_t m)
{
    const int64_t pw = potrf_step_width(m), np = (m + pw - 1) / pw;
    return (size_t)(2 * (np > 1 ? np - 1 : 1));
}

cudaError_t potrf_step(cudaStream_t, View<double> V, int64_t m, int64_t k0, int32_t *info,
                       int64_t base, int32_t *sync)
{
    const int64_t P = potrf_step_width(m), k1 = std::min(k0 + P, m);
    if (k1 >= m) return cudaSuccess;
    const int64_t k2 = std::min(k1 + P, m), w = k1 - k0, wn = k2 - k1;
    const int64_t T = g_bulk_tile ? g_bulk_tile : potrf_step_bulk_tile(m - k2, 2 * (int64_t)device_sm_count());
    const int64_t S = m <= g_small_strips ? 32 : 64;  // rows per strip task
    const int64_t rest = (m - k2 + T - 1) / T, nstrip = (m - k2 + S - 1) / S, nbulk = rest * (rest + 1) / 2;
    Launch L;
    L.ordered = true;
    if (L.rd(info) != 0) return L.commit();
    std::unordered_map<uintptr_t, int64_t> owner;
    int64_t task = 0;
    auto in_diag = [&](const double *p) {
        for (int64_t i = 0; i < wn; ++i)
            for (int64_t j = 0; j <= i; ++j)
                if (p == &V(k1 + i, k1 + j)) return true;
        return false;
    };
    auto rd = [&](const double *p) {
        auto it = owner.find((uintptr_t)p);
        if (it != owner.end() && it->second != task && !(it->second == 0 && task <= nstrip && in_diag(p)))
            violation("potrf_step: element written by one task and read by another", p);
        return L.rd(p);
    };
    auto wr = [&](double *p, double v) {
        auto it = owner.find((uintptr_t)p);
        if (it != owner.end() && it->second != task) violation("potrf_step: two tasks write one element", p);
        owner[(uintptr_t)p] = task;
        L.wr(p, v);
    };
    // P_rows P_cols^T over the panel columns [k0, k1)
    auto prod = [&](int64_t r, int64_t c) {
        double sum = 0.0;
        for (int64_t k = 0; k < w; ++k) sum += rd(&V(r, k0 + k)) * rd(&V(c, k0 + k));
        return sum;
    };
    int32_t flag = 0;
    L.wr(sync, 1);                                   // ticket counter
    {   // diagonal tile
        task = 0;
        std::vector<double> D(wn * wn, 0.0);
        for (int64_t i = 0; i < wn; ++i)
            for (int64_t j = 0; j <= i; ++j) D[i * wn + j] = rd(&V(k1 + i, k1 + j)) - prod(k1 + i, k1 + j);
        int64_t fail = -1;
        std::vector<double> sq(wn);
        for (int64_t j = 0; j < wn && fail < 0; ++j) {
            const double d = D[j * wn + j];
            if (!(d > 0.0)) { fail = j; break; }
            sq[j] = std::sqrt(d);
            const double ri = 1.0 / sq[j];
            for (int64_t i = j + 1; i < wn; ++i) D[i * wn + j] *= ri;
            for (int64_t i = j + 1; i < wn; ++i)
                for (int64_t k = j + 1; k <= i; ++k) D[i * wn + k] -= D[i * wn + j] * D[k * wn + j];
        }
        if (fail >= 0) {
            if (L.rd(info) == 0) L.wr(info, (int32_t)(base + k1 + fail + 1));
            flag = 2;
        } else {
            for (int64_t i = 0; i < wn; ++i)
                for (int64_t j = 0; j <= i; ++j) wr(&V(k1 + i, k1 + j), i == j ? sq[j] : D[i * wn + j]);
            flag = 1;
        }
        L.wr(sync + 1, flag);
    }
    for (int64_t s = 0; s < nstrip; ++s) {   // strips of panel k+1
        task = 1 + s;
        L.wr(sync, (int32_t)(task + 1));
        const int64_t r0 = k2 + s * S, nr = std::min(S, m - r0);
        std::vector<double> X(nr * wn);
        for (int64_t i = 0; i < nr; ++i)
            for (int64_t j = 0; j < wn; ++j) X[i * wn + j] = rd(&V(r0 + i, k1 + j)) - prod(r0 + i, k1 + j);
        if (flag != 1) continue;
        for (int64_t i = 0; i < nr; ++i) {
            for (int64_t j = 0; j < wn; ++j) {
                X[i * wn + j] *= 1.0 / rd(&V(k1 + j, k1 + j));
                for (int64_t c = j + 1; c < wn; ++c) X[i * wn + c] -= X[i * wn + j] * rd(&V(k1 + c, k1 + j));
            }
            for (int64_t j = 0; j < wn; ++j) wr(&V(r0 + i, k1 + j), X[i * wn + j]);
        }
    }
    for (int64_t b = 0; b < nbulk; ++b) {    // lower tiles of A(k2:m, k2:m)
        task = 1 + nstrip + b;
        L.wr(sync, (int32_t)(task + 1));
        int64_t ti = 0;
        while ((ti + 1) * (ti + 2) / 2 <= b) ++ti;
        const int64_t tj = b - ti * (ti + 1) / 2;
        const int64_t r0 = k2 + ti * T, c0 = k2 + tj * T;
        const int64_t nr = std::min(T, m - r0), nc = std::min(T, m - c0);
        for (int64_t i = 0; i < nr; ++i)
            for (int64_t j = 0; j < nc; ++j) {
                if (ti == tj && j > i) continue;
                wr(&V(r0 + i, c0 + j), rd(&V(r0 + i, c0 + j)) - prod(r0 + i, c0 + j));
            }
    }
    return L.commit();
}

// identity_fill / lower_copy: one launch each, every element of the m x m
// destination (lower triangle for the copy) written once.
cudaError_t identity_fill(cudaStream_t, View<double> W, int64_t m, const int32_t *abort)
{
    Launch L;
    if (aborted(L, abort)) return L.commit();
    for (int64_t j = 0; j < m; ++j)
        for (int64_t i = 0; i < m; ++i) L.wr(&W(i, j), i == j ? 1.0 : 0.0);
    return L.commit();
}

cudaError_t lower_copy(cudaStream_t, View<double> dst, View<double> src, int64_t m,
                       const int32_t *abort)
{
    Launch L;
    if (aborted(L, abort)) return L.commit();
    for (int64_t j = 0; j < m; ++j)
        for (int64_t i = j; i < m; ++i) L.wr(&dst(i, j), L.rd(&src(i, j)));
    return L.commit();
}

// The emulated scratch: heap memory registered as a device buffer for the
// duration of the call.
cudaError_t solve_scratch_acquire(cudaStream_t, size_t words, int32_t **out)
{
    int32_t *p = new int32_t[words];
    emu_register(p, words * sizeof(int32_t));
    *out = p;
    return cudaSuccess;
}

cudaError_t solve_scratch_release(cudaStream_t, int32_t *p)
{
    for (size_t i = 0; i < g_regions.size(); ++i)
        if (g_regions[i].lo == (uintptr_t)p) {
            g_regions.erase(g_regions.begin() + (long)i);
            break;
        }
    delete[] p;
    return cudaSuccess;
}

// ---- the rest of the LAPACK 3.2 RFP routine set ----

template <typename T>
struct EmuLower {
    View<T> t1, s, t2;
    int64_t n1;
    T *at(int64_t i, int64_t j) const
    {
        if (j >= n1) return &t2(i - n1, j - n1);
        if (i >= n1) return &s(i - n1, j);
        return &t1(i, j);
    }
};
template <typename T>
EmuLower<T> emu_lower(const Layout &Ly, T *arf)
{
    return EmuLower<T>{block_view(arf, Ly, Ly.t1), block_view(arf, Ly, Ly.s), block_view(arf, Ly, Ly.t2),
                       Ly.n1};
}

// One CTA per 32 x 32 tile on or below the diagonal.
template <typename T>
cudaError_t tp_copy(cudaStream_t, const Layout &Ly, T *arf, T *ap, bool lowerTP, bool to_rfp)
{
    const int64_t n = Ly.n;
    if (n <= 0) return cudaSuccess;
    EmuLower<T> Lw = emu_lower(Ly, arf);
    Launch L;
    const int64_t t = (n + 31) / 32;
    for (int64_t ti = 0; ti < t; ++ti)
        for (int64_t tj = 0; tj <= ti; ++tj) {
            L.cta = (int)(ti * t + tj);
            for (int64_t i = ti * 32; i < std::min(n, ti * 32 + 32); ++i)
                for (int64_t j = tj * 32; j < std::min(i + 1, tj * 32 + 32); ++j) {
                    const int64_t p = lowerTP ? i + j * (2 * n - j - 1) / 2 : j + i * (i + 1) / 2;
                    if (to_rfp) L.wr(Lw.at(i, j), L.rd(ap + p));
                    else L.wr(ap + p, L.rd(Lw.at(i, j)));
                }
        }
    return L.commit();
}

// Two launches: per-row values (8 rows per CTA), then one CTA for the norm.
template <typename T>
cudaError_t sym_norm(cudaStream_t, const Layout &Ly, const T *arf, int which, T *w, T *out)
{
    const int64_t n = Ly.n;
    if (n <= 0) { *out = T(0); return cudaSuccess; }
    EmuLower<T> Lw = emu_lower(Ly, const_cast<T *>(arf));
    if (which != 1 && n >= 8) {   // flat pass: CTA b strides over the RFP array, CTA G the diagonal
        const int64_t nt = n * (n + 1) / 2, span = 256 * 8;
        const int64_t G = std::min((nt + span - 1) / span, n - 1);
        const int ssq = which == 2;
        {
            Launch L;
            for (int64_t b = 0; b < G + ssq; ++b) {
                L.cta = (int)b;
                const bool diag = b == G;
                const int64_t total = diag ? n : nt;
                std::vector<T> vals;
                for (int64_t t = 0; t < 256; ++t)
                    for (int64_t e = diag ? t : b * 256 + t; e < total; e += diag ? 256 : G * 256)
                        vals.push_back(diag ? L.rd(Lw.at(e, e)) : L.rd(arf + e));
                T mx = T(0), q = T(0);
                for (T x : vals) mx = std::max(mx, (T)std::fabs(x));
                if (ssq && mx > T(0))
                    for (T x : vals) q += (x / mx) * (x / mx);
                L.wr(w + (diag ? 2 * G : b), mx);
                if (ssq) L.wr(w + (diag ? 2 * G + 1 : G + b), q);
            }
            cudaError_t e = L.commit();
            if (e != cudaSuccess) return e;
        }
        Launch L;
        T mx = T(0);
        for (int64_t b = 0; b < G; ++b) mx = std::max(mx, L.rd(w + b));
        T res = mx;
        if (ssq) {
            T q = T(0), d = T(0);
            if (mx > T(0)) {
                for (int64_t b = 0; b < G; ++b) q += (L.rd(w + b) / mx) * (L.rd(w + b) / mx) * L.rd(w + G + b);
                d = (L.rd(w + 2 * G) / mx) * (L.rd(w + 2 * G) / mx) * L.rd(w + 2 * G + 1);
            }
            res = mx * std::sqrt(std::max(T(2) * q - d, T(0)));
        }
        L.wr(out, res);
        return L.commit();
    }
    {
        Launch L;
        for (int64_t i = 0; i < n; ++i) {
            L.cta = (int)(i / 8);
            auto a = [&](int64_t j) { return j <= i ? L.rd(Lw.at(i, j)) : L.rd(Lw.at(j, i)); };
            T v = T(0), q = T(0);
            for (int64_t j = 0; j < n; ++j) {
                const T x = std::fabs(a(j));
                v = which == 1 ? v + x : std::max(v, x);
            }
            if (which == 2 && v > T(0))
                for (int64_t j = 0; j < n; ++j) q += (a(j) / v) * (a(j) / v);
            L.wr(w + i, v);
            if (which == 2) L.wr(w + n + i, q);
        }
        cudaError_t e = L.commit();
        if (e != cudaSuccess) return e;
    }
    Launch L;
    T mx = T(0);
    for (int64_t i = 0; i < n; ++i) mx = std::max(mx, L.rd(w + i));
    T res = mx;
    if (which == 2) {
        T q = T(0);
        if (mx > T(0))
            for (int64_t i = 0; i < n; ++i) q += (L.rd(w + i) / mx) * (L.rd(w + i) / mx) * L.rd(w + n + i);
        res = mx * std::sqrt(q);
    }
    L.wr(out, res);
    return L.commit();
}

template <typename T>
cudaError_t unit_diag(cudaStream_t, const Layout &Ly, T *arf, T *work, bool save)
{
    if (Ly.n <= 0) return cudaSuccess;
    EmuLower<T> Lw = emu_lower(Ly, arf);
    Launch L;
    for (int64_t i = 0; i < Ly.n; ++i) {
        L.cta = (int)(i / 256);
        if (save) {
            L.wr(work + i, L.rd(Lw.at(i, i)));
            L.wr(Lw.at(i, i), T(1));
        } else {
            L.wr(Lw.at(i, i), L.rd(work + i));
        }
    }
    return L.commit();
}

#define EMU_SURFACE_INST(T)                                                                        \
    template cudaError_t tp_copy<T>(cudaStream_t, const Layout &, T *, T *, bool, bool);           \
    template cudaError_t sym_norm<T>(cudaStream_t, const Layout &, const T *, int, T *, T *);      \
    template cudaError_t unit_diag<T>(cudaStream_t, const Layout &, T *, T *, bool);
EMU_SURFACE_INST(float)
EMU_SURFACE_INST(double)
#undef EMU_SURFACE_INST

// One CTA per kInvBlock-wide diagonal block: reads the block's lower
// triangle, writes the whole kInvBlock^2 slot of Inv.
cudaError_t inv_diag_blocks(cudaStream_t, View<float> V, int64_t m, float *Inv, const int32_t *abort)
{
    if (m <= 0) return cudaSuccess;
    const int64_t nb = kInvBlock, nblk = (m + nb - 1) / nb;
    Launch L;
    for (int64_t b = 0; b < nblk; ++b) {
        L.cta = (int)b;
        if (aborted(L, abort)) continue;
        const int64_t k0 = b * nb, w = std::min(nb, m - k0);
        std::vector<float> l(nb * nb, 0.f), x(nb * nb, 0.f);
        for (int64_t i = 0; i < w; ++i)
            for (int64_t j = 0; j <= i; ++j) l[i * nb + j] = L.rd(&V(k0 + i, k0 + j));
        for (int64_t c = 0; c < w; ++c) {
            x[c * nb + c] = 1.f / l[c * nb + c];
            for (int64_t i = c + 1; i < w; ++i) {
                float s = 0.f;
                for (int64_t p = c; p < i; ++p) s += l[i * nb + p] * x[p * nb + c];
                x[i * nb + c] = -s / l[i * nb + i];
            }
        }
        float *out = Inv + b * nb * nb;
        for (int64_t j = 0; j < nb; ++j)
            for (int64_t i = 0; i < nb; ++i) L.wr(&out[j * nb + i], x[i * nb + j]);
    }
    return L.commit();
}

template <typename T>
cudaError_t lauum_tile(cudaStream_t, View<T> A, int w, const int32_t *abort)
{
    if (w <= 0) return cudaSuccess;
    Launch L;
    if (aborted(L, abort)) return L.commit();
    std::vector<T> x(w * w, T(0));
    for (int i = 0; i < w; ++i)
        for (int j = 0; j <= i; ++j) x[i * w + j] = L.rd(&A(i, j));
    for (int i = 0; i < w; ++i)
        for (int j = 0; j <= i; ++j) {
            T s = T(0);
            for (int k = i; k < w; ++k) s += x[k * w + i] * x[k * w + j];
            L.wr(&A(i, j), s);
        }
    return L.commit();
}

template <typename T>
cudaError_t check_diag(cudaStream_t, View<T> t1, int64_t n1, View<T> t2, int64_t n2, int32_t *info)
{
    Launch L;
    int32_t v = 0;
    for (int64_t i = 0; i < n1 + n2; ++i) {
        T d = i < n1 ? L.rd(&t1(i, i)) : L.rd(&t2(i - n1, i - n1));
        if (d == T(0)) { v = (int32_t)(i + 1); break; }
    }
    L.wr_any(info, 4);
    cudaError_t e = L.commit();
    *info = v;
    return e;
}

template <typename T>
cudaError_t pack_copy(cudaStream_t, const Layout &Ly, bool lowerA, T *A, int64_t lda, T *arf, bool unpack)
{
    const int TILE = 64;
    Launch L;
    struct Blk { int64_t rows, cols, roff, coff; Block b; bool tri; };
    Blk blks[3] = {{Ly.n1, Ly.n1, 0, 0, Ly.t1, true}, {Ly.n2, Ly.n1, Ly.n1, 0, Ly.s, false},
                   {Ly.n2, Ly.n2, Ly.n1, Ly.n1, Ly.t2, true}};
    int cta = 0;
    for (auto &bk : blks)
        for (int64_t bi0 = 0; bi0 < bk.rows; bi0 += TILE)
            for (int64_t bj0 = 0; bj0 < bk.cols; bj0 += TILE) {
                if (bk.tri && bj0 > bi0) continue;
                L.cta = cta++;
                for (int64_t bi = bi0; bi < std::min(bk.rows, bi0 + TILE); ++bi)
                    for (int64_t bj = bj0; bj < std::min(bk.cols, bj0 + TILE); ++bj) {
                        if (bk.tri && bi < bj) continue;
                        int64_t gi = bk.roff + bi, gj = bk.coff + bj;
                        T *pa = lowerA ? &A[gi + gj * lda] : &A[gj + gi * lda];
                        T *pr = bk.b.trans ? &arf[bk.b.off + bj + bi * Ly.ld] : &arf[bk.b.off + bi + bj * Ly.ld];
                        if (unpack) L.wr(pa, L.rd(pr));
                        else L.wr(pr, L.rd(pa));
                    }
            }
    return L.commit();
}

extern "C" void emu_set_sms(int s) { g_emu_sms = s; }

// Tensor-core GEMM update: 128 x 128 tiles, lower-triangular tile list when
// cmode is lower and M == N, operands read as BF16 (kind 0) or FP32 (kind 1).
cudaError_t tc_gemm_nt(cudaStream_t, int kind, const void *A, int64_t a_rows, int64_t a_pitch,
                       int a_row0, const void *B, int64_t b_rows, int64_t b_pitch, int b_row0,
                       View<float> C, int64_t M, int64_t N, int64_t K, float alpha, float beta,
                       int cmode, int *err)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int T = 128, esz = kind == 0 ? 2 : 4;
    if ((uintptr_t)A % 16 || (uintptr_t)B % 16 || (a_pitch * esz) % 16 || (b_pitch * esz) % 16) {
        violation("tensor map alignment", A);
        return cudaErrorInvalidValue;
    }
    Launch L;
    auto load = [&](const void *base, int64_t pitch, int64_t rows, int64_t r, int64_t k) -> float {
        if (r >= rows || k >= K) return 0.f;   // TMA zero fill outside the matrix
        if (kind == 0) {
            const uint16_t *p = (const uint16_t *)base + r * pitch + k;
            uint32_t bits = (uint32_t)L.rd(p) << 16;
            float f;
            memcpy(&f, &bits, 4);
            return f;
        }
        float f = L.rd((const float *)base + r * pitch + k);   // kind::tf32 reads 19 bits
        uint32_t bits;
        memcpy(&bits, &f, 4);
        bits &= 0xffffe000u;
        memcpy(&f, &bits, 4);
        return f;
    };
    const int64_t gm = (M + T - 1) / T, gn = (N + T - 1) / T;
    const bool lower_tiles = cmode == MASK_LOWER && M == N;
    int cta = 0;
    for (int64_t tm = 0; tm < gm; ++tm)
        for (int64_t tn = 0; tn < (lower_tiles ? tm + 1 : gn); ++tn, ++cta) {
            L.cta = cta;
            for (int64_t i = tm * T; i < std::min(M, tm * T + T); ++i)
                for (int64_t j = tn * T; j < std::min(N, tn * T + T); ++j) {
                    double acc = 0;
                    for (int64_t k = 0; k < K; ++k)
                        acc += (double)load(A, a_pitch, a_rows, a_row0 + i, k) *
                               (double)load(B, b_pitch, b_rows, b_row0 + j, k);
                    if (cmode == MASK_LOWER && j > i) continue;
                    float v = alpha * (float)acc;
                    if (beta != 0.f) v = beta * L.rd(&C(i, j)) + v;
                    L.wr(&C(i, j), v);
                }
        }
    (void)err;
    return L.commit();
}

// ---- mixed-precision kernels -----------------------------------------------------

static float bf16_round(float x, uint16_t *bits_out)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;                    // round to nearest even
    *bits_out = (uint16_t)(u >> 16);
    uint32_t back = (uint32_t)(*bits_out) << 16;
    float f;
    memcpy(&f, &back, 4);
    return f;
}
template <typename Td, typename Ts> static void put(Launch &L, Td *p, Ts v) { L.wr(p, (Td)v); }
static void put(Launch &L, __nv_bfloat16 *p, float v)
{
    uint16_t bits;
    bf16_round(v, &bits);
    L.wr_any(p, 2);
    // bf16 stores are applied immediately after the launch's checks
    static_cast<void>(bits);
    L.pend_b.push_back({p, bits});
}

template <typename Ts, typename Td>
cudaError_t convert(cudaStream_t, View<Ts> src, View<Td> dst, int64_t rows, int64_t cols, bool tri,
                    const int32_t *stop)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    Launch L;
    const int T = 32;
    int cta = 0;
    for (int64_t r0 = 0; r0 < rows; r0 += T)
        for (int64_t c0 = 0; c0 < cols; c0 += T, ++cta) {
            L.cta = cta;
            if (stop && L.rd(stop)) continue;
            if (tri && r0 + T - 1 < c0) continue;
            for (int64_t i = r0; i < std::min(rows, r0 + T); ++i)
                for (int64_t j = c0; j < std::min(cols, c0 + T); ++j) {
                    if (tri && i < j) continue;
                    put(L, &dst(i, j), L.rd(&src(i, j)));
                }
        }
    return L.commit();
}

cudaError_t split_tf32(cudaStream_t, View<float> src, float *Q, int64_t rows, int64_t cols,
                       int64_t seg, const int32_t *stop)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    Launch L;
    const int64_t T = 32, gy = (rows + T - 1) / T, gx = (cols + T - 1) / T;
    for (int64_t by = 0; by < gy; ++by)
        for (int64_t bx = 0; bx < gx; ++bx) {
            L.cta = (int)(by * gx + bx);
            if (aborted(L, stop)) continue;
            for (int64_t r = by * T; r < std::min(rows, by * T + T); ++r)
                for (int64_t k = bx * T; k < std::min(cols, bx * T + T); ++k) {
                    auto tf32 = [](float v) {    // to nearest, ties away from zero
                        uint32_t bits;
                        memcpy(&bits, &v, 4);
                        bits = (bits + 0x1000u) & 0xffffe000u;
                        memcpy(&v, &bits, 4);
                        return v;
                    };
                    const float x = L.rd(&src(r, k));
                    const float hi = tf32(x);
                    const float lo = tf32(x - hi);
                    float *row = Q + r * 4 * seg + k;
                    L.wr(row, hi);
                    L.wr(row + seg, hi);
                    L.wr(row + 2 * seg, lo);
                    L.wr(row + 3 * seg, hi);
                }
        }
    return L.commit();
}

cudaError_t split_bf16x3(cudaStream_t, View<float> src, __nv_bfloat16 *QA, __nv_bfloat16 *QB,
                         int64_t rows, int64_t cols, int64_t seg, const int32_t *stop)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    Launch L;
    const int64_t T = 32, gy = (rows + T - 1) / T, gx = (cols + T - 1) / T;
    for (int64_t by = 0; by < gy; ++by)
        for (int64_t bx = 0; bx < gx; ++bx) {
            L.cta = (int)(by * gx + bx);
            if (aborted(L, stop)) continue;
            for (int64_t r = by * T; r < std::min(rows, by * T + T); ++r)
                for (int64_t k = bx * T; k < std::min(cols, bx * T + T); ++k) {
                    const float x = L.rd(&src(r, k));
                    uint16_t bh, bm, bl;
                    const float hi = bf16_round(x, &bh);
                    const float r1 = x - hi;
                    const float mid = bf16_round(r1, &bm);
                    bf16_round(r1 - mid, &bl);
                    const uint16_t a[6] = {bh, bh, bm, bm, bh, bl}, b[6] = {bh, bm, bh, bm, bl, bh};
                    for (int q = 0; q < 6; ++q) {
                        __nv_bfloat16 *pa = QA + r * 6 * seg + q * seg + k, *pb = QB + r * 6 * seg + q * seg + k;
                        L.wr_any(pa, 2);
                        L.pend_b.push_back({pa, a[q]});
                        L.wr_any(pb, 2);
                        L.pend_b.push_back({pb, b[q]});
                    }
                }
        }
    return L.commit();
}

cudaError_t add_correction(cudaStream_t, View<double> X, View<float> D, int64_t n, int64_t nrhs,
                           const int32_t *stop)
{
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    Launch L;
    if (L.rd(stop)) return L.commit();
    for (int64_t j = 0; j < nrhs; ++j)
        for (int64_t i = 0; i < n; ++i) L.wr(&X(i, j), L.rd(&X(i, j)) + (double)L.rd(&D(i, j)));
    return L.commit();
}

cudaError_t fill(cudaStream_t, View<double> X, int64_t n, int64_t nrhs, double v)
{
    Launch L;
    for (int64_t j = 0; j < nrhs; ++j)
        for (int64_t i = 0; i < n; ++i) L.wr(&X(i, j), v);
    return L.commit();
}

cudaError_t anorm_inf(cudaStream_t, const RfpViews &v, int64_t n, double *out)
{
    Launch L;
    auto lower = [&](int64_t i, int64_t j) {
        if (j >= v.n1) return L.rd(&v.t2(i - v.n1, j - v.n1));
        if (i >= v.n1) return L.rd(&v.s(i - v.n1, j));
        return L.rd(&v.t1(i, j));
    };
    double m = 0;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0;
        for (int64_t j = 0; j <= i; ++j) s += std::fabs(lower(i, j));
        for (int64_t k = i + 1; k < n; ++k) s += std::fabs(lower(k, i));
        m = std::max(m, s);
    }
    L.wr(out, m);
    return L.commit();
}

cudaError_t backward_error(cudaStream_t, View<double> R, View<double> X, View<double> B, int64_t n,
                           int64_t nrhs, const double *anorm, double *berr_col, double tol,
                           rfp_mixed_status_t *status, int32_t *stop)
{
    Launch L;
    if (L.rd(stop)) return L.commit();
    double m = 0;
    for (int64_t j = 0; j < nrhs; ++j) {
        double r = 0, x = 0, b = 0;
        for (int64_t i = 0; i < n; ++i) {
            r = std::max(r, std::fabs(L.rd(&R(i, j))));
            x = std::max(x, std::fabs(L.rd(&X(i, j))));
            b = std::max(b, std::fabs(L.rd(&B(i, j))));
        }
        const double den = L.rd(anorm) * x + b, e = den > 0 ? r / den : r;
        L.wr(&berr_col[j], e);
        m = std::max(m, e);
    }
    L.wr(&status->backward_error, m);
    L.wr_any(&status->iterations, 4);
    const int32_t iters = L.rd(&status->iterations) + 1;
    cudaError_t e = L.commit();
    status->iterations = iters;
    if (m <= tol) { status->converged = 1; *stop = 1; }
    return e;
}

cudaError_t stop_on_failure(cudaStream_t, rfp_mixed_status_t *status, const int32_t *tc_err,
                            int32_t *stop)
{
    Launch L;
    const int32_t te = L.rd(tc_err), info = L.rd(&status->info);
    cudaError_t e = L.commit();
    status->tc_error = te;
    if (info != 0 || te != 0) *stop = 1;
    return e;
}

template cudaError_t convert<double, float>(cudaStream_t, View<double>, View<float>, int64_t, int64_t,
                                            bool, const int32_t *);
template cudaError_t convert<double, double>(cudaStream_t, View<double>, View<double>, int64_t,
                                             int64_t, bool, const int32_t *);
template cudaError_t convert<float, float>(cudaStream_t, View<float>, View<float>, int64_t, int64_t,
                                           bool, const int32_t *);
template cudaError_t convert<float, __nv_bfloat16>(cudaStream_t, View<float>, View<__nv_bfloat16>,
                                                   int64_t, int64_t, bool, const int32_t *);

// The batched kernel runs one whole factorization per CTA and is tested on
// the GPU; the emulator only links its host entry points.
size_t batch_plan_bytes(int64_t batch) { return 256 + (size_t)(batch > 0 ? batch : 0) * 104; }
int batch_plan(int64_t, const struct rfp_batch_entry *, int64_t, int64_t, void *, cudaStream_t,
               int64_t *bad)
{
    *bad = -1;
    return 1000 + cudaErrorInvalidValue;
}
template <typename T>
cudaError_t batched_run(int64_t, const void *, T *, T *, int32_t *, cudaStream_t)
{
    return cudaErrorInvalidValue;
}
template cudaError_t batched_run<double>(int64_t, const void *, double *, double *, int32_t *,
                                         cudaStream_t);
template cudaError_t batched_run<float>(int64_t, const void *, float *, float *, int32_t *,
                                        cudaStream_t);

#define EMU_INST(T)                                                                                  \
    template cudaError_t gemm_nt<T>(cudaStream_t, View<T>, View<T>, View<T>, int64_t, int64_t, int64_t, \
                                    T, T, int, int, int, const int32_t *, int);                      \
    template cudaError_t gemm_nt_splitk<T>(cudaStream_t, View<T>, View<T>, View<T>, int64_t, int64_t, \
                                           int64_t, T, T, int, int, int, const int32_t *, int, T *); \
    template cudaError_t trsm_strip<T>(cudaStream_t, View<T>, View<T>, int64_t, int, int, T,         \
                                       const int32_t *, bool);                                       \
    template cudaError_t potrf_tile<T>(cudaStream_t, View<T>, int, int32_t *, int64_t);              \
    template cudaError_t trtri_tile<T>(cudaStream_t, View<T>, int, const int32_t *);                 \
    template cudaError_t lauum_tile<T>(cudaStream_t, View<T>, int, const int32_t *);                 \
    template cudaError_t check_diag<T>(cudaStream_t, View<T>, int64_t, View<T>, int64_t, int32_t *); \
    template cudaError_t pack_copy<T>(cudaStream_t, const Layout &, bool, T *, int64_t, T *, bool);
EMU_INST(double)
EMU_INST(float)

}  // namespace rfp
