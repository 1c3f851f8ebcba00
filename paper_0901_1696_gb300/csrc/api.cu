// extern "C" entry points declared in include/rfp.h: argument checks on the
// host (LAPACK convention: -i for argument i), then the enqueued kernels.
#include <atomic>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/rfp.h"
#include "mixed_internal.cuh"
#include "rfp_internal.cuh"

namespace rfp {

// Placement of T1 (L11), S (L21) and T2 (L22) for the eight layouts.  For
// TRANSR='N' each block starts at row r0, column c0 of A_R (LDAR rows,
// column-major) and is stored as drawn in Figs. 4-6:
//   lower, odd : T1 (0,0) as is;  S (n1,0) as is;   T2 (0,1) transposed (L22^T)
//   lower, even: T1 (1,0);        S (k+1,0);        T2 (0,0) transposed
//   upper, odd : T1 (n2,0) (=U11^T); S (0,0) transposed (=U12); T2 (n1,0) transposed (=U22)
//   upper, even: T1 (k+1,0);      S (0,0) transposed; T2 (k,0) transposed
// TRANSR='T' stores A_R^T (ld = ceil(N/2)): row and column swap roles and
// every block flips its transposition.
bool make_layout(char transr, char uplo, int64_t n, Layout *out)
{
    const bool lower = (uplo == 'L' || uplo == 'l');
    const bool trans = (transr == 'T' || transr == 't');
    const int64_t n1 = lower ? (n + 1) / 2 : n / 2, n2 = n - n1;
    const bool odd = (n % 2) == 1;
    const int64_t ldar = odd ? n : n + 1, nc = (n + 1) / 2, k = n / 2;
    struct RC { int64_t r0, c0; int tr; } b1, bs, b2;
    if (lower) {
        if (odd) { b1 = {0, 0, 0}; bs = {n1, 0, 0}; b2 = {0, 1, 1}; }
        else { b1 = {1, 0, 0}; bs = {k + 1, 0, 0}; b2 = {0, 0, 1}; }
    } else {
        if (odd) { b1 = {n2, 0, 0}; bs = {0, 0, 1}; b2 = {n1, 0, 1}; }
        else { b1 = {k + 1, 0, 0}; bs = {0, 0, 1}; b2 = {k, 0, 1}; }
    }
    auto place = [&](RC x) -> Block {
        if (!trans) return Block{x.r0 + x.c0 * ldar, x.tr};
        return Block{x.c0 + x.r0 * nc, x.tr ? 0 : 1};
    };
    out->n = n; out->n1 = n1; out->n2 = n2;
    out->ld = trans ? nc : ldar;
    out->t1 = place(b1); out->s = place(bs); out->t2 = place(b2);
    return true;
}

// ---- instrumentation ------------------------------------------------------------

namespace {
std::atomic<int64_t> g_launch_count{0};
constexpr size_t kMaxEvents = 8192;
// Step timing history of one host thread: events[i] closes the step named
// names[i]; an entry with a null name opens a new routine call.
struct StageLog {
    bool enabled = false;
    std::vector<cudaEvent_t> pool;      // created lazily, reused across enables
    std::vector<const char *> names;    // one per recorded event
};
thread_local StageLog g_stages;

void stage_record(cudaStream_t st, const char *name)
{
    StageLog &g = g_stages;
    if (!g.enabled || g.names.size() >= kMaxEvents) return;
    if (g.names.size() == g.pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        g.pool.push_back(e);
    }
    cudaEventRecord(g.pool[g.names.size()], st);
    g.names.push_back(name);
}
}  // namespace

void note_launch() { g_launch_count.fetch_add(1, std::memory_order_relaxed); }
void stage_begin(cudaStream_t st) { stage_record(st, nullptr); }
void stage_mark(cudaStream_t st, const char *name)
{
    if (!g_stages.names.empty()) stage_record(st, name);
}

}  // namespace rfp

namespace {

thread_local const char *g_last_cuda_error = "no error";

bool valid_transr(char c) { return c == 'N' || c == 'n' || c == 'T' || c == 't'; }
bool valid_uplo(char c) { return c == 'L' || c == 'l' || c == 'U' || c == 'u'; }
bool is_lower(char c) { return c == 'L' || c == 'l'; }
constexpr int64_t kMaxN = int64_t(1) << 24;   // n(n+1)/2 and tile counts stay far from overflow

template <typename T>
bool aligned(const T *p) { return (reinterpret_cast<uintptr_t>(p) % alignof(T)) == 0; }

int finish(cudaError_t e)
{
    if (e == cudaSuccess) return RFP_OK;
    g_last_cuda_error = cudaGetErrorName(e);
    return RFP_ERR_CUDA;
}

}  // namespace

namespace rfp {

int finish_cuda(cudaError_t e) { return finish(e); }

int mixed_check_args(char transr, char uplo, int64_t n, int64_t nrhs, const double *arf,
                     const double *B, int64_t ldb, const double *X, int64_t ldx, int prec,
                     int max_iter, double tol, const rfp_mixed_status_t *status)
{
    if (!valid_transr(transr)) return -1;
    if (!valid_uplo(uplo)) return -2;
    if (n < 0 || n > kMaxN || n > (int64_t(1) << 31) - 1) return -3;
    if (nrhs < 0 || nrhs > (int64_t(1) << 31) - 1) return -4;
    if (prec < RFP_PREC_BF16 || prec > RFP_PREC_BF16X6) return -10;
    if (max_iter < 0) return -11;
    if (!(tol >= 0.0)) return -12;
    if (!status || !aligned(status)) return -15;
    if (n == 0 || nrhs == 0) return 0;
    if (!arf || !aligned(arf)) return -5;
    if (!B || !aligned(B)) return -6;
    if (ldb < n) return -7;
    if (!X || !aligned(X)) return -8;
    if (ldx < n) return -9;
    return 0;
}

}  // namespace rfp

namespace {

template <typename T>
int pack_entry(char transr, char uplo, int64_t n, T *A, int64_t lda, T *arf, void *stream,
               bool unpack)
{
    // argument numbering differs: pack (A=4, lda=5, arf=6), unpack (arf=4, A=5, lda=6)
    if (!valid_transr(transr)) return -1;
    if (!valid_uplo(uplo)) return -2;
    if (n < 0 || n > kMaxN) return -3;
    if (n == 0) return RFP_OK;
    const int argA = unpack ? 5 : 4, argLda = unpack ? 6 : 5, argArf = unpack ? 4 : 6;
    if (unpack) {
        if (!arf || !aligned(arf)) return -argArf;
        if (!A || !aligned(A)) return -argA;
    } else {
        if (!A || !aligned(A)) return -argA;
    }
    if (lda < (n > 1 ? n : 1)) return -argLda;
    if (!unpack && (!arf || !aligned(arf))) return -argArf;
    rfp::Layout L;
    rfp::make_layout(transr, uplo, n, &L);
    return finish(rfp::pack_copy<T>((cudaStream_t)stream, L, is_lower(uplo), A, lda, arf, unpack));
}

template <typename T>
int pftrf_entry(char transr, char uplo, int64_t n, T *arf, int32_t *info, void *stream)
{
    if (!valid_transr(transr)) return -1;
    if (!valid_uplo(uplo)) return -2;
    if (n < 0 || n > kMaxN) return -3;
    if (n > 0 && (!arf || !aligned(arf))) return -4;
    if (!info || !aligned(info)) return -5;
    if (n == 0) return finish(cudaMemsetAsync(info, 0, sizeof(int32_t), (cudaStream_t)stream));
    rfp::Layout L;
    rfp::make_layout(transr, uplo, n, &L);
    return finish(rfp::pftrf_impl<T>((cudaStream_t)stream, L, arf, info));
}

template <typename T>
int pftrs_entry(char transr, char uplo, int64_t n, int64_t nrhs, const T *arf, T *B, int64_t ldb,
                void *stream)
{
    if (!valid_transr(transr)) return -1;
    if (!valid_uplo(uplo)) return -2;
    if (n < 0 || n > kMaxN) return -3;
    if (nrhs < 0 || nrhs > (int64_t(1) << 31) - 1) return -4;
    if (n == 0 || nrhs == 0) return RFP_OK;
    if (!arf || !aligned(arf)) return -5;
    if (!B || !aligned(B)) return -6;
    if (ldb < (n > 1 ? n : 1)) return -7;
    rfp::Layout L;
    rfp::make_layout(transr, uplo, n, &L);
    return finish(rfp::pftrs_impl<T>((cudaStream_t)stream, L, arf, B, ldb, nrhs));
}

template <typename T>
int pftri_entry(char transr, char uplo, int64_t n, T *arf, int32_t *info, void *stream)
{
    if (!valid_transr(transr)) return -1;
    if (!valid_uplo(uplo)) return -2;
    if (n < 0 || n > kMaxN) return -3;
    if (n > 0 && (!arf || !aligned(arf))) return -4;
    if (!info || !aligned(info)) return -5;
    if (n == 0) return finish(cudaMemsetAsync(info, 0, sizeof(int32_t), (cudaStream_t)stream));
    rfp::Layout L;
    rfp::make_layout(transr, uplo, n, &L);
    return finish(rfp::pftri_impl<T>((cudaStream_t)stream, L, arf, info));
}

bool is_trans(char c) { return c == 'T' || c == 't'; }
bool valid_trans(char c) { return c == 'N' || c == 'n' || is_trans(c); }
bool valid_diag(char c) { return c == 'N' || c == 'n' || c == 'U' || c == 'u'; }
bool is_unit(char c) { return c == 'U' || c == 'u'; }

template <typename T>
int tp_entry(char transr, char uplo, int64_t n, T *src, T *dst, void *stream, bool to_rfp)
{
    if (!valid_transr(transr)) return -1;
    if (!valid_uplo(uplo)) return -2;
    if (n < 0 || n > kMaxN) return -3;
    if (n == 0) return RFP_OK;
    if (!src || !aligned(src)) return -4;
    if (!dst || !aligned(dst)) return -5;
    rfp::Layout L;
    rfp::make_layout(transr, uplo, n, &L);
    // to_rfp: src = AP, dst = ARF; else src = ARF, dst = AP
    return finish(rfp::tp_copy<T>((cudaStream_t)stream, L, to_rfp ? dst : src, to_rfp ? src : dst,
                                  is_lower(uplo), to_rfp));
}

template <typename T>
int tftri_entry(char transr, char uplo, char diag, int64_t n, T *arf, int32_t *info, T *work,
                void *stream)
{
    if (!valid_transr(transr)) return -1;
    if (!valid_uplo(uplo)) return -2;
    if (!valid_diag(diag)) return -3;
    if (n < 0 || n > kMaxN) return -4;
    if (n > 0 && (!arf || !aligned(arf))) return -5;
    if (!info || !aligned(info)) return -6;
    if (n > 0 && is_unit(diag) && (!work || !aligned(work))) return -7;
    if (n == 0) return finish(cudaMemsetAsync(info, 0, sizeof(int32_t), (cudaStream_t)stream));
    rfp::Layout L;
    rfp::make_layout(transr, uplo, n, &L);
    cudaStream_t st = (cudaStream_t)stream;
    if (!is_unit(diag)) return finish(rfp::tftri_impl<T>(st, L, arf, info));
    cudaError_t e = rfp::unit_diag<T>(st, L, arf, work, true);
    if (e == cudaSuccess) e = rfp::tftri_impl<T>(st, L, arf, info);
    if (e == cudaSuccess) e = rfp::unit_diag<T>(st, L, arf, work, false);
    return finish(e);
}

template <typename T>
int sfrk_entry(char transr, char uplo, char trans, int64_t n, int64_t k, T alpha, const T *A,
               int64_t lda, T beta, T *C, void *stream)
{
    if (!valid_transr(transr)) return -1;
    if (!valid_uplo(uplo)) return -2;
    if (!valid_trans(trans)) return -3;
    if (n < 0 || n > kMaxN) return -4;
    if (k < 0 || k > (int64_t(1) << 40)) return -5;
    const bool use_a = n > 0 && k > 0 && alpha != T(0);
    if (use_a && (!A || !aligned(A))) return -7;
    const int64_t rows = is_trans(trans) ? k : n;
    if (lda < (rows > 1 ? rows : 1)) return -8;
    if (n > 0 && (!C || !aligned(C))) return -10;
    if (n == 0 || ((!use_a) && beta == T(1))) return RFP_OK;
    rfp::Layout L;
    rfp::make_layout(transr, uplo, n, &L);
    T *a = const_cast<T *>(A);   // read only
    // op(A) as an n x k view: A (n x k, lda) or A^T (A k x n, lda)
    rfp::View<T> opA = is_trans(trans) ? rfp::View<T>{a, lda, 1} : rfp::View<T>{a, 1, lda};
    const int64_t kk = use_a ? k : 0;
    return finish(rfp::sfrk_impl<T>((cudaStream_t)stream, L, C, opA, kk, use_a ? alpha : T(0), beta));
}

template <typename T>
int tfsm_entry(char transr, char side, char uplo, char trans, char diag, int64_t m, int64_t n,
               T alpha, const T *arf, T *B, int64_t ldb, void *stream)
{
    if (!valid_transr(transr)) return -1;
    const bool left = side == 'L' || side == 'l';
    if (!left && side != 'R' && side != 'r') return -2;
    if (!valid_uplo(uplo)) return -3;
    if (!valid_trans(trans)) return -4;
    if (!valid_diag(diag)) return -5;
    if (m < 0 || m > kMaxN) return -6;
    if (n < 0 || n > kMaxN) return -7;
    if (m == 0 || n == 0) return RFP_OK;
    if (alpha != T(0) && (!arf || !aligned(arf))) return -9;
    if (!B || !aligned(B)) return -10;
    if (ldb < (m > 1 ? m : 1)) return -11;
    rfp::Layout L;
    rfp::make_layout(transr, uplo, left ? m : n, &L);
    // op(A) in terms of the logical lower L: UPLO 'L' stores L, 'U' stores L^T
    const bool opT = is_lower(uplo) ? is_trans(trans) : !is_trans(trans);
    return finish(rfp::tfsm_impl<T>((cudaStream_t)stream, L, arf, left, opT, is_unit(diag), m, n,
                                    alpha, B, ldb));
}

template <typename T>
int lansf_entry(char norm, char transr, char uplo, int64_t n, const T *arf, T *work, T *value,
                void *stream)
{
    int which;
    switch (norm) {
    case 'M': case 'm': which = 0; break;
    case '1': case 'O': case 'o': case 'I': case 'i': which = 1; break;
    case 'F': case 'f': case 'E': case 'e': which = 2; break;
    default: return -1;
    }
    if (!valid_transr(transr)) return -2;
    if (!valid_uplo(uplo)) return -3;
    if (n < 0 || n > kMaxN) return -4;
    if (n > 0 && (!arf || !aligned(arf))) return -5;
    if (n > 0 && (!work || !aligned(work))) return -6;
    if (!value || !aligned(value)) return -7;
    rfp::Layout L;
    rfp::make_layout(transr, uplo, n, &L);
    return finish(rfp::sym_norm<T>((cudaStream_t)stream, L, arf, which, work, value));
}

template <typename T>
int batched_entry(int64_t batch, const void *d_plan, T *arf, T *B, int32_t *d_info, void *stream)
{
    if (batch < 0 || batch > (int64_t(1) << 31) - 1) return -1;
    if (batch == 0) return RFP_OK;
    if (!d_plan || (reinterpret_cast<uintptr_t>(d_plan) % 256)) return -2;
    if (!arf || !aligned(arf)) return -3;
    if (B && !aligned(B)) return -4;
    if (!d_info || !aligned(d_info)) return -5;
    return finish(rfp::batched_run<T>(batch, d_plan, arf, B, d_info, (cudaStream_t)stream));
}

}  // namespace

extern "C" {

int rfp_layout(char transr, char uplo, int64_t n, rfp_layout_t *out)
{
    if (!valid_transr(transr)) return -1;
    if (!valid_uplo(uplo)) return -2;
    if (n < 0 || n > kMaxN) return -3;
    if (!out) return -4;
    rfp::Layout L;
    rfp::make_layout(transr, uplo, n, &L);
    out->n = L.n; out->n1 = L.n1; out->n2 = L.n2; out->ld = L.ld;
    out->t1_off = L.t1.off; out->s_off = L.s.off; out->t2_off = L.t2.off;
    out->t1_trans = L.t1.trans; out->s_trans = L.s.trans; out->t2_trans = L.t2.trans;
    return RFP_OK;
}

int rfp_dpack(char transr, char uplo, int64_t n, const double *A, int64_t lda, double *arf,
              void *stream)
{
    return pack_entry<double>(transr, uplo, n, const_cast<double *>(A), lda, arf, stream, false);
}
int rfp_spack(char transr, char uplo, int64_t n, const float *A, int64_t lda, float *arf,
              void *stream)
{
    return pack_entry<float>(transr, uplo, n, const_cast<float *>(A), lda, arf, stream, false);
}
int rfp_dunpack(char transr, char uplo, int64_t n, const double *arf, double *A, int64_t lda,
                void *stream)
{
    return pack_entry<double>(transr, uplo, n, A, lda, const_cast<double *>(arf), stream, true);
}
int rfp_sunpack(char transr, char uplo, int64_t n, const float *arf, float *A, int64_t lda,
                void *stream)
{
    return pack_entry<float>(transr, uplo, n, A, lda, const_cast<float *>(arf), stream, true);
}

int rfp_dpftrf(char transr, char uplo, int64_t n, double *arf, int32_t *info, void *stream)
{
    return pftrf_entry<double>(transr, uplo, n, arf, info, stream);
}
int rfp_spftrf(char transr, char uplo, int64_t n, float *arf, int32_t *info, void *stream)
{
    return pftrf_entry<float>(transr, uplo, n, arf, info, stream);
}
int rfp_dpftrs(char transr, char uplo, int64_t n, int64_t nrhs, const double *arf, double *B,
               int64_t ldb, void *stream)
{
    return pftrs_entry<double>(transr, uplo, n, nrhs, arf, B, ldb, stream);
}
int rfp_spftrs(char transr, char uplo, int64_t n, int64_t nrhs, const float *arf, float *B,
               int64_t ldb, void *stream)
{
    return pftrs_entry<float>(transr, uplo, n, nrhs, arf, B, ldb, stream);
}
int rfp_dpftri(char transr, char uplo, int64_t n, double *arf, int32_t *info, void *stream)
{
    return pftri_entry<double>(transr, uplo, n, arf, info, stream);
}
int rfp_spftri(char transr, char uplo, int64_t n, float *arf, int32_t *info, void *stream)
{
    return pftri_entry<float>(transr, uplo, n, arf, info, stream);
}

int rfp_ssyrk_tc(char uplo, int64_t n, int64_t k, float alpha, const void *A, int64_t lda,
                 int prec, float beta, float *C, int64_t ldc, int32_t *d_err, void *stream)
{
    if (uplo != 'L' && uplo != 'l') return -1;
    if (n < 0 || n > (int64_t(1) << 30)) return -2;
    if (k < 0 || k > (int64_t(1) << 30)) return -3;
    if (prec != RFP_PREC_BF16 && prec != RFP_PREC_TF32) return -7;
    const int esz = prec == RFP_PREC_BF16 ? 2 : 4;
    if (n == 0) return RFP_OK;
    if (!A || (reinterpret_cast<uintptr_t>(A) % 16)) return -5;
    if (lda < (k > 1 ? k : 1) || (lda * esz) % 16) return -6;
    if (!C || !aligned(C)) return -9;
    if (ldc < n) return -10;
    if (!d_err || !aligned(d_err)) return -11;
    rfp::View<float> Cv{C, 1, ldc};
    return finish(rfp::tc_gemm_nt((cudaStream_t)stream, prec, A, n, lda, 0, A, n, lda, 0, Cv, n,
                                  n, k, alpha, beta, rfp::MASK_LOWER, d_err));
}

size_t rfp_dpfsv_mixed_workspace(int64_t n, int64_t nrhs, int prec)
{
    if (n <= 0 || nrhs <= 0 || n > kMaxN) return 0;
    if (prec < RFP_PREC_BF16 || prec > RFP_PREC_BF16X6) return 0;
    return rfp::mixed_workspace_bytes(n, nrhs, prec);
}

int rfp_dpfsv_mixed(char transr, char uplo, int64_t n, int64_t nrhs, const double *arf,
                    const double *B, int64_t ldb, double *X, int64_t ldx, int prec, int max_iter,
                    double tol, void *work, size_t work_bytes, rfp_mixed_status_t *status,
                    void *stream)
{
    const int bad = rfp::mixed_check_args(transr, uplo, n, nrhs, arf, B, ldb, X, ldx, prec,
                                          max_iter, tol, status);
    if (bad) return bad;
    if (n == 0 || nrhs == 0)
        return finish(cudaMemsetAsync(status, 0, sizeof(rfp_mixed_status_t), (cudaStream_t)stream));
    rfp::MixedWork w;
    if (!work) return -13;
    if (!rfp::mixed_carve(work, work_bytes, n, nrhs, prec, &w))
        return (reinterpret_cast<uintptr_t>(work) % 256) ? -13 : -14;
    rfp::Layout L;
    rfp::make_layout(transr, uplo, n, &L);
    return finish(rfp::pfsv_mixed_impl((cudaStream_t)stream, L, arf, B, ldb, X, ldx, nrhs, prec,
                                       max_iter, tol, w, status));
}

size_t rfp_batch_plan_bytes(int64_t batch) { return rfp::batch_plan_bytes(batch); }

int rfp_batch_plan(int64_t batch, const rfp_batch_entry_t *h_entries, int64_t arf_len,
                   int64_t b_len, void *d_plan, size_t plan_bytes, int64_t *bad_entry,
                   void *stream)
{
    if (batch < 0 || batch > (int64_t(1) << 31) - 1) return -1;
    if (batch > 0 && !h_entries) return -2;
    if (!d_plan || (reinterpret_cast<uintptr_t>(d_plan) % 256)) return -5;
    if (plan_bytes < rfp::batch_plan_bytes(batch)) return -6;
    int64_t bad = -1;
    const int rc = rfp::batch_plan(batch, h_entries, arf_len, b_len, d_plan, (cudaStream_t)stream, &bad);
    if (bad_entry) *bad_entry = bad;
    if (rc >= 1000) return finish((cudaError_t)(rc - 1000));
    return rc;
}

int rfp_dpfsv_batched(int64_t batch, const void *d_plan, double *arf, double *B, int32_t *d_info,
                      void *stream)
{
    return batched_entry<double>(batch, d_plan, arf, B, d_info, stream);
}

int rfp_spfsv_batched(int64_t batch, const void *d_plan, float *arf, float *B, int32_t *d_info,
                      void *stream)
{
    return batched_entry<float>(batch, d_plan, arf, B, d_info, stream);
}

const char *rfp_status_string(int status)
{
    if (status == RFP_OK) return "success";
    if (status == RFP_ERR_CUDA) return "a CUDA call failed (see rfp_last_cuda_error)";
    if (status < 0) return "invalid argument (the value is minus its 1-based position)";
    return "unknown status";
}

const char *rfp_last_cuda_error(void) { return g_last_cuda_error; }

int64_t rfp_kernel_launches(void) { return rfp::g_launch_count.load(); }

int rfp_stage_timing(int enable)
{
    rfp::g_stages.enabled = enable != 0;
    rfp::g_stages.names.clear();
    return RFP_OK;
}

int rfp_stage_times(int max, float *ms, const char **names)
{
    rfp::StageLog &g = rfp::g_stages;
    if (g.names.empty()) return 0;
    cudaError_t e = cudaEventSynchronize(g.pool[g.names.size() - 1]);
    if (e != cudaSuccess) return -finish(e);
    int k = 0;
    for (size_t i = 1; i < g.names.size() && k < max; ++i) {
        if (!g.names[i]) continue;                // start of the next call
        float t = 0.f;
        cudaEventElapsedTime(&t, g.pool[i - 1], g.pool[i]);
        if (ms) ms[k] = t;
        if (names) names[k] = g.names[i];
        ++k;
    }
    return k;
}

// ---- the rest of the LAPACK 3.2 RFP routine set ----
int rfp_dtpttf(char transr, char uplo, int64_t n, const double *ap, double *arf, void *stream)
{
    return tp_entry<double>(transr, uplo, n, const_cast<double *>(ap), arf, stream, true);
}
int rfp_stpttf(char transr, char uplo, int64_t n, const float *ap, float *arf, void *stream)
{
    return tp_entry<float>(transr, uplo, n, const_cast<float *>(ap), arf, stream, true);
}
int rfp_dtfttp(char transr, char uplo, int64_t n, const double *arf, double *ap, void *stream)
{
    return tp_entry<double>(transr, uplo, n, const_cast<double *>(arf), ap, stream, false);
}
int rfp_stfttp(char transr, char uplo, int64_t n, const float *arf, float *ap, void *stream)
{
    return tp_entry<float>(transr, uplo, n, const_cast<float *>(arf), ap, stream, false);
}
int rfp_dtftri(char transr, char uplo, char diag, int64_t n, double *arf, int32_t *info,
               double *work, void *stream)
{
    return tftri_entry<double>(transr, uplo, diag, n, arf, info, work, stream);
}
int rfp_stftri(char transr, char uplo, char diag, int64_t n, float *arf, int32_t *info,
               float *work, void *stream)
{
    return tftri_entry<float>(transr, uplo, diag, n, arf, info, work, stream);
}
int rfp_dsfrk(char transr, char uplo, char trans, int64_t n, int64_t k, double alpha,
              const double *A, int64_t lda, double beta, double *C, void *stream)
{
    return sfrk_entry<double>(transr, uplo, trans, n, k, alpha, A, lda, beta, C, stream);
}
int rfp_ssfrk(char transr, char uplo, char trans, int64_t n, int64_t k, float alpha,
              const float *A, int64_t lda, float beta, float *C, void *stream)
{
    return sfrk_entry<float>(transr, uplo, trans, n, k, alpha, A, lda, beta, C, stream);
}
int rfp_dtfsm(char transr, char side, char uplo, char trans, char diag, int64_t m, int64_t n,
              double alpha, const double *arf, double *B, int64_t ldb, void *stream)
{
    return tfsm_entry<double>(transr, side, uplo, trans, diag, m, n, alpha, arf, B, ldb, stream);
}
int rfp_stfsm(char transr, char side, char uplo, char trans, char diag, int64_t m, int64_t n,
              float alpha, const float *arf, float *B, int64_t ldb, void *stream)
{
    return tfsm_entry<float>(transr, side, uplo, trans, diag, m, n, alpha, arf, B, ldb, stream);
}
int rfp_dlansf(char norm, char transr, char uplo, int64_t n, const double *arf, double *work,
               double *value, void *stream)
{
    return lansf_entry<double>(norm, transr, uplo, n, arf, work, value, stream);
}
int rfp_slansf(char norm, char transr, char uplo, int64_t n, const float *arf, float *work,
               float *value, void *stream)
{
    return lansf_entry<float>(norm, transr, uplo, n, arf, work, value, stream);
}

}  // extern "C"
