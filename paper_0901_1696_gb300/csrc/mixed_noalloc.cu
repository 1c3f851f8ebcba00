// rfp_dpfsv_mixed_noalloc: the mixed-precision solve for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// that runs inside a memory pool owned by someone else, a plugin whose host
// application forbids device allocations after start-up, or a real-time loop
// where an allocation could block or fail.  This entry point runs exactly the
// launch sequence of rfp_dpfsv_mixed, but its workspace is a fixed array
// compiled into the library (kScratchBytes = 32 MiB), so it allocates nothing.
//
// Costs and rules that come with that:
//   * the array is reserved on a device when the library's code for it is
//     loaded there: with CUDA's default lazy module loading that is the first
//     call on that device (CUDA_MODULE_LOADING=EAGER reserves it when the
//     context is created).  Make that first call at start-up, while device
//     memory is still free, and before any stream capture; from then on the
//     device holds the 32 MiB until the process exits;
//   * problems whose workspace (rfp_dpfsv_mixed_workspace) exceeds 32 MiB are
//     rejected (for example n = 2048 with nrhs up to 256 fits in the FP32,
//     TF32 and BF16 modes, n = 1664 in the split-TF32 mode and n = 1472 in
//     the split-BF16 mode);
//   * all calls share the one array: calls whose work overlaps on the GPU (two
//     streams, or two host threads) race on it and give wrong results;
//     serialize them;
//   * the array's device address is looked up (cudaGetSymbolAddress) on the
//     first call on each device, and again whenever the calling thread's
//     current context differs from the one it was looked up in (a device
//     reset, or a context the caller created itself).
// The array keeps whatever the previous call left in it; the solve clears
// what must start at zero (its stop and error words and the status) itself.
#include <mutex>

#include "mixed_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

// The fixed workspace.  In host code g_scratch is only a stand-in for the
// device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Driver entry points that identify the current context, fetched through the
// runtime (the library does not link the driver library directly).
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

struct ScratchCache {
    unsigned long long ctx_id;   // 0: unknown context, look the address up again
    void *ptr;
};

std::mutex g_mutex;
ScratchCache g_cache[kMaxDevices] = {};
bool g_fns_looked_up = false;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Identifier of the calling thread's current context, 0 if there is none or
// it cannot be told (the caller then looks the address up every time).
// Called with g_mutex held.
unsigned long long current_context_id()
{
    if (!g_fns_looked_up) {
        g_fns_looked_up = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    void *ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
    unsigned long long id = 0;
    if (g_ctx_get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_scratch in the current context of the current device;
// nullptr (and *err set) on failure.
void *scratch_address(cudaError_t *err)
{
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= kMaxDevices) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    ScratchCache &c = g_cache[dev];
    const unsigned long long id = current_context_id();
    if (c.ptr && id != 0 && c.ctx_id == id) return c.ptr;
    void *p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_scratch);   // loads the module on first use
    if (*err != cudaSuccess) {
        c.ptr = nullptr;
        return nullptr;
    }
    // The lookup itself makes the device's primary context current when no
    // context was; ask again so that the entry is keyed on it.
    c.ctx_id = id != 0 ? id : current_context_id();
    c.ptr = p;
    return p;
}

}  // namespace

extern "C" {

size_t rfp_dpfsv_mixed_noalloc_capacity(void) { return kScratchBytes; }

int rfp_dpfsv_mixed_noalloc(char transr, char uplo, int64_t n, int64_t nrhs, const double *arf,
                            const double *B, int64_t ldb, double *X, int64_t ldx, int prec,
                            int max_iter, double tol, rfp_mixed_status_t *status, void *stream)
{
    // Every argument is checked first, with rfp_dpfsv_mixed's own checks; its
    // status argument (15 there) is argument 13 here.
    const int bad = rfp::mixed_check_args(transr, uplo, n, nrhs, arf, B, ldb, X, ldx, prec,
                                          max_iter, tol, status);
    if (bad) return bad == -15 ? -13 : bad;
    if (n > 0 && nrhs > 0) {
        // Valid problems larger than the fixed array: -3 when n alone does
        // not fit (even with one right-hand side), else -4 (too many
        // right-hand sides).
        if (rfp_dpfsv_mixed_workspace(n, 1, prec) > kScratchBytes) return -3;
        if (rfp_dpfsv_mixed_workspace(n, nrhs, prec) > kScratchBytes) return -4;
    }
    cudaError_t e = cudaSuccess;
    void *scratch = scratch_address(&e);
    if (!scratch) return rfp::finish_cuda(e);
    // Arguments 13 and 14 of rfp_dpfsv_mixed (work, work_bytes) are the fixed
    // array; its other arguments were checked above.
    int rc = rfp_dpfsv_mixed(transr, uplo, n, nrhs, arf, B, ldb, X, ldx, prec, max_iter, tol,
                             scratch, kScratchBytes, status, stream);
    if (rc == -15) rc = -13;   // status is argument 13 here
    if (rc == -16) rc = -14;   // stream is argument 14 here
    return rc;
}

}  // extern "C"
