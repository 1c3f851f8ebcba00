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
//   * every GPU that loads the library holds the 32 MiB array until the
//     process exits;
//   * problems whose workspace (rfp_dpfsv_mixed_workspace) exceeds 32 MiB are
//     rejected (for example n = 2048 with nrhs up to 256 fits in the FP32,
//     TF32 and BF16 modes, n = 1664 in the split-TF32 mode and n = 1472 in
//     the split-BF16 mode);
//   * all calls share the one array: calls whose work overlaps on the GPU (two
//     streams, or two host threads) race on it and give wrong results;
//     serialize them;
//   * the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress); make that first call before any stream capture.
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

std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per
// device, with that device current); nullptr on failure.
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
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_scratch);
        if (*err != cudaSuccess) return nullptr;
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

}  // namespace

extern "C" {

size_t rfp_dpfsv_mixed_noalloc_capacity(void) { return kScratchBytes; }

int rfp_dpfsv_mixed_noalloc(char transr, char uplo, int64_t n, int64_t nrhs, const double *arf,
                            const double *B, int64_t ldb, double *X, int64_t ldx, int prec,
                            int max_iter, double tol, rfp_mixed_status_t *status, void *stream)
{
    if (n > 0 && nrhs > 0) {
        // Problems larger than the fixed array: -3 when n alone does not fit
        // (even with one right-hand side), else -4 (too many right-hand sides).
        if (rfp_dpfsv_mixed_workspace(n, 1, prec) > kScratchBytes) return -3;
        if (rfp_dpfsv_mixed_workspace(n, nrhs, prec) > kScratchBytes) return -4;
    }
    cudaError_t e = cudaSuccess;
    void *scratch = scratch_address(&e);
    if (!scratch) return RFP_ERR_CUDA;
    // Arguments 13 and 14 of rfp_dpfsv_mixed (work, work_bytes) are the fixed
    // array; its other argument checks and return codes apply unchanged.
    int rc = rfp_dpfsv_mixed(transr, uplo, n, nrhs, arf, B, ldb, X, ldx, prec, max_iter, tol,
                             scratch, kScratchBytes, status, stream);
    if (rc == -15) rc = -13;   // status is argument 13 here
    if (rc == -16) rc = -14;   // stream is argument 14 here
    return rc;
}

}  // extern "C"
