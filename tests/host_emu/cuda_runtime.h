// Minimal stand-in for <cuda_runtime.h> used ONLY to compile the library's
// host orchestration (chol.cu, api.cu) with g++ against the kernel emulator
// in emu_kernels.cpp.  Never used by the product build.
#pragma once
#include <cstddef>
#include <cstdint>

#define __host__
#define __device__
#define __global__
#define __forceinline__ inline

typedef int cudaError_t;
typedef void *cudaStream_t;
enum { cudaSuccess = 0, cudaErrorInvalidValue = 1, cudaErrorIllegalAddress = 700,
       cudaErrorNotSupported = 801 };

typedef void *cudaEvent_t;
cudaError_t cudaMemsetAsync(void *p, int v, size_t n, cudaStream_t s);
cudaError_t cudaEventCreate(cudaEvent_t *e);
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t s);
cudaError_t cudaEventSynchronize(cudaEvent_t e);
cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t a, cudaEvent_t b);
const char *cudaGetErrorName(cudaError_t e);
cudaError_t cudaGetLastError(void);
