// Stand-in for <cuda_bf16.h> used ONLY by the CPU emulation build.
#pragma once
#include <cstdint>
struct __nv_bfloat16 {
    uint16_t x;
};
