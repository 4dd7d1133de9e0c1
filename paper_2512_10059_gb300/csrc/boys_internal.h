// Host-side plumbing shared by the libboys translation units: export macro,
// per-thread error text, CUDA error mapping and launch-shape helpers.
#pragma once

#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "../../include/boys.h"

#define BOYS_API extern "C" __attribute__((visibility("default")))

namespace boys {

// Records a formatted message as this thread's last error and returns `s`.
boys_status fail(boys_status s, const char* fmt, ...);
// Maps a CUDA error to BOYS_ERR_CUDA (recording its text) or BOYS_OK.
boys_status check_cuda(cudaError_t e, const char* what);
// Number of SMs of the current device (cached per device).
int sm_count();
// Resident blocks per SM for `kernel` at `block` threads (cached by pointer).
int blocks_per_sm(const void* kernel, int block, size_t smem = 0);
// Grid size for a grid-stride kernel over `work` items of `per_block` each:
// at most `waves` full waves of resident blocks.
int64_t grid_for(const void* kernel, int block, int64_t work, int64_t per_block, int waves = 4,
                 size_t smem = 0);

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace boys
