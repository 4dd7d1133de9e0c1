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
// at most `waves` full waves of resident blocks.  The default, 64 waves,
// leaves most threads one or two items and lets the block scheduler balance
// the tail: swept on GB300 at N = 2^26 against 4 waves, stored kmax 32 4.66 ->
// 4.59 ms, kmax 16 3.02 -> 2.93, kmax 4 1.91 -> 1.87, fused kmax 32 6.52 ->
// 6.39, gradient 1.007 -> 0.957 (one wave per item, i.e. no cap, was slower
// at stored kmax 32: 4.71).  BOYS_GRID_WAVES overrides it.
#ifndef BOYS_GRID_WAVES
#define BOYS_GRID_WAVES 64
#endif
int64_t grid_for(const void* kernel, int block, int64_t work, int64_t per_block, int waves = BOYS_GRID_WAVES,
                 size_t smem = 0);

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace boys
