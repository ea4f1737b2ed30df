// Device-side bounds checks of the debug build (compiled with -DPAT_DEBUG_BOUNDS).
//
// Each check guards an access whose index comes from run-time data rather than
// from the compile-time tile shape: the sensor stencil tables of the plan (sensor
// index, grid column, row of a stencil entry), the time step of a trace and the
// slot of the pressure history.  A failed check ORs PAT_STATUS_BOUNDS into the
// workspace status word (read by pat_status) and the caller skips the access or
// falls back to an index that is in range, so an index error shows up as a status
// bit instead of faulting the GPU.  The release build compiles every check to
// `true`.
#pragma once

#include <cuda_runtime.h>

#include "../../include/pat.h"

namespace pat {

#ifdef PAT_DEBUG_BOUNDS
constexpr bool kDebugBounds = true;
__device__ __forceinline__ bool in_range(long long i, long long n, int* status) {
    if (i >= 0 && i < n) return true;
    if (status) atomicOr(status, PAT_STATUS_BOUNDS);
    return false;
}
#else
constexpr bool kDebugBounds = false;
__device__ __forceinline__ constexpr bool in_range(long long, long long, int*) { return true; }
#endif

// i if it lies in [0, n), else 0 (and the status bit in the debug build)
__device__ __forceinline__ int in_range_or_zero(int i, int n, int* status) {
    return in_range(i, n, status) ? i : 0;
}

}  // namespace pat
