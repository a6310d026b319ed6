// Bounds-checked builds.  Compiled with -DPS_DEBUG, every index that PS_IN_RANGE guards is
// compared with its array's extent before the access; an index out of range is counted in this
// translation unit's device counter and the access is skipped, so a bad index shows up as a
// count (and usually a wrong result) instead of a fault.  Without PS_DEBUG the guard is the
// constant true and the compiler removes it.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ps {

#ifdef PS_DEBUG
constexpr bool kBoundsChecked = true;
static __device__ unsigned long long g_bounds_hits;  // one counter per translation unit

__device__ __forceinline__ bool in_range(int64_t i, int64_t n) {
  if (i >= 0 && i < n) return true;
  atomicAdd(&g_bounds_hits, 1ull);
  return false;
}
#define PS_IN_RANGE(i, n) (::ps::in_range((int64_t)(i), (int64_t)(n)))

// out-of-range accesses counted so far by the kernels of this translation unit
static inline unsigned long long bounds_hits_here() {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_hits, sizeof(v)) != cudaSuccess) return ~0ull;
  return v;
}
#else
constexpr bool kBoundsChecked = false;
#define PS_IN_RANGE(i, n) true
static inline unsigned long long bounds_hits_here() { return 0; }
#endif

}  // namespace ps
