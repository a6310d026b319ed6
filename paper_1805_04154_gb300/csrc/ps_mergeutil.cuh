// Small helpers shared by the merge kernels: the buffer pair, the stable key order, the
// serial merge-path co-rank and the tile -> work-item lookup.
#pragma once

#include "ps_common.cuh"

namespace ps {

struct Bufs {
  void* k[2];      // key buffers: [0] the caller's array, [1] scratch
  uint32_t* v[2];  // payload buffers (null when there is no payload)
};

template <class K>
__device__ __forceinline__ bool key_le(typename K::T a, typename K::T b) {
  return K::le(a, b);
}

// co-rank of output position diag in the merge of A[0..la) and B[0..lb)
template <class K, class TA, class TB>
__device__ __forceinline__ int32_t corank_serial(TA A, TB B, int32_t la, int32_t lb, int32_t diag) {
  int32_t lo = max(0, diag - lb), hi = min(diag, la);
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (key_le<K>(A[mid], B[diag - 1 - mid])) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// tile t -> item slot: largest s with tile_off[s] <= t
__device__ __forceinline__ int32_t slot_of_tile(const uint32_t* __restrict__ tile_off, uint32_t nitems, uint32_t t) {
  int32_t a = 0, b = (int32_t)nitems;
  while (b - a > 1) {
    const int32_t mid = (a + b) >> 1;
    if (tile_off[mid] <= t) a = mid; else b = mid;
  }
  return a;
}

}  // namespace ps
