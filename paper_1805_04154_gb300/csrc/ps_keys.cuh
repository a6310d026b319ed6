// Host launchers of the key-dependent kernels, instantiated once per key type by the
// ps_keys_*.cu translation units.
#pragma once

#include "ps_detect.cuh"
#include "ps_internal.h"
#include "ps_merge.cuh"

namespace ps {

template <class K>
struct Launch {
  typedef typename K::T T;

  static cudaError_t detect(const Ctx& c) {
    detect_runs_kernel<K><<<c.detect_tiles, kDetectThreads, 0, c.stream>>>(
        (const T*)c.k[0], c.n, c.offsets, c.count, c.S, c.run_desc, c.run_seg, c.detect_state, c.hdr,
        c.lib_status);
    return cudaGetLastError();
  }

  template <bool V>
  static cudaError_t small_v(const Ctx& c, uint32_t ntasks) {
    static bool attr = false;
    const size_t bytes = SubLayout<K, V>::kBytes;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(subtree_kernel<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)bytes);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    Bufs b{{c.k[0], c.k[1]}, {c.v[0], c.v[1]}};
    subtree_kernel<K, V><<<ntasks, kSubThreads, bytes, c.stream>>>(b, c.S, c.run_desc, c.nodeL, c.nodeR,
                                                                    c.ndepth, c.ldepth, c.small_tasks, c.hdr,
                                                                    c.lib_status);
    return cudaGetLastError();
  }
  static cudaError_t small(const Ctx& c, uint32_t ntasks) {
    if (ntasks == 0) return cudaSuccess;
    return c.has_vals ? small_v<true>(c, ntasks) : small_v<false>(c, ntasks);
  }

  static cudaError_t place(const Ctx& c, uint32_t nitems, uint32_t ntiles) {
    if (ntiles == 0) return cudaSuccess;
    Bufs b{{c.k[0], c.k[1]}, {c.v[0], c.v[1]}};
    if (c.has_vals)
      leaf_place_kernel<K, true><<<ntiles, 256, 0, c.stream>>>(b, c.S, c.run_desc, c.ldepth, c.leaf_items,
                                                               c.leaf_tile_off, nitems);
    else
      leaf_place_kernel<K, false><<<ntiles, 256, 0, c.stream>>>(b, c.S, c.run_desc, c.ldepth, c.leaf_items,
                                                                c.leaf_tile_off, nitems);
    return cudaGetLastError();
  }

  template <bool V>
  static cudaError_t merge_v(const Ctx& c, int depth, uint32_t ntiles) {
    static bool attr = false;
    const size_t bytes = MergeLayout<K, V>::kBytes;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(merge_tile_kernel<K, V>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    const int src = (depth + 1) & 1, dst = depth & 1;
    merge_tile_kernel<K, V><<<ntiles, kMergeThreads, bytes, c.stream>>>(
        (const T*)c.k[src], c.v[src], (T*)c.k[dst], c.v[dst], c.tiles, c.hdr, c.lib_status);
    return cudaGetLastError();
  }

  static cudaError_t corank(const Ctx& c, int depth, uint32_t nitems, uint32_t ntiles) {
    if (ntiles == 0) return cudaSuccess;
    const int src = (depth + 1) & 1;
    const size_t off = (size_t)depth * c.level_cap;
    const uint32_t warps_per_block = 8;
    corank_kernel<K><<<(ntiles + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, c.stream>>>(
        (const T*)c.k[src], c.S, c.nodeL, c.nodeR, c.level_items + off, c.level_tile_off + off, nitems, ntiles,
        c.tiles);
    return cudaGetLastError();
  }

  static cudaError_t merge(const Ctx& c, int depth, uint32_t ntiles) {
    if (ntiles == 0) return cudaSuccess;
    return c.has_vals ? merge_v<true>(c, depth, ntiles) : merge_v<false>(c, depth, ntiles);
  }

  static KeyLaunch table() { return KeyLaunch{&detect, &small, &place, &corank, &merge}; }
};

}  // namespace ps
