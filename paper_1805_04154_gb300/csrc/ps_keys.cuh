// Host launchers of the key-dependent kernels, instantiated once per key type by the
// ps_keys_*.cu translation units.
#pragma once

#include <algorithm>
#include <cstdlib>

#include "ps_detect.cuh"
#include "ps_detect_minrun.cuh"
#include "ps_internal.h"
#include "ps_level.cuh"
#include "ps_merge.cuh"

namespace ps {

template <class K>
struct Launch {
  typedef typename K::T T;

  static cudaError_t detect(const Ctx& c) {
    if (c.min_run > 1) return detect_minrun(c);
    detect_reduce_kernel<K><<<c.detect_tiles, kDetectThreads, 0, c.stream>>>(
        (const T*)c.k[0], c.n, c.offsets, c.count, c.detect_state, c.thr_L, c.thr_F, c.thr_fn);
    detect_scan_kernel<<<1, 1024, 0, c.stream>>>(c.detect_state, c.detect_tiles, c.n, c.run_cap,
                                                 c.detect_state + c.detect_tiles, c.S, c.hdr);
    detect_emit_kernel<K><<<c.detect_tiles, kDetectThreads, 0, c.stream>>>(
        c.n, c.run_cap, c.offsets, c.count, c.detect_state + c.detect_tiles, c.thr_L, c.thr_F, c.thr_fn, c.S, c.run_desc,
        c.run_seg);
    return cudaGetLastError();
  }

  // five launches: tile tables, group tables, the walk over groups, tile entries, emit
  static cudaError_t detect_minrun(const Ctx& c) {
    const int32_t tiles = c.detect_tiles, groups = (tiles + kMrGroup - 1) / kMrGroup;
    const size_t nthreads = (size_t)tiles * kDetectThreads;
    uint64_t* tile_pre = c.detect_state + c.detect_tiles;
    minrun_reduce_kernel<K><<<tiles, kDetectThreads, 0, c.stream>>>((const T*)c.k[0], c.n, c.offsets, c.count,
                                                                    c.min_run, c.mr_tile_tab, c.thr_L, c.thr_F);
    minrun_group_kernel<<<groups, 256, 0, c.stream>>>(c.mr_tile_tab, tiles, c.min_run, c.mr_grp_tab);
    minrun_top_kernel<<<1, 256, 0, c.stream>>>(c.mr_grp_tab, groups, c.n, c.run_cap, c.mr_grp_pre, c.S, c.hdr);
    minrun_tile_kernel<<<groups, 256, 0, c.stream>>>(c.mr_tile_tab, tiles, c.mr_grp_pre, tile_pre);
    minrun_emit_kernel<K><<<tiles, kDetectThreads, 0, c.stream>>>(c.n, c.run_cap, c.offsets, c.count, c.min_run, tile_pre,
                                                                  c.thr_L, c.thr_F, nthreads, c.S, c.run_desc,
                                                                  c.run_seg);
    return cudaGetLastError();
  }

  static int sm_count() {
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms <= 0) sms = 152;
    }
    return sms;
  }

  // ntasks == kCountOnDevice: persistent grid, the count is read from the plan on the device
  template <bool V>
  static cudaError_t small_v(const Ctx& c, uint32_t ntasks) {
    static bool attr = false;
    const size_t bytes = SubLayout<K, V>::kBytes;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(subtree_kernel<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)bytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(subtree_persistent_kernel<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    Bufs b{{c.k[0], c.k[1]}, {c.v[0], c.v[1]}};
    const uint32_t cap = (uint32_t)std::min<int64_t>(c.run_cap, 0xffffffffll);
    if (ntasks == kCountOnDevice) {
      // one CTA per task up to a bound known without the plan: a small task is a segment's root
      // or a child of a node larger than the subtree limit, whose subtrees hold more than half the
      // limit in balanced parts of the tree, so 2n / limit + segments covers ordinary inputs (a
      // random permutation has about 1.4n / limit tasks, the 10,000-segment batch 0.2n / limit);
      // surplus CTAs return at once, and the persistent kernel takes any tasks beyond the bound
      uint32_t grid = (uint32_t)std::min<int64_t>((int64_t)cap, 2 * c.n / c.sub_lim + (int64_t)c.count + 64);
      // PS_SUBTREE_GRID (tests only): a smaller one-task grid, so that the persistent kernel
      // takes the remaining tasks
      static const uint32_t forced = [] {
        const char* e = std::getenv("PS_SUBTREE_GRID");
        return e ? (uint32_t)std::strtoul(e, nullptr, 10) : 0u;
      }();
      if (forced) grid = std::min(grid, forced);
      subtree_kernel<K, V><<<grid, kSubThreads, bytes, c.stream>>>(b, c.S, c.run_desc, c.nodeL, c.nodeR, c.ndepth,
                                                                    c.ldepth, c.micro, c.small_tasks, cap, c.hdr,
                                                                    c.lib_status);
      subtree_persistent_kernel<K, V><<<(uint32_t)sm_count() * 4, kSubThreads, bytes, c.stream>>>(
          b, c.S, c.run_desc, c.nodeL, c.nodeR, c.ndepth, c.ldepth, c.micro, c.small_tasks, grid, cap, c.hdr,
          c.lib_status);
    } else {
      subtree_kernel<K, V><<<ntasks, kSubThreads, bytes, c.stream>>>(b, c.S, c.run_desc, c.nodeL, c.nodeR,
                                                                      c.ndepth, c.ldepth, c.micro, c.small_tasks, 0u,
                                                                      c.hdr, c.lib_status);
    }
    return cudaGetLastError();
  }
  static cudaError_t small(const Ctx& c, uint32_t ntasks) {
    if (ntasks == 0) return cudaSuccess;
    return c.has_vals ? small_v<true>(c, ntasks) : small_v<false>(c, ntasks);
  }

  // resident CTAs per SM of a 256-thread kernel without dynamic shared memory
  template <class Kern>
  static int resident(Kern kern) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 256, 0) != cudaSuccess || b < 1) b = 1;
    return b;
  }

  static cudaError_t place(const Ctx& c, uint32_t nitems, uint32_t ntiles) {
    if (ntiles == 0) return cudaSuccess;
    Bufs b{{c.k[0], c.k[1]}, {c.v[0], c.v[1]}};
    const uint32_t cap = (uint32_t)c.level_cap;
    static int occ_v = 0, occ_k = 0;
    if (occ_v == 0) {
      occ_v = resident(leaf_place_kernel<K, true>);
      occ_k = resident(leaf_place_kernel<K, false>);
    }
    const uint32_t full = (uint32_t)sm_count() * (uint32_t)(c.has_vals ? occ_v : occ_k);
    if (ntiles == kCountOnDevice) {
      if (c.has_vals)
        leaf_place_persistent_kernel<K, true><<<full, 256, 0, c.stream>>>(b, c.S, c.run_desc, c.ldepth, c.leaf_items,
                                                                          c.leaf_tile_off, cap, c.hdr);
      else
        leaf_place_persistent_kernel<K, false><<<full, 256, 0, c.stream>>>(b, c.S, c.run_desc, c.ldepth,
                                                                           c.leaf_items, c.leaf_tile_off, cap, c.hdr);
    } else {
      const uint32_t grid = std::min(ntiles, full);
      if (c.has_vals)
        leaf_place_kernel<K, true><<<grid, 256, 0, c.stream>>>(b, c.S, c.run_desc, c.ldepth, c.leaf_items,
                                                               c.leaf_tile_off, nitems, ntiles, c.hdr);
      else
        leaf_place_kernel<K, false><<<grid, 256, 0, c.stream>>>(b, c.S, c.run_desc, c.ldepth, c.leaf_items,
                                                                c.leaf_tile_off, nitems, ntiles, c.hdr);
    }
    return cudaGetLastError();
  }

  template <bool V, int NS, int IPT>
  static cudaError_t merge_vs(const Ctx& c, int depth, uint32_t nitems, uint32_t ntiles) {
    static int blocks_per_sm = 0;
    static int sms = 0;
    const size_t bytes = PassLayout<K, V, NS, IPT>::kBytes;
    if (blocks_per_sm == 0) {
      cudaError_t e = cudaFuncSetAttribute(level_pass_kernel<K, V, NS, IPT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, level_pass_kernel<K, V, NS, IPT>,
                                                        kLevelThreads, bytes);
      if (e != cudaSuccess) return e;
      if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const int src = (depth + 1) & 1, dst = depth & 1;
    const size_t off = (size_t)depth * c.level_cap;
    const bool on_dev = ntiles == kCountOnDevice;
    const uint32_t grid = on_dev ? (uint32_t)(sms * blocks_per_sm)
                                 : (uint32_t)std::min<uint64_t>(ntiles, (uint64_t)sms * blocks_per_sm);
    level_pass_kernel<K, V, NS, IPT><<<grid, kLevelThreads, bytes, c.stream>>>(
        (const T*)c.k[src], c.v[src], (T*)c.k[dst], c.v[dst], c.level_items + off, c.level_tile_off + off, nitems,
        ntiles, on_dev ? &c.hdr->level_ctr[depth] : nullptr, (uint32_t)c.level_cap, c.hdr, c.lib_status, c.poll_limit,
        c.withhold_depth == depth ? 1 : 0);
    return cudaGetLastError();
  }

  // the level-pass configurations the library carries (items per thread, ring stages); the
  // autotuner chooses among them
  template <bool V>
  static cudaError_t merge_v(const Ctx& c, int depth, uint32_t nitems, uint32_t ntiles) {
    switch (pass_variant(c.pass_ipt, c.pass_stages)) {
      case pass_variant(12, 3): return merge_vs<V, 3, 12>(c, depth, nitems, ntiles);
      case pass_variant(12, 4): return merge_vs<V, 4, 12>(c, depth, nitems, ntiles);
      case pass_variant(8, 2): return merge_vs<V, 2, 8>(c, depth, nitems, ntiles);
      case pass_variant(8, 3): return merge_vs<V, 3, 8>(c, depth, nitems, ntiles);
      case pass_variant(16, 2): return merge_vs<V, 2, 16>(c, depth, nitems, ntiles);
      case pass_variant(6, 2): return merge_vs<V, 2, 6>(c, depth, nitems, ntiles);
      case pass_variant(10, 2): return merge_vs<V, 2, 10>(c, depth, nitems, ntiles);
      default: return merge_vs<V, 2, 12>(c, depth, nitems, ntiles);
    }
  }

  static cudaError_t merge(const Ctx& c, int depth, uint32_t nitems, uint32_t ntiles) {
    if (ntiles == 0) return cudaSuccess;
    return c.has_vals ? merge_v<true>(c, depth, nitems, ntiles) : merge_v<false>(c, depth, nitems, ntiles);
  }

  static KeyLaunch table() { return KeyLaunch{&detect, &small, &place, &merge}; }
};

}  // namespace ps
