// Host-side internals shared by the library's translation units: the per-call context (device
// pointers carved from the workspace) and the launcher entry points of each stage.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ps_common.cuh"

namespace ps {

// Stage 1 with a minimal run length w (Sec. 5.1): w <= kMinRunMax; transfer functions are
// tables of kMrStates entries; the tile scan composes groups of kMrGroup tiles.
constexpr int kMinRunMax = 32;
constexpr int kMrStates = kMinRunMax + 2;
constexpr int kMrGroup = 256;

struct Ctx {
  cudaStream_t stream = nullptr;
  int kt = 0;            // key type (powersort.h ps_key_type)
  int key_bytes = 4;
  bool has_vals = false;
  int64_t n = 0;         // elements (all segments), < kMaxElems
  const int64_t* offsets = nullptr;  // device, count+1 entries, or null for one array
  int64_t max_segment = 0;  // > 0: the caller's bound on every segment's length (checked on the device)
  int32_t count = 1;

  void* k[2] = {nullptr, nullptr};   // [0] caller's keys, [1] scratch keys
  uint32_t* v[2] = {nullptr, nullptr};

  // per-run / per-boundary metadata (run_cap entries: r + 1 <= run_cap)
  int64_t run_cap = 0;
  pos_t* S = nullptr;           // run starts, S[r] = n
  uint8_t* run_desc = nullptr;  // run was strictly descending
  int32_t* run_seg = nullptr;   // segment of each run (segmented calls only)
  uint8_t* P = nullptr;         // node power of boundary j (0 for sentinels / segment borders)
  int32_t* nodeL = nullptr;     // node j merges [S[nodeL[j]], S[j]) and [S[j], S[nodeR[j]])
  int32_t* nodeR = nullptr;
  uint8_t* ndepth = nullptr;    // node depth
  uint8_t* ldepth = nullptr;    // leaf depth
  uint8_t* micro = nullptr;     // 1 for a node that is a micro root (see micro_tile)

  uint64_t* detect_state = nullptr;
  int32_t detect_tiles = 0;
  uint64_t* thr_L = nullptr;    // per detection thread: pair bits of its 32 positions
  uint64_t* thr_F = nullptr;    // forced-start bits (segmented calls only)
  uint32_t* thr_fn = nullptr;   // its transition function with run counts
  int min_run = 1;              // minimal run length w (1: greedy runs only)
  uint32_t* mr_tile_tab = nullptr;  // w > 1: per tile, kMrStates table entries
  uint32_t* mr_grp_tab = nullptr;   //        per group of kMrGroup tiles
  uint64_t* mr_grp_pre = nullptr;   //        entry state and runs before each group
  int32_t* tree_sum = nullptr;  // [32 power values][tree_stride tiles]
  int32_t tree_stride = 0;
  int32_t* tree_pre = nullptr;

  int32_t sub_lim = 0;          // subtree-in-SMEM element limit
  int pass_stages = 2;          // shared-memory stages of the level-pass ring
  int pass_ipt = kMergeItems;   // outputs per consumer thread of a level pass
  int32_t merge_tile = kMergeTile;  // outputs per level-pass tile (pass_ipt x kMergeThreads)
  int tree = 0;                 // merge tree: 0 powersort (Alg. 2), 1 peeksort (Alg. 1)
  int2* peek_front[2] = {nullptr, nullptr};  // peeksort: run ranges of one tree level
  uint32_t* peek_count = nullptr;            // peeksort: ranges per level [kMaxLevels + 1]
  int32_t peek_front_cap = 0;
  int32_t* small_tasks = nullptr;
  int32_t* leaf_items = nullptr;
  uint32_t* leaf_tile_off = nullptr;
  NodeItem* level_items = nullptr;     // [kMaxLevels][level_cap]: node ranges and reversed children
  uint32_t* level_tile_off = nullptr;
  int32_t level_cap = 0;

  uint32_t poll_limit = kMbarTries;  // bound of every level-pass wait
  int withhold_depth = -1;      // failure self-test: the level pass of this depth withholds a stage

  PlanHeader* hdr = nullptr;
  uint32_t* lib_status = nullptr;  // per-device status word owned by the library
  double* d_entropy = nullptr;
};

// Key-dependent stages (one table per key type).
struct KeyLaunch {
  cudaError_t (*detect)(const Ctx&);
  cudaError_t (*small)(const Ctx&, uint32_t ntasks);
  cudaError_t (*place)(const Ctx&, uint32_t nitems, uint32_t ntiles);
  cudaError_t (*merge)(const Ctx&, int depth, uint32_t nitems, uint32_t ntiles);
};
extern const KeyLaunch kLaunchI32, kLaunchU32, kLaunchF32, kLaunchU64;

// Key-independent stages (ps_meta.cu).
cudaError_t launch_meta_stages(const Ctx& c);
int meta_launches(const Ctx& c);
cudaError_t launch_entropy(const Ctx& c, double* d_out);
cudaError_t launch_check_offsets(const Ctx& c);
cudaError_t launch_header_out(const Ctx& c, PlanHeader* mapped);
cudaError_t launch_status_out(const Ctx& c);
cudaError_t launch_wait_timeout_probe(uint32_t polls, uint32_t* lib_status, cudaStream_t s);

// Bounds-checked builds (-DPS_DEBUG): out-of-range accesses counted by each translation unit's
// kernels (0 in other builds).
unsigned long long bounds_hits_meta();
unsigned long long bounds_hits_keys32();
unsigned long long bounds_hits_keys64();

}  // namespace ps
