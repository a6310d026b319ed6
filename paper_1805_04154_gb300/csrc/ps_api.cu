// C-ABI entry points of libpowersort.so (declared in include/powersort.h): argument checks,
// workspace layout, and the stage sequence
//   detect runs -> node powers -> merge tree -> plan -> [one D2H of the plan header]
//   -> small subtrees in SMEM + large-leaf placement -> level passes, deepest first.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "powersort.h"
#include "ps_debug.cuh"
#include "ps_internal.h"

namespace {

using namespace ps;

constexpr int kMaxDevices = 64;

const KeyLaunch* launch_for(int kt) {
  switch (kt) {
    case PS_KEY_I32: return &kLaunchI32;
    case PS_KEY_U32: return &kLaunchU32;
    case PS_KEY_U64: return &kLaunchU64;
    case PS_KEY_F32: return &kLaunchF32;
  }
  return nullptr;
}

int key_bytes(int kt) { return kt == PS_KEY_U64 ? 8 : 4; }

// Carve the workspace into the per-call arrays.  With base == nullptr only the size is computed.
size_t carve(Ctx& c, uint8_t* base, int kt, bool vals, int64_t n, bool segmented, int tree = 0) {
  size_t cur = 0;
  auto take = [&](size_t bytes) -> void* {
    cur = (cur + 255) & ~(size_t)255;
    void* p = base ? (void*)(base + cur) : nullptr;
    cur += std::max<size_t>(bytes, 16);
    return p;
  };
  const size_t kb = (size_t)key_bytes(kt);
  // Run-indexed arrays hold N entries: runs 0..r-1 and the boundaries 0..r.  A greedy run is at
  // least two elements long unless it starts at the last position of its array or segment, so
  // one array has r <= n/2 + 1 runs; segments of one element each can make r = n.
  const size_t N = segmented ? (size_t)n + 2 : (size_t)n / 2 + 3;
  c.run_cap = (int64_t)N;
  c.k[1] = take((((size_t)n * kb + 15) & ~(size_t)15) + 16);
  c.v[1] = vals ? (uint32_t*)take((((size_t)n * 4 + 15) & ~(size_t)15) + 16) : nullptr;
  c.S = (pos_t*)take(N * 4);
  c.run_desc = (uint8_t*)take(N);
  c.run_seg = segmented ? (int32_t*)take(N * 4) : nullptr;
  c.P = (uint8_t*)take(N + 8);  // the tree passes read whole aligned words up to byte r + 3
  c.nodeL = (int32_t*)take(N * 4);
  c.nodeR = (int32_t*)take(N * 4);
  c.ndepth = (uint8_t*)take(N);
  c.ldepth = (uint8_t*)take(N);
  c.micro = (uint8_t*)take(N);
  c.detect_tiles = (int32_t)((n + kDetectTile - 1) / kDetectTile);
  c.detect_state = (uint64_t*)take((size_t)std::max<int32_t>(c.detect_tiles, 1) * 16);  // functions + prefixes
  const size_t dthreads = (size_t)std::max<int32_t>(c.detect_tiles, 1) * kDetectThreads;
  c.thr_L = (uint64_t*)take(dthreads * 8);
  c.thr_F = segmented ? (uint64_t*)take(dthreads * 8) : nullptr;
  c.thr_fn = (uint32_t*)take(dthreads * 4);
  {
    // minimal-run-length tables (reserved always: about 0.02 bytes per element)
    const size_t tiles = (size_t)std::max<int32_t>(c.detect_tiles, 1);
    const size_t groups = (tiles + kMrGroup - 1) / kMrGroup;
    c.mr_tile_tab = (uint32_t*)take(tiles * kMrStates * 4);
    c.mr_grp_tab = (uint32_t*)take(groups * kMrStates * 4);
    c.mr_grp_pre = (uint64_t*)take(groups * 8);
  }
  const size_t tree_tiles = (size_t)(n + 1) / kTreeTile + 1;
  c.tree_stride = (int32_t)tree_tiles;
  c.tree_sum = (int32_t*)take(tree_tiles * 32 * 4);
  c.tree_pre = (int32_t*)take(tree_tiles * 32 * 4);
  c.sub_lim = sub_tile((int)kb);
  c.small_tasks = (int32_t*)take(N * 4);
  const size_t cap = (size_t)n / (size_t)(c.sub_lim + 1) + 2;
  c.tree = tree;
  if (tree == PS_TREE_PEEKSORT) {
    // ranges of one tree level: disjoint, each holding >= 2 runs, so at most (r + 1) / 2
    c.peek_front_cap = (int32_t)(N / 2 + 2);
    c.peek_front[0] = (int2*)take((size_t)c.peek_front_cap * sizeof(int2));
    c.peek_front[1] = (int2*)take((size_t)c.peek_front_cap * sizeof(int2));
    c.peek_count = (uint32_t*)take((kMaxLevels + 2) * sizeof(uint32_t));
  }
  c.leaf_items = (int32_t*)take(cap * 4);
  c.leaf_tile_off = (uint32_t*)take(cap * 4);
  c.level_cap = (int32_t)cap;
  c.level_items = (NodeItem*)take((size_t)kMaxLevels * cap * sizeof(NodeItem));
  c.level_tile_off = (uint32_t*)take((size_t)kMaxLevels * cap * 4);
  c.hdr = (PlanHeader*)take(sizeof(PlanHeader));
  c.d_entropy = (double*)take(sizeof(double));
  return (cur + 255) & ~(size_t)255;
}

// ---- per-device library state: status word and memory pool --------------------------------
std::mutex g_mu;
uint32_t* g_status[kMaxDevices] = {};
cudaMemPool_t g_pool[kMaxDevices] = {};

uint32_t* lib_status_word(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  if (!g_status[dev]) {
    uint32_t* p = nullptr;
    if (cudaMalloc(&p, 64) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, 64) != cudaSuccess) return nullptr;
    g_status[dev] = p;
  }
  return g_status[dev];
}

cudaMemPool_t lib_pool(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;  // keep freed blocks for reuse instead of returning them at syncs
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}

// ---- measurement: per-stage device time (CUDA events on the caller's stream), launches,
// algorithmic bytes --------------------------------------------------------------------------
constexpr int kStages = 8;  // 0 detect, 1 powers+tree+plan, 2 SMEM subtrees, 3 leaf placement,
                            // 4 (unused), 5 level passes
std::atomic<int> g_prof_on{0};
std::atomic<unsigned long long> g_launches{0};
struct ProfRec {
  int stage, dev;
  cudaEvent_t a, b;
  uint64_t bytes, launches;
};
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof_pending;
// Events are reused across sorts (creating one per stage would put host time between the
// plan read-back and the merge launches of every profiled sort).
std::vector<cudaEvent_t> g_ev_free[kMaxDevices];

cudaEvent_t prof_event(int dev) {
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (dev >= 0 && dev < kMaxDevices && !g_ev_free[dev].empty()) {
      cudaEvent_t e = g_ev_free[dev].back();
      g_ev_free[dev].pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// with g_prof_mu held
void prof_release(int dev, cudaEvent_t e) {
  if (!e) return;
  if (dev >= 0 && dev < kMaxDevices) g_ev_free[dev].push_back(e);
  else cudaEventDestroy(e);
}
double g_prof_ms[kStages] = {};
uint64_t g_prof_launch[kStages] = {}, g_prof_bytes[kStages] = {};

// Stage scopes: an NVTX range on the host (visible to Nsight tools; inert without one) and,
// while profiling is enabled, CUDA events on the stream around the stage's launches.
const char* const kStageNames[kStages] = {"ps:detect", "ps:meta", "ps:subtree_smem", "ps:leaf_place",
                                          "ps:unused", "ps:level_pass", "ps:stage6", "ps:stage7"};

struct StageTimer {
  int stage;
  int dev = 0;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  bool on;
  StageTimer(int st, cudaStream_t strm) : stage(st), s(strm), on(g_prof_on.load() != 0) {
    nvtxRangePushA(kStageNames[st]);
    if (on && cudaGetDevice(&dev) == cudaSuccess && (a = prof_event(dev)) != nullptr) cudaEventRecord(a, s);
    else on = false;
  }
  ~StageTimer() { nvtxRangePop(); }
  StageTimer(const StageTimer&) = delete;
  StageTimer& operator=(const StageTimer&) = delete;
  void done(uint64_t bytes, uint64_t launches) {
    g_launches += launches;
    if (!on) return;
    cudaEvent_t b = prof_event(dev);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!b) {
      prof_release(dev, a);
      return;
    }
    cudaEventRecord(b, s);
    g_prof_pending.push_back(ProfRec{stage, dev, a, b, bytes, launches});
  }
};

struct AnalyzeOut {
  int64_t* runs;
  uint64_t* cost;
  int64_t* starts;
  uint8_t* desc;
  uint8_t* power;
  uint8_t* leaf_depth;
  int32_t* node_left;
  int32_t* node_right;
  uint8_t* node_depth;
  ps_stats* stats;
};

// Level-pass configuration (items per consumer thread, ring stages), per key type and payload
// choice: 8 items and 2 stages for 4-byte keys, 6 items and 2 stages for 8-byte keys (measured the
// fastest on GB300: at 6 items a warp's 8-byte shared-memory reads meet 4-way bank conflicts where
// 8 items give 16-way ones), unless PS_PASS_STAGES picks another compiled ring depth for that item
// count, or ps_tune_set or ps_autotune choose otherwise.  Packed as pass_variant(ipt, stages).
int default_pass_ipt(int key_bytes) { return key_bytes == 8 ? 6 : 8; }

bool known_variant(int ipt, int stages) {
  for (int i = 0; i < kPassVariants; ++i)
    if (kPassVariantIpt[i] == ipt && kPassVariantStages[i] == stages) return true;
  return false;
}

int default_variant(int key_bytes) {
  static int stages = -1;
  if (stages < 0) {
    const char* e = std::getenv("PS_PASS_STAGES");
    stages = e ? std::atoi(e) : 2;
  }
  const int ipt = default_pass_ipt(key_bytes);
  return known_variant(ipt, stages) ? pass_variant(ipt, stages) : pass_variant(ipt, 2);
}

// Tuned configurations: a default per key type and payload choice (ps_tune_set), and entries per
// plain / segmented call and size bucket of the call's n (ps_autotune, ps_autotune_segmented),
// which take precedence.  0 = not set.
constexpr int kTuneBuckets = 4;
int tune_bucket(int64_t n) { return n < (1 << 20) ? 0 : n < (1 << 24) ? 1 : n < (1 << 28) ? 2 : 3; }
std::atomic<int> g_tune[4][2];                       // [key type][payload]
std::atomic<int> g_tune_bucket[4][2][2][kTuneBuckets];  // [key type][payload][segmented][bucket]
thread_local int t_variant_override = 0;  // set by the autotuner around its trial sorts
// Failure self-test (ps_selftest_level_pass_timeout): the poll bound of the level passes and
// whether the deepest one withholds a stage; set only around that entry point's sort.
thread_local uint32_t t_selftest_polls = 0;

void apply_pass_config(Ctx& c, int kt, bool vals, int64_t n, bool segmented) {
  int v = t_variant_override;
  if (!v) v = g_tune_bucket[kt][vals ? 1 : 0][segmented ? 1 : 0][tune_bucket(n)].load();
  if (!v) v = g_tune[kt][vals ? 1 : 0].load();
  if (!v) v = default_variant(key_bytes(kt));
  c.pass_ipt = v / 16;
  c.pass_stages = v % 16;
  c.merge_tile = c.pass_ipt * kMergeThreads;
}

ps_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PS_OK;
  if (e == cudaErrorMemoryAllocation) return PS_ERR_OUT_OF_MEMORY;
  return PS_ERR_CUDA;
}

#define PS_TRY(expr)                                \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return cuda_status(e_);  \
  } while (0)

ps_status check_args(int kt, const void* keys, const uint32_t* vals, int64_t n) {
  if (!launch_for(kt)) return PS_ERR_INVALID_ARG;
  if (n < 0) return PS_ERR_INVALID_ARG;
  if (n >= kMaxElems) return PS_ERR_UNSUPPORTED;
  if (n > 0 && (!keys || ((uintptr_t)keys % (uintptr_t)key_bytes(kt)) != 0)) return PS_ERR_INVALID_ARG;
  if (vals && ((uintptr_t)vals & 3u) != 0) return PS_ERR_INVALID_ARG;
  return PS_OK;
}

// Plan header read-back.  A kernel writes the header into a mapped pinned host buffer (one per
// host thread and device) and the host waits on an event recorded after it.  A small
// device-to-host copy would instead queue on the copy engine behind whatever large copies other
// streams have in flight (e.g. the copy-out of the previous array in a pipelined caller).
struct HeaderMailbox {
  PlanHeader* host = nullptr;
  PlanHeader* dev = nullptr;
  cudaEvent_t ev = nullptr;
  ~HeaderMailbox() {
    if (ev) cudaEventDestroy(ev);
    if (host) cudaFreeHost(host);
  }
};
thread_local HeaderMailbox t_mailbox[kMaxDevices];

ps_status read_plan_header(const Ctx& c, int dev, PlanHeader& h) {
  if (dev < 0 || dev >= kMaxDevices) return PS_ERR_CUDA;
  HeaderMailbox& m = t_mailbox[dev];
  if (!m.host) {
    PS_TRY(cudaHostAlloc((void**)&m.host, sizeof(PlanHeader), cudaHostAllocMapped));
    PS_TRY(cudaHostGetDevicePointer((void**)&m.dev, m.host, 0));
    PS_TRY(cudaEventCreateWithFlags(&m.ev, cudaEventDisableTiming));
  }
  PS_TRY(launch_header_out(c, m.dev));
  PS_TRY(cudaEventRecord(m.ev, c.stream));
  PS_TRY(cudaEventSynchronize(m.ev));
  std::memcpy(&h, (const void*)m.host, sizeof(PlanHeader));
  return PS_OK;
}

// The counts the merge launches are sized with must fit the plan's arrays: subtree tasks
// (<= run_cap slots), large leaves (<= level_cap items, <= n tiles) and, per depth, level-pass
// items (<= level_cap) and tiles (a node of size s spans at most s / tile + 2 tiles).  A plan
// that breaks one of them is reported instead of launched.
bool plan_counts_ok(const Ctx& c, const PlanHeader& h, int64_t n) {
  if (h.runs < 1 || h.runs > n || (int64_t)h.runs + 1 > c.run_cap) return false;
  if ((uint64_t)h.n_small > (uint64_t)c.run_cap) return false;
  if ((h.leaf_ctr >> 32) > (uint64_t)c.level_cap || (h.leaf_ctr & 0xffffffffull) > (uint64_t)n) return false;
  for (int d = 0; d < kMaxLevels; ++d) {
    const uint64_t items = h.level_ctr[d] >> 32, tiles = h.level_ctr[d] & 0xffffffffull;
    if (tiles == 0) continue;
    if (items > (uint64_t)c.level_cap) return false;
    if (tiles > (uint64_t)n / (uint64_t)c.merge_tile + 2ull * items + 1) return false;
  }
  return true;
}

// The whole pipeline.  With `an` set, stops after planning and reports the plan instead.
ps_status run(int kt, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets, int64_t count,
              bool segmented, void* ws, size_t ws_bytes, cudaStream_t s, AnalyzeOut* an, int tree = 0,
              int min_run = 1) {
  ps_status st = check_args(kt, keys, vals, n);
  if (st != PS_OK) return st;
  if (tree != PS_TREE_POWERSORT && tree != PS_TREE_PEEKSORT) return PS_ERR_INVALID_ARG;
  if (min_run < 1 || min_run > kMinRunMax) return PS_ERR_INVALID_ARG;
  if (min_run > 1 && tree != PS_TREE_POWERSORT) return PS_ERR_UNSUPPORTED;
  if (segmented && (!d_offsets || count < 1 || count >= ((int64_t)1 << 31))) return PS_ERR_INVALID_ARG;
  if (n == 0 || (n == 1 && !an)) {
    if (an) {
      if (an->runs) *an->runs = 0;
      if (an->cost) *an->cost = 0;
      if (an->starts) an->starts[0] = 0;
      if (an->power) an->power[0] = 0;
      if (an->stats) {
        std::memset(an->stats, 0, sizeof(ps_stats));
      }
    }
    return PS_OK;
  }
  Ctx c;
  const size_t need = carve(c, (uint8_t*)ws, kt, vals != nullptr, n, segmented, tree);
  if (!ws || ws_bytes < need || ((uintptr_t)ws & 255u)) return ws ? PS_ERR_OUT_OF_MEMORY : PS_ERR_INVALID_ARG;
  int dev = 0;
  PS_TRY(cudaGetDevice(&dev));
  c.stream = s;
  c.kt = kt;
  c.key_bytes = key_bytes(kt);
  c.has_vals = vals != nullptr;
  c.n = n;
  c.offsets = segmented ? d_offsets : nullptr;
  c.count = segmented ? (int32_t)count : 1;
  c.k[0] = keys;
  c.v[0] = vals;
  c.lib_status = lib_status_word(dev);
  c.min_run = min_run;
  apply_pass_config(c, kt, vals != nullptr, n, segmented);
  const KeyLaunch* kl = launch_for(kt);

  PS_TRY(cudaMemsetAsync(c.hdr, 0, sizeof(PlanHeader), s));
  const uint64_t eb = (uint64_t)c.key_bytes + (c.has_vals ? 4u : 0u);  // bytes per element
  {
    StageTimer t(0, s);
    if (segmented) PS_TRY(launch_check_offsets(c));
    PS_TRY(kl->detect(c));
    t.done((uint64_t)n * c.key_bytes, (segmented ? 1 : 0) + (min_run > 1 ? 5 : 3));
  }
  {
    StageTimer t(1, s);
    PS_TRY(launch_meta_stages(c));
    t.done(0, (uint64_t)meta_launches(c));
  }
  if (an && an->stats) {
    PS_TRY(cudaMemsetAsync(c.d_entropy, 0, sizeof(double), s));
    PS_TRY(launch_entropy(c, c.d_entropy));
    g_launches += 1;
  }
  PlanHeader h;
  st = read_plan_header(c, dev, h);
  if (st != PS_OK) return st;
  g_launches += 1;
  if (h.status & kDevBadOffsets) return PS_ERR_INVALID_ARG;
  if (h.status & kDevTimeout) return PS_ERR_TIMEOUT;
  if (h.status & kDevInternal) return PS_ERR_INTERNAL;
  if (h.status & kDevTooManyRuns) return PS_ERR_UNSUPPORTED;
  const int32_t r = h.runs;
  if (!plan_counts_ok(c, h, n)) return PS_ERR_INTERNAL;

  if (an) {
    if (an->runs) *an->runs = r;
    if (an->cost) *an->cost = h.cost;
    const size_t R1 = (size_t)r + 1;
    // run starts are 32-bit on the device (n < 2^32): copied into the upper half of the caller's
    // int64 array, then widened in place from the front
    if (an->starts) PS_TRY(cudaMemcpyAsync((uint32_t*)an->starts + R1, c.S, R1 * 4, cudaMemcpyDeviceToHost, s));
    if (an->desc) PS_TRY(cudaMemcpyAsync(an->desc, c.run_desc, (size_t)r, cudaMemcpyDeviceToHost, s));
    if (an->power) PS_TRY(cudaMemcpyAsync(an->power, c.P, R1, cudaMemcpyDeviceToHost, s));
    if (an->leaf_depth) PS_TRY(cudaMemcpyAsync(an->leaf_depth, c.ldepth, (size_t)r, cudaMemcpyDeviceToHost, s));
    if (an->node_left) PS_TRY(cudaMemcpyAsync(an->node_left, c.nodeL, R1 * 4, cudaMemcpyDeviceToHost, s));
    if (an->node_right) PS_TRY(cudaMemcpyAsync(an->node_right, c.nodeR, R1 * 4, cudaMemcpyDeviceToHost, s));
    if (an->node_depth) PS_TRY(cudaMemcpyAsync(an->node_depth, c.ndepth, R1, cudaMemcpyDeviceToHost, s));
    double ent = 0.0;
    if (an->stats) PS_TRY(cudaMemcpyAsync(&ent, c.d_entropy, sizeof(double), cudaMemcpyDeviceToHost, s));
    PS_TRY(cudaStreamSynchronize(s));
    if (an->starts) {
      const uint32_t* narrow = (const uint32_t*)an->starts + R1;
      for (size_t i = 0; i < R1; ++i) an->starts[i] = (int64_t)narrow[i];
    }
    if (an->stats) {
      ps_stats* o = an->stats;
      o->n = n;
      o->runs = r;
      o->merge_cost = h.cost;
      const double dn = (double)n;
      o->entropy_bits = (dn * std::log2(dn) - ent) / dn;
      o->max_depth = h.max_leaf_depth;
      int passes = 0;
      for (int d = 0; d < kMaxLevels; ++d)
        if (h.level_ctr[d] & 0xffffffffull) ++passes;
      o->merge_passes = passes;
      o->small_tasks = h.n_small;
    }
    return PS_OK;
  }

  if (h.n_small) {
    StageTimer t(2, s);
    PS_TRY(kl->small(c, h.n_small));
    t.done(2 * h.small_elems * eb, 1);
  }
  const uint32_t leaf_tiles = (uint32_t)(h.leaf_ctr & 0xffffffffull);
  if (leaf_tiles) {
    StageTimer t(3, s);
    PS_TRY(kl->place(c, (uint32_t)(h.leaf_ctr >> 32), leaf_tiles));
    t.done(2 * h.place_elems * eb, 1);
  }
  if (t_selftest_polls) {
    c.poll_limit = t_selftest_polls;
    for (int d = kMaxLevels - 1; d >= 0 && c.withhold_depth < 0; --d)
      if (h.level_ctr[d] & 0xffffffffull) c.withhold_depth = d;
    if (c.withhold_depth < 0) return PS_ERR_UNSUPPORTED;  // no large merge to withhold a stage of
  }
  for (int d = kMaxLevels - 1; d >= 0; --d) {
    const uint32_t items = (uint32_t)(h.level_ctr[d] >> 32), tiles = (uint32_t)(h.level_ctr[d] & 0xffffffffull);
    if (tiles == 0) continue;
    StageTimer t(5, s);
    PS_TRY(kl->merge(c, d, items, tiles));
    t.done(2 * h.level_elems[d] * eb, 1);
  }
  return PS_OK;
}

// Device-driven pipeline: no host round trip between planning and merging.  Every launch after
// planning takes its work count from the plan header on the device (persistent grids; level
// passes for every depth the tree can have, empty ones return at once), so the call only queues
// work and can be captured into a CUDA graph.  Binary passes; errors found on the device reach
// ps_stream_status, and with rejected segment offsets nothing is moved.
ps_status run_async(int kt, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets, int64_t count,
                    bool segmented, void* ws, size_t ws_bytes, cudaStream_t s, int tree, int64_t max_segment = 0) {
  ps_status st = check_args(kt, keys, vals, n);
  if (st != PS_OK) return st;
  if (tree != PS_TREE_POWERSORT && tree != PS_TREE_PEEKSORT) return PS_ERR_INVALID_ARG;
  if (max_segment < 0 || (!segmented && max_segment > 0 && n > max_segment)) return PS_ERR_INVALID_ARG;
  if (segmented && (!d_offsets || count < 1 || count >= ((int64_t)1 << 31))) return PS_ERR_INVALID_ARG;
  if (n <= 1) return PS_OK;
  Ctx c;
  const size_t need = carve(c, (uint8_t*)ws, kt, vals != nullptr, n, segmented, tree);
  if (!ws || ws_bytes < need || ((uintptr_t)ws & 255u)) return ws ? PS_ERR_OUT_OF_MEMORY : PS_ERR_INVALID_ARG;
  int dev = 0;
  PS_TRY(cudaGetDevice(&dev));
  c.stream = s;
  c.kt = kt;
  c.key_bytes = key_bytes(kt);
  c.has_vals = vals != nullptr;
  c.n = n;
  c.offsets = segmented ? d_offsets : nullptr;
  c.count = segmented ? (int32_t)count : 1;
  c.max_segment = max_segment;
  c.k[0] = keys;
  c.v[0] = vals;
  c.lib_status = lib_status_word(dev);
  if (!c.lib_status) return PS_ERR_CUDA;
  apply_pass_config(c, kt, vals != nullptr, n, segmented);
  const KeyLaunch* kl = launch_for(kt);
  // Deepest node a level pass can meet: depth < power (powers grow from a node to its children)
  // and power <= floor(lg n) + 1 for Alg. 2; the plan's limit for Alg. 1.  Only nodes larger than
  // sub_lim reach a level pass, and a node of power p spans fewer than 4 n_s / 2^p elements of its
  // segment (n_s <= n).  The boundaries inside its range all have power >= p, so the midpoints
  // c_L < .. < c_R' of its runs (normalised by n_s) lie in one dyadic interval of length 2^(1-p).
  // Its first run starts after 2 c_L - c_(L+1) and its last ends before 2 c_R' - c_(R'-1) (a run's
  // half length is below the distance to its neighbour's midpoint), so its size / n_s is below
  // 2 (c_R' - c_L) - (c_(R'-1) - c_(L+1)) <= 2 (c_R' - c_L) with three runs or more, and equals
  // 2 (c_R' - c_L) with two; both are below 2 * 2^(1-p).  So 2^p < 4 n_s / sub_lim for the
  // longest segment n_s (n, or the caller's checked bound), and launches for deeper levels would
  // find no node.
  int maxd = kMaxLevels - 1;
  if (tree == PS_TREE_POWERSORT) {
    maxd = 0;
    while (maxd < kMaxLevels - 1 && ((int64_t)1 << (maxd + 1)) <= n) ++maxd;
    const int64_t ns = max_segment > 0 ? std::min(max_segment, n) : n;  // longest segment
    int pmax = 0;  // smallest p with 2^p >= 4 ns / sub_lim: every level-pass node has power < pmax
    while (pmax < 62 && ((int64_t)c.sub_lim << pmax) < 4 * ns) ++pmax;
    maxd = std::min(maxd, std::max(pmax - 2, 0));
  }
  PS_TRY(cudaMemsetAsync(c.hdr, 0, sizeof(PlanHeader), s));
  {
    StageTimer t(0, s);
    if (segmented) PS_TRY(launch_check_offsets(c));
    PS_TRY(kl->detect(c));
    t.done(0, segmented ? 4 : 3);
  }
  {
    StageTimer t(1, s);
    PS_TRY(launch_meta_stages(c));
    t.done(0, (uint64_t)meta_launches(c));
  }
  {
    StageTimer t(2, s);
    PS_TRY(kl->small(c, kCountOnDevice));
    t.done(0, 2);  // the one-task grid and the persistent kernel for any tasks beyond it
  }
  {
    StageTimer t(3, s);
    PS_TRY(kl->place(c, kCountOnDevice, kCountOnDevice));
    t.done(0, 1);
  }
  {
    StageTimer t(5, s);
    for (int d = maxd; d >= 0; --d) PS_TRY(kl->merge(c, d, kCountOnDevice, kCountOnDevice));
    t.done(0, (uint64_t)maxd + 1);
  }
  PS_TRY(launch_status_out(c));
  g_launches += 1;
  return PS_OK;
}

ps_status with_pool(int kt, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets, int64_t count,
                    bool segmented, cudaStream_t s, AnalyzeOut* an) {
  ps_status st = check_args(kt, keys, vals, n);
  if (st != PS_OK) return st;
  if (n <= 1 && !an) return PS_OK;
  int dev = 0;
  PS_TRY(cudaGetDevice(&dev));
  cudaMemPool_t pool = lib_pool(dev);
  if (!pool) return PS_ERR_CUDA;
  Ctx tmp;
  const size_t bytes = carve(tmp, nullptr, kt, vals != nullptr, n, segmented);
  void* ws = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&ws, bytes, pool, s);
  if (e != cudaSuccess) return PS_ERR_OUT_OF_MEMORY;
  st = run(kt, keys, vals, n, d_offsets, count, segmented, ws, bytes, s, an);
  e = cudaFreeAsync(ws, s);
  if (st == PS_OK && e != cudaSuccess) st = PS_ERR_CUDA;
  return st;
}

// ---- host merge cost (ps_merge_cost) --------------------------------------------------------
// Node powers from the first 62 fractional bits of the normalised midpoints (exact for
// n <= 2^62, since then b - a >= 1/n), the Cartesian tree by a stack, depths top-down by power.
ps_status host_merge_cost(const int64_t* len, int64_t r, uint64_t* out) {
  std::vector<uint64_t> S((size_t)r + 1, 0);
  for (int64_t i = 0; i < r; ++i) {
    if (len[i] <= 0) return PS_ERR_INVALID_ARG;
    S[i + 1] = S[i] + (uint64_t)len[i];
    if (S[i + 1] > ((uint64_t)1 << 62)) return PS_ERR_INVALID_ARG;
  }
  const unsigned __int128 two_n = (unsigned __int128)(2 * S[r]);
  std::vector<int> P((size_t)r + 1, 0);
  for (int64_t j = 1; j < r; ++j) {
    const unsigned __int128 l2 = (unsigned __int128)(S[j - 1] + S[j]);
    const unsigned __int128 r2 = (unsigned __int128)(S[j] + S[j + 1]);
    const uint64_t x = (uint64_t)((l2 << 62) / two_n), y = (uint64_t)((r2 << 62) / two_n);
    P[j] = __builtin_clzll(x ^ y) - 1;
  }
  // parent of every boundary in the min-Cartesian tree (sentinels 0 and r have power 0)
  std::vector<int64_t> left((size_t)r + 1, 0), right((size_t)r + 1, r), stk;
  for (int64_t j = 0; j <= r; ++j) {
    while (!stk.empty() && P[stk.back()] >= P[j]) stk.pop_back();
    left[j] = stk.empty() ? 0 : stk.back();
    stk.push_back(j);
  }
  stk.clear();
  for (int64_t j = r; j >= 0; --j) {
    while (!stk.empty() && P[stk.back()] >= P[j]) stk.pop_back();
    right[j] = stk.empty() ? r : stk.back();
    stk.push_back(j);
  }
  // depths in increasing power order (a parent's power is smaller than its child's)
  std::vector<std::vector<int64_t>> by_power(64);
  for (int64_t j = 1; j < r; ++j) by_power[P[j]].push_back(j);
  std::vector<int> depth((size_t)r + 1, 0);
  for (int p = 1; p < 64; ++p)
    for (int64_t j : by_power[p]) {
      const int64_t L = left[j], R = right[j];
      const int pl = P[L], pr = P[R];
      if (pl == 0 && pr == 0) depth[j] = 0;
      else depth[j] = depth[pl > pr ? L : R] + 1;
    }
  uint64_t cost = 0;
  for (int64_t i = 0; i < r; ++i) {
    const int pl = P[i], pr = P[i + 1];
    const int d = (pl == 0 && pr == 0) ? 0 : depth[pl > pr ? i : i + 1] + 1;
    cost += (uint64_t)d * (uint64_t)len[i];
  }
  *out = cost;
  return PS_OK;
}

}  // namespace

extern "C" {

size_t ps_workspace_size(int key_type, int has_vals, int64_t n, int segmented) {
  if (!launch_for(key_type) || n < 0) return 0;
  Ctx c;
  return carve(c, nullptr, key_type, has_vals != 0, n, segmented != 0);
}

ps_status ps_sort_ws(int key_type, void* keys, uint32_t* vals, int64_t n, void* workspace,
                     size_t workspace_bytes, void* stream) {
  return run(key_type, keys, vals, n, nullptr, 1, false, workspace, workspace_bytes, (cudaStream_t)stream,
             nullptr);
}

ps_status ps_sort(int key_type, void* keys, uint32_t* vals, int64_t n, void* stream) {
  return with_pool(key_type, keys, vals, n, nullptr, 1, false, (cudaStream_t)stream, nullptr);
}

ps_status ps_sort_i32(int32_t* keys, uint32_t* vals, int64_t n, void* stream) {
  return ps_sort(PS_KEY_I32, keys, vals, n, stream);
}
ps_status ps_sort_u32(uint32_t* keys, uint32_t* vals, int64_t n, void* stream) {
  return ps_sort(PS_KEY_U32, keys, vals, n, stream);
}
ps_status ps_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, void* stream) {
  return ps_sort(PS_KEY_U64, keys, vals, n, stream);
}
ps_status ps_sort_f32(float* keys, uint32_t* vals, int64_t n, void* stream) {
  return ps_sort(PS_KEY_F32, keys, vals, n, stream);
}

ps_status ps_sort_segmented_ws(int key_type, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets,
                               int64_t count, void* workspace, size_t workspace_bytes, void* stream) {
  return run(key_type, keys, vals, n, d_offsets, count, true, workspace, workspace_bytes, (cudaStream_t)stream,
             nullptr);
}

ps_status ps_sort_segmented(int key_type, void* keys, uint32_t* vals, const int64_t* d_offsets, int64_t count,
                            void* stream) {
  if (!d_offsets || count < 1) return PS_ERR_INVALID_ARG;
  int64_t n = 0;
  cudaStream_t s = (cudaStream_t)stream;
  PS_TRY(cudaMemcpyAsync(&n, d_offsets + count, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PS_TRY(cudaStreamSynchronize(s));
  return with_pool(key_type, keys, vals, n, d_offsets, count, true, s, nullptr);
}

ps_status ps_merge_cost(const int64_t* run_lengths, int64_t r, uint64_t* out_cost) {
  if (!run_lengths || !out_cost || r <= 0) return PS_ERR_INVALID_ARG;
  return host_merge_cost(run_lengths, r, out_cost);
}

ps_status ps_analyze(int key_type, const void* keys, int64_t n, const int64_t* d_offsets, int64_t count,
                     void* workspace, size_t workspace_bytes, int64_t* out_runs, uint64_t* out_cost,
                     int64_t* starts, uint8_t* desc, uint8_t* power, uint8_t* leaf_depth, int32_t* node_left,
                     int32_t* node_right, uint8_t* node_depth, void* stream) {
  AnalyzeOut an{out_runs, out_cost, starts, desc, power, leaf_depth, node_left, node_right, node_depth, nullptr};
  const bool seg = d_offsets != nullptr;
  return run(key_type, const_cast<void*>(keys), nullptr, n, d_offsets, seg ? count : 1, seg, workspace,
             workspace_bytes, (cudaStream_t)stream, &an);
}

ps_status ps_selftest_wait_timeout(uint32_t polls, void* stream) {
  int dev = 0;
  PS_TRY(cudaGetDevice(&dev));
  uint32_t* w = lib_status_word(dev);
  if (!w) return PS_ERR_CUDA;
  PS_TRY(launch_wait_timeout_probe(polls, w, (cudaStream_t)stream));
  g_launches += 1;
  return PS_OK;
}

ps_status ps_selftest_level_pass_timeout(int key_type, void* keys, uint32_t* vals, int64_t n, uint32_t polls,
                                         void* workspace, size_t workspace_bytes, void* stream) {
  if (polls == 0) return PS_ERR_INVALID_ARG;
  t_selftest_polls = polls;
  const ps_status st = run(key_type, keys, vals, n, nullptr, 1, false, workspace, workspace_bytes,
                           (cudaStream_t)stream, nullptr);
  t_selftest_polls = 0;
  return st;
}

ps_status ps_tune_set(int key_type, int has_vals, int items_per_thread, int stages) {
  if (!launch_for(key_type)) return PS_ERR_INVALID_ARG;
  const int hv = has_vals ? 1 : 0;
  if (items_per_thread == 0 && stages == 0) {  // back to the default, tuned entries cleared
    g_tune[key_type][hv].store(0);
    for (int sg = 0; sg < 2; ++sg)
      for (int b = 0; b < kTuneBuckets; ++b) g_tune_bucket[key_type][hv][sg][b].store(0);
    return PS_OK;
  }
  if (!known_variant(items_per_thread, stages)) return PS_ERR_UNSUPPORTED;
  g_tune[key_type][hv].store(pass_variant(items_per_thread, stages));
  for (int sg = 0; sg < 2; ++sg)
    for (int b = 0; b < kTuneBuckets; ++b) g_tune_bucket[key_type][hv][sg][b].store(0);
  return PS_OK;
}

ps_status ps_tune_get(int key_type, int has_vals, int* items_per_thread, int* stages) {
  if (!launch_for(key_type) || !items_per_thread || !stages) return PS_ERR_INVALID_ARG;
  Ctx c;
  apply_pass_config(c, key_type, has_vals != 0, 0, false);
  *items_per_thread = c.pass_ipt;
  *stages = c.pass_stages;
  return PS_OK;
}

ps_status ps_tune_get_for(int key_type, int has_vals, int64_t n, int segmented, int* items_per_thread, int* stages) {
  if (!launch_for(key_type) || !items_per_thread || !stages || n < 0) return PS_ERR_INVALID_ARG;
  Ctx c;
  apply_pass_config(c, key_type, has_vals != 0, n, segmented != 0);
  *items_per_thread = c.pass_ipt;
  *stages = c.pass_stages;
  return PS_OK;
}

}  // extern "C"

namespace {

// Time every level-pass configuration on copies of keys/vals (plain when d_offsets is null, else
// segmented with the caller's device offsets) and store the fastest for the call's kind and size.
ps_status autotune(int key_type, const void* keys, const uint32_t* vals, int64_t n, const int64_t* d_offsets,
                   int64_t count, ps_tune_result* out, cudaStream_t s) {
  ps_status st = check_args(key_type, keys, vals, n);
  if (st != PS_OK) return st;
  const bool seg = d_offsets != nullptr;
  if (!out || n < 2 || (seg && (count < 1 || count >= ((int64_t)1 << 31)))) return PS_ERR_INVALID_ARG;
  int dev = 0;
  PS_TRY(cudaGetDevice(&dev));
  cudaMemPool_t pool = lib_pool(dev);
  if (!pool) return PS_ERR_CUDA;
  const size_t kb = (size_t)key_bytes(key_type);
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t kbytes = up((size_t)n * kb + 16), vbytes = vals ? up((size_t)n * 4 + 16) : 0;
  Ctx tmp;
  const size_t wbytes = carve(tmp, nullptr, key_type, vals != nullptr, n, seg);
  uint8_t* base = nullptr;
  if (cudaMallocFromPoolAsync((void**)&base, kbytes + vbytes + wbytes, pool, s) != cudaSuccess)
    return PS_ERR_OUT_OF_MEMORY;
  void* dk = base;
  uint32_t* dv = vals ? (uint32_t*)(base + kbytes) : nullptr;
  void* ws = base + kbytes + vbytes;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::memset(out, 0, sizeof(*out));
  int best = -1;
  double best_ms = 0.0;
  constexpr int kReps = 3;
  for (int i = 0; i < kPassVariants && st == PS_OK; ++i) {
    t_variant_override = pass_variant(kPassVariantIpt[i], kPassVariantStages[i]);
    double t[kReps];
    for (int rep = 0; rep <= kReps && st == PS_OK; ++rep) {  // rep 0 warms up
      cudaError_t e = cudaMemcpyAsync(dk, keys, (size_t)n * kb, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess && dv) e = cudaMemcpyAsync(dv, vals, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      if (e != cudaSuccess) {
        st = cuda_status(e);
        break;
      }
      st = run(key_type, dk, dv, n, d_offsets, seg ? count : 1, seg, ws, wbytes, s, nullptr);
      if (st != PS_OK) break;
      e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) st = cuda_status(e);
      if (rep > 0) t[rep - 1] = ms;
    }
    if (st != PS_OK) break;
    std::sort(t, t + kReps);
    const double med = t[kReps / 2];
    out->variant_items[i] = kPassVariantIpt[i];
    out->variant_stages[i] = kPassVariantStages[i];
    out->variant_ms[i] = med;
    out->n_variants = i + 1;
    if (best < 0 || med < best_ms) {
      best = i;
      best_ms = med;
    }
  }
  t_variant_override = 0;
  cudaFreeAsync(base, s);
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PS_OK) return st;
  g_tune_bucket[key_type][vals ? 1 : 0][seg ? 1 : 0][tune_bucket(n)].store(
      pass_variant(kPassVariantIpt[best], kPassVariantStages[best]));
  out->items_per_thread = kPassVariantIpt[best];
  out->stages = kPassVariantStages[best];
  return PS_OK;
}

}  // namespace

extern "C" {

ps_status ps_autotune(int key_type, const void* keys, const uint32_t* vals, int64_t n, ps_tune_result* out,
                      void* stream) {
  return autotune(key_type, keys, vals, n, nullptr, 1, out, (cudaStream_t)stream);
}

ps_status ps_autotune_segmented(int key_type, const void* keys, const uint32_t* vals, int64_t n,
                                const int64_t* d_offsets, int64_t count, ps_tune_result* out, void* stream) {
  if (!d_offsets) return PS_ERR_INVALID_ARG;
  return autotune(key_type, keys, vals, n, d_offsets, count, out, (cudaStream_t)stream);
}

ps_status ps_sort_async_ws(int key_type, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets,
                           int64_t count, int tree, void* workspace, size_t workspace_bytes, void* stream) {
  const bool seg = d_offsets != nullptr;
  return run_async(key_type, keys, vals, n, d_offsets, seg ? count : 1, seg, workspace, workspace_bytes,
                   (cudaStream_t)stream, tree);
}

ps_status ps_sort_async_bounded_ws(int key_type, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets,
                                   int64_t count, int64_t max_segment, void* workspace, size_t workspace_bytes,
                                   void* stream) {
  if (max_segment < 1) return PS_ERR_INVALID_ARG;
  const bool seg = d_offsets != nullptr;
  return run_async(key_type, keys, vals, n, d_offsets, seg ? count : 1, seg, workspace, workspace_bytes,
                   (cudaStream_t)stream, PS_TREE_POWERSORT, max_segment);
}

size_t ps_workspace_size_tree(int key_type, int has_vals, int64_t n, int segmented, int tree) {
  if (!launch_for(key_type) || n < 0 || (tree != PS_TREE_POWERSORT && tree != PS_TREE_PEEKSORT)) return 0;
  Ctx c;
  return carve(c, nullptr, key_type, has_vals != 0, n, segmented != 0, tree);
}

ps_status ps_sort_tree_ws(int key_type, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets,
                          int64_t count, int tree, void* workspace, size_t workspace_bytes, void* stream) {
  const bool seg = d_offsets != nullptr;
  return run(key_type, keys, vals, n, d_offsets, seg ? count : 1, seg, workspace, workspace_bytes,
             (cudaStream_t)stream, nullptr, tree);
}

ps_status ps_analyze_tree(int key_type, const void* keys, int64_t n, const int64_t* d_offsets, int64_t count,
                          int tree, void* workspace, size_t workspace_bytes, int64_t* out_runs, uint64_t* out_cost,
                          int64_t* starts, uint8_t* desc, uint8_t* power, uint8_t* leaf_depth, int32_t* node_left,
                          int32_t* node_right, uint8_t* node_depth, void* stream) {
  AnalyzeOut an{out_runs, out_cost, starts, desc, power, leaf_depth, node_left, node_right, node_depth, nullptr};
  const bool seg = d_offsets != nullptr;
  return run(key_type, const_cast<void*>(keys), nullptr, n, d_offsets, seg ? count : 1, seg, workspace,
             workspace_bytes, (cudaStream_t)stream, &an, tree);
}

ps_status ps_sort_minrun_ws(int key_type, void* keys, uint32_t* vals, int64_t n, const int64_t* d_offsets,
                            int64_t count, int min_run, void* workspace, size_t workspace_bytes, void* stream) {
  const bool seg = d_offsets != nullptr;
  return run(key_type, keys, vals, n, d_offsets, seg ? count : 1, seg, workspace, workspace_bytes,
             (cudaStream_t)stream, nullptr, PS_TREE_POWERSORT, min_run);
}

ps_status ps_analyze_minrun(int key_type, const void* keys, int64_t n, const int64_t* d_offsets, int64_t count,
                            int min_run, void* workspace, size_t workspace_bytes, int64_t* out_runs,
                            uint64_t* out_cost, int64_t* starts, uint8_t* desc, uint8_t* power, uint8_t* leaf_depth,
                            int32_t* node_left, int32_t* node_right, uint8_t* node_depth, void* stream) {
  AnalyzeOut an{out_runs, out_cost, starts, desc, power, leaf_depth, node_left, node_right, node_depth, nullptr};
  const bool seg = d_offsets != nullptr;
  return run(key_type, const_cast<void*>(keys), nullptr, n, d_offsets, seg ? count : 1, seg, workspace,
             workspace_bytes, (cudaStream_t)stream, &an, PS_TREE_POWERSORT, min_run);
}

ps_status ps_debug_bounds(unsigned long long* hits) {
  if (!hits) return PS_ERR_INVALID_ARG;
  if (!kBoundsChecked) return PS_ERR_UNSUPPORTED;
  const unsigned long long parts[3] = {bounds_hits_meta(), bounds_hits_keys32(), bounds_hits_keys64()};
  unsigned long long sum = 0;
  for (unsigned long long x : parts) {
    if (x == ~0ull) return PS_ERR_CUDA;
    sum += x;
  }
  *hits = sum;
  return PS_OK;
}

ps_status ps_sort_stats(int key_type, const void* keys, int64_t n, ps_stats* out, void* stream) {
  if (!out) return PS_ERR_INVALID_ARG;
  AnalyzeOut an{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, out};
  return with_pool(key_type, const_cast<void*>(keys), nullptr, n, nullptr, 1, false, (cudaStream_t)stream, &an);
}

ps_status ps_stream_status(void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return PS_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PS_ERR_CUDA;
  uint32_t* w = lib_status_word(dev);
  if (!w) return PS_ERR_CUDA;
  uint32_t v = 0;
  if (cudaMemcpy(&v, w, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PS_ERR_CUDA;
  if (v) {
    if (cudaMemset(w, 0, 4) != cudaSuccess) return PS_ERR_CUDA;
    if (v & kDevBadOffsets) return PS_ERR_INVALID_ARG;
    if (v & kDevTimeout) return PS_ERR_TIMEOUT;
    if (v & kDevInternal) return PS_ERR_INTERNAL;
    if (v & kDevTooManyRuns) return PS_ERR_UNSUPPORTED;
    return PS_ERR_INTERNAL;
  }
  return PS_OK;
}

ps_status ps_sort_host_ws(int key_type, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                          uint32_t* vals_out, int64_t n, void* dev_keys, uint32_t* dev_vals, void* workspace,
                          size_t workspace_bytes, void* stream) {
  if (!launch_for(key_type) || n < 0) return PS_ERR_INVALID_ARG;
  if (n >= kMaxElems) return PS_ERR_UNSUPPORTED;
  if (n > 0 && (!keys_in || !keys_out || !dev_keys)) return PS_ERR_INVALID_ARG;
  if ((vals_in == nullptr) != (vals_out == nullptr) || (vals_in != nullptr) != (dev_vals != nullptr))
    return PS_ERR_INVALID_ARG;
  if (n == 0) return PS_OK;
  const size_t kb = (size_t)key_bytes(key_type);
  cudaStream_t s = (cudaStream_t)stream;
  PS_TRY(cudaMemcpyAsync(dev_keys, keys_in, (size_t)n * kb, cudaMemcpyHostToDevice, s));
  if (dev_vals) PS_TRY(cudaMemcpyAsync(dev_vals, vals_in, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  // device-driven: no host round trip, so the caller's next call (on another stream) is queued
  // while this array is still being copied in
  const ps_status st = run_async(key_type, dev_keys, dev_vals, n, nullptr, 1, false, workspace, workspace_bytes, s,
                                 PS_TREE_POWERSORT);
  if (st != PS_OK) return st;
  PS_TRY(cudaMemcpyAsync(keys_out, dev_keys, (size_t)n * kb, cudaMemcpyDeviceToHost, s));
  if (dev_vals) PS_TRY(cudaMemcpyAsync(vals_out, dev_vals, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  return PS_OK;
}

ps_status ps_sort_host(int key_type, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                       uint32_t* vals_out, int64_t n, void* stream) {
  if (!launch_for(key_type) || n < 0) return PS_ERR_INVALID_ARG;
  if (n >= kMaxElems) return PS_ERR_UNSUPPORTED;
  if (n > 0 && (!keys_in || !keys_out)) return PS_ERR_INVALID_ARG;
  if ((vals_in == nullptr) != (vals_out == nullptr)) return PS_ERR_INVALID_ARG;
  const size_t kb = (size_t)key_bytes(key_type);
  if (n <= 1) {
    if (n == 1) {
      std::memmove(keys_out, keys_in, kb);
      if (vals_in) std::memmove(vals_out, vals_in, 4);
    }
    return PS_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  PS_TRY(cudaGetDevice(&dev));
  cudaMemPool_t pool = lib_pool(dev);
  if (!pool) return PS_ERR_CUDA;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t kbytes = up((size_t)n * kb + 16), vbytes = vals_in ? up((size_t)n * 4 + 16) : 0;
  Ctx tmp;
  const size_t wbytes = carve(tmp, nullptr, key_type, vals_in != nullptr, n, false);
  uint8_t* base = nullptr;
  if (cudaMallocFromPoolAsync((void**)&base, kbytes + vbytes + wbytes, pool, s) != cudaSuccess)
    return PS_ERR_OUT_OF_MEMORY;
  void* dk = base;
  uint32_t* dv = vals_in ? (uint32_t*)(base + kbytes) : nullptr;
  void* ws = base + kbytes + vbytes;
  ps_status st = PS_OK;
  cudaError_t e = cudaMemcpyAsync(dk, keys_in, (size_t)n * kb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && dv) e = cudaMemcpyAsync(dv, vals_in, (size_t)n * 4, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) st = cuda_status(e);
  if (st == PS_OK) st = run(key_type, dk, dv, n, nullptr, 1, false, ws, wbytes, s, nullptr);
  if (st == PS_OK) {
    e = cudaMemcpyAsync(keys_out, dk, (size_t)n * kb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && dv) e = cudaMemcpyAsync(vals_out, dv, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_status(e);
  }
  cudaFreeAsync(base, s);
  e = cudaStreamSynchronize(s);
  if (st == PS_OK && e != cudaSuccess) st = PS_ERR_CUDA;
  return st;
}

ps_status ps_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& p : g_prof_pending) {
    cudaEventSynchronize(p.b);  // the events are reused
    prof_release(p.dev, p.a);
    prof_release(p.dev, p.b);
  }
  g_prof_pending.clear();
  for (int i = 0; i < kStages; ++i) {
    g_prof_ms[i] = 0;
    g_prof_launch[i] = 0;
    g_prof_bytes[i] = 0;
  }
  g_prof_on = on ? 1 : 0;
  return PS_OK;
}

ps_status ps_profile_read(ps_profile* out) {
  if (!out) return PS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ps_status st = PS_OK;
  for (auto& p : g_prof_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess)
      st = PS_ERR_CUDA;
    g_prof_ms[p.stage] += ms;
    g_prof_launch[p.stage] += p.launches;
    g_prof_bytes[p.stage] += p.bytes;
    prof_release(p.dev, p.a);
    prof_release(p.dev, p.b);
  }
  g_prof_pending.clear();
  for (int i = 0; i < kStages; ++i) {
    out->ms[i] = g_prof_ms[i];
    out->launches[i] = g_prof_launch[i];
    out->bytes[i] = g_prof_bytes[i];
  }
  return st;
}

uint64_t ps_launch_count(void) { return g_launches.load(); }

const char* ps_status_string(ps_status status) {
  switch (status) {
    case PS_OK: return "ok";
    case PS_ERR_INVALID_ARG: return "invalid argument";
    case PS_ERR_UNSUPPORTED: return "unsupported size (n >= 2^32, or 2^31 - 1 runs or more)";
    case PS_ERR_OUT_OF_MEMORY: return "out of device memory / workspace too small";
    case PS_ERR_CUDA: return "CUDA runtime error";
    case PS_ERR_TIMEOUT: return "a bounded device wait timed out";
    case PS_ERR_INTERNAL: return "internal error";
  }
  return "unknown status";
}

int ps_version(void) { return 100; }

}  // extern "C"

// =============================================================================================
// Allocation-free entry point (ps_sort_noalloc).
//
// Some callers cannot allocate device memory while they run: cudaMalloc / cudaFree may
// synchronize the whole device (stalling every other stream of a latency-critical loop), an
// allocation can fail once a fixed memory budget has been handed out, and hosts that manage all
// device memory through their own allocator (inference servers, plugins inside another
// framework) forbid stray allocations.  For them this entry point sorts small arrays with all
// of its scratch in one fixed array of device memory that lives in the library's module image:
// every GPU that loads the library holds it (kNoAllocScratchBytes, about 9 MiB) until the
// process exits.  Nothing here calls cudaMalloc, cudaFree or an allocating library routine.
//
// All calls share that array and it keeps whatever the last call left in it; every part that
// must start at zero is cleared on the stream at the start of each call.  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on the array and
// corrupt each other's results: serialize them.
// =============================================================================================
static constexpr size_t kNoAllocScratchBytes = (size_t)9 << 20;
static __device__ __align__(256) unsigned char ps_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
uint8_t* g_noalloc_addr[kMaxDevices] = {};

// Device address of ps_noalloc_scratch on the current device.  The symbol name in host code
// is only a host-side stand-in, so the address is looked up once per device, with that device
// current, and cached.
uint8_t* noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, ps_noalloc_scratch) != cudaSuccess || p == nullptr) return nullptr;
    g_noalloc_addr[dev] = (uint8_t*)p;
  }
  return g_noalloc_addr[dev];
}

ps_status run_noalloc(int kt, void* keys, uint32_t* vals, int64_t n, cudaStream_t s) {
  ps_status st = check_args(kt, keys, vals, n);
  if (st != PS_OK) return st;
  if (n > PS_NOALLOC_MAX_N) return PS_ERR_INVALID_ARG;
  if (n <= 1) return PS_OK;
  int dev = 0;
  PS_TRY(cudaGetDevice(&dev));
  uint8_t* scratch = noalloc_scratch(dev);
  if (!scratch) return PS_ERR_CUDA;
  Ctx c;
  const size_t need = carve(c, scratch, kt, vals != nullptr, n, false);
  if (need + 256 > kNoAllocScratchBytes) return PS_ERR_INTERNAL;
  c.stream = s;
  c.kt = kt;
  c.key_bytes = key_bytes(kt);
  c.has_vals = vals != nullptr;
  c.n = n;
  c.offsets = nullptr;
  c.count = 1;
  c.k[0] = keys;
  c.v[0] = vals;
  c.lib_status = (uint32_t*)(scratch + kNoAllocScratchBytes - 256);  // this entry's own status word
  apply_pass_config(c, kt, vals != nullptr, n, false);  // the level-pass configuration every other sort uses
  const KeyLaunch* kl = launch_for(kt);

  PS_TRY(cudaMemsetAsync(c.hdr, 0, sizeof(PlanHeader), s));
  PS_TRY(cudaMemsetAsync(c.lib_status, 0, 4, s));
  PS_TRY(kl->detect(c));
  PS_TRY(launch_meta_stages(c));
  g_launches += 3 + (uint64_t)meta_launches(c);
  PlanHeader h;
  PS_TRY(cudaMemcpyAsync(&h, c.hdr, sizeof(PlanHeader), cudaMemcpyDeviceToHost, s));
  PS_TRY(cudaStreamSynchronize(s));
  if (h.status & kDevTimeout) return PS_ERR_TIMEOUT;
  if (h.status & kDevInternal) return PS_ERR_INTERNAL;
  if (h.status & kDevTooManyRuns) return PS_ERR_UNSUPPORTED;
  // the same bounds on the plan's counts as every other entry point: a plan that broke them
  // would make the launches below write past their regions of the shared scratch array
  if (!plan_counts_ok(c, h, n)) return PS_ERR_INTERNAL;
  PS_TRY(kl->small(c, h.n_small));
  PS_TRY(kl->place(c, (uint32_t)(h.leaf_ctr >> 32), (uint32_t)(h.leaf_ctr & 0xffffffffull)));
  g_launches += (h.n_small ? 1 : 0) + ((h.leaf_ctr & 0xffffffffull) ? 1 : 0);
  for (int d = kMaxLevels - 1; d >= 0; --d) {
    const uint32_t items = (uint32_t)(h.level_ctr[d] >> 32), tiles = (uint32_t)(h.level_ctr[d] & 0xffffffffull);
    if (tiles == 0) continue;
    PS_TRY(kl->merge(c, d, items, tiles));
    g_launches += 1;
  }
  // device-posted errors of the merge stage come back synchronously: this entry point has no
  // library status word to defer them to
  uint32_t dev_status = 0;
  PS_TRY(cudaMemcpyAsync(&dev_status, c.lib_status, 4, cudaMemcpyDeviceToHost, s));
  PS_TRY(cudaStreamSynchronize(s));
  if (dev_status & kDevTimeout) return PS_ERR_TIMEOUT;
  if (dev_status) return PS_ERR_INTERNAL;
  return PS_OK;
}

}  // namespace

extern "C" ps_status ps_sort_noalloc(int key_type, void* keys, uint32_t* vals, int64_t n, void* stream) {
  return run_noalloc(key_type, keys, vals, n, (cudaStream_t)stream);
}
