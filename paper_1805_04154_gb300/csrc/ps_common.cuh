// Shared device definitions of the GB300 powersort library: key-order maps, tile constants,
// the plan header that the device fills for the host, and inline-PTX helpers for mbarriers and
// bulk (TMA) copies.  Everything here is sm_103a device code or plain host structs.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ps {

// ---------------------------------------------------------------------------------------
// Sizes.  One call sorts fewer than 2^32 elements in total, so every element position fits an
// unsigned 32-bit integer (pos_t: run starts, node ranges, tile bounds, co-ranks); addresses and
// the few sums that can pass 2^32 are formed in 64 bits.  Run and boundary indices are int32 (a
// call has fewer than 2^31 runs); offsets inside a tile or a shared-memory task are int32.  Node
// powers are at most floor(lg n) + 1 <= 32 (Definition "Node Power"), so node depths are < 32.
// ---------------------------------------------------------------------------------------
typedef uint32_t pos_t;
constexpr int64_t kMaxElems = (int64_t)1 << 32;      // n < kMaxElems
constexpr int32_t kMaxRuns = 0x7ffffffe;            // r <= kMaxRuns (boundary indices 0..r fit int32)
constexpr int kMaxLevels = 32;  // node depths are < 32

// Stage 1 (run detection): one CTA scans a tile of kDetectTile positions.
constexpr int kDetectThreads = 256;
constexpr int kDetectItems = 32;
constexpr int kDetectTile = kDetectThreads * kDetectItems;  // 8192

// Stage 3 (nearest-smaller-value tree): 256 threads x 32 consecutive boundaries per tile.
constexpr int kTreeThreads = 256;
constexpr int kTreeChunk = 32;
constexpr int kTreeTile = kTreeThreads * kTreeChunk;  // 8192

// Level-pass configurations (items per consumer thread, shared-memory ring stages) compiled
// into the library; the tile of a pass is items x kMergeThreads outputs.
__host__ __device__ constexpr int pass_variant(int ipt, int stages) { return ipt * 16 + stages; }
constexpr int kPassVariants = 8;
constexpr int kPassVariantIpt[kPassVariants] = {12, 12, 12, 8, 8, 16, 6, 10};
constexpr int kPassVariantStages[kPassVariants] = {2, 3, 4, 2, 3, 2, 2, 2};
// 6 and 10 items: a consumer thread's share of keys is an odd multiple of 8 bytes (4-byte keys:
// 24 or 40 bytes; 8-byte keys: 48 or 80 bytes), so the shared-memory reads of a warp whose lanes
// walk one input at lane stride IPT keys spread over more banks than at 8 or 12 items.

// Stage 4 (merge passes over HBM): one CTA produces kMergeTile outputs of one merge.
constexpr int kMergeThreads = 256;
constexpr int kMergeItems = 12;
constexpr int kMergeTile = kMergeThreads * kMergeItems;  // 3072

// Buffer (0 = the caller's arrays, 1 = scratch) that holds the sorted output of a materialised
// node or leaf at depth d: a node at depth d writes buffer d mod 2 and reads its children from
// buffer (d + 1) mod 2, so the root lands in the caller's arrays.
__host__ __device__ constexpr int out_buffer(int d) { return d & 1; }

// Stage 4 (whole small subtrees in shared memory): a tree node whose range holds at most
// sub_tile(key size) elements is merged completely inside one CTA.
constexpr int kSubThreads = 256;
__host__ __device__ constexpr int sub_tile(int key_bytes) { return key_bytes == 8 ? 2048 : 4096; }
// Inside a task, a subtree of at most micro_tile(key size) elements whose parent is larger (a
// "micro root") is sorted by one thread in registers instead of level by level.
__host__ __device__ constexpr int micro_tile(int key_bytes) { return key_bytes == 8 ? 8 : 16; }

// ---------------------------------------------------------------------------------------
// Key orders.  Every key type is compared through an order-preserving map to an unsigned
// integer: int32 flips the sign bit; float32 uses IEEE totalOrder (negative patterns are
// complemented, non-negative ones get the sign bit set); unsigned types are themselves.
// ---------------------------------------------------------------------------------------
// le(a, b) is a <= b in the key order, written directly where a native compare exists.
struct KeyI32 {
  typedef uint32_t T;
  static constexpr int kType = 0;
  __device__ __forceinline__ static uint32_t ord(uint32_t x) { return x ^ 0x80000000u; }
  __device__ __forceinline__ static uint32_t unord(uint32_t u) { return u ^ 0x80000000u; }
  __device__ __forceinline__ static bool le(uint32_t a, uint32_t b) { return (int32_t)a <= (int32_t)b; }
};
struct KeyU32 {
  typedef uint32_t T;
  static constexpr int kType = 1;
  __device__ __forceinline__ static uint32_t ord(uint32_t x) { return x; }
  __device__ __forceinline__ static uint32_t unord(uint32_t u) { return u; }
  __device__ __forceinline__ static bool le(uint32_t a, uint32_t b) { return a <= b; }
};
struct KeyU64 {
  typedef uint64_t T;
  static constexpr int kType = 2;
  __device__ __forceinline__ static uint64_t ord(uint64_t x) { return x; }
  __device__ __forceinline__ static bool le(uint64_t a, uint64_t b) { return a <= b; }
};
struct KeyF32 {
  typedef uint32_t T;
  static constexpr int kType = 3;
  __device__ __forceinline__ static uint32_t ord(uint32_t x) {
    return x ^ ((uint32_t)((int32_t)x >> 31) | 0x80000000u);
  }
  // inverse of ord: a set top bit marks a non-negative pattern
  __device__ __forceinline__ static uint32_t unord(uint32_t u) {
    return u ^ ((uint32_t)((int32_t)~u >> 31) | 0x80000000u);
  }
  __device__ __forceinline__ static bool le(uint32_t a, uint32_t b) { return ord(a) <= ord(b); }
};

// ---------------------------------------------------------------------------------------
// Device-posted status bits (plan header and the library-wide status word).
// ---------------------------------------------------------------------------------------
enum DevStatus : uint32_t {
  kDevOk = 0,
  kDevTimeout = 1u << 0,      // a bounded wait gave up
  kDevBadOffsets = 1u << 1,   // segment offsets not non-decreasing / out of range
  kDevInternal = 1u << 2,     // an internal consistency check failed
  kDevTooManyRuns = 1u << 3,  // more runs than boundary indices can hold (segments of 1 element)
};

// What the device tells the host after planning (one D2H copy per sort).
struct PlanHeader {
  int32_t runs;             // r: number of detected runs (all segments)
  uint32_t status;          // DevStatus bits
  uint32_t pad1;
  int32_t max_leaf_depth;
  unsigned long long cost;  // merge cost M = sum of leaf depth x run length
  uint32_t n_small;         // subtree-in-SMEM tasks
  uint32_t small_next;      // device-driven subtree kernel: next task to take (work counter)
  unsigned long long leaf_ctr;               // (count << 32) | tiles of large-leaf placement
  unsigned long long level_ctr[kMaxLevels];  // per depth: (count << 32) | merge tiles
  // element counts for the algorithmic-traffic accounting of stage 4
  unsigned long long small_elems;            // elements of all subtree-in-SMEM tasks
  unsigned long long place_elems;            // elements moved by large-leaf placement
  unsigned long long level_elems[kMaxLevels];  // outputs of the merges of each depth pass
};

// ---------------------------------------------------------------------------------------
// PTX helpers (sm_90+ mbarrier / bulk async copies; used on sm_103a).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 1-D bulk copy global -> shared, completion counted on an mbarrier.  Both addresses and the
// size must be multiples of 16 bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Post status bits to the per-call plan header and to the library's per-device status word
// (read and cleared by ps_stream_status); either pointer may be null.
__device__ __forceinline__ void post_status(uint32_t* hdr_status, uint32_t* lib_status, uint32_t bits) {
  if (hdr_status) atomicOr(hdr_status, bits);
  if (lib_status) atomicOr(lib_status, bits);
}

// A merge of the level passes: node [lo, mid) + [mid, hi) in element positions, and which of
// its children are large descending runs read backwards (bit 0 left, bit 1 right).
struct __align__(16) NodeItem {
  pos_t lo, mid, hi;
  int32_t rev;
};

// Launch-argument sentinel: take the work count from the plan header on the device.
constexpr uint32_t kCountOnDevice = 0xFFFFFFFFu;

// Bounded waits: iterations before a wait gives up and posts kDevTimeout.  Look-back polls
// sleep 64 ns between reads (about 0.3 s in all); an mbarrier try_wait suspends for a
// hardware-defined interval per call.
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr uint32_t kMbarTries = 1u << 20;

}  // namespace ps
