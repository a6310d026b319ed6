// Stage 4: the level pass -- all large merges of one tree depth in one persistent launch.
// (Kept in its own file: the benchmark ties the level pass's recorded DRAM traffic to the hash of
// this file and ps_common.cuh / ps_mergeutil.cuh, the sources the kernel is built from.)
#pragma once

#include "ps_common.cuh"
#include "ps_debug.cuh"
#include "ps_mergeutil.cuh"

namespace ps {

// ---------------------------------------------------------------------------------------
// One level pass: all merges of the tree nodes at one depth whose ranges exceed the subtree
// limit, split into output tiles that start at the node's lo and then at the multiples of the
// tile size (IPT outputs per consumer thread x 256 threads) inside it.  Persistent and warp-specialized:
//  * CTA b owns the contiguous tile range [b*T/G, (b+1)*T/G) of the pass (T tiles, G CTAs), so
//    the co-rank at the end of one tile is the co-rank at the start of the next;
//  * warp 9 (searcher) walks the CTA's tiles in batches: it finds each tile's end co-rank with
//    an 8-way search in global memory inside the window the last known co-rank allows, and
//    publishes the searched tiles in a shared-memory queue of kQueue entries (one mbarrier pair
//    per entry), running ahead of the copies so that the searches' global-memory latency
//    overlaps the merges;
//  * warp 8 (issuer, one thread) takes the next searched tile, waits for a free stage, and
//    issues the tile's four bulk copies (left/right keys and payloads, 16-byte aligned chunks)
//    on that stage's "full" mbarrier;
//  * warps 0-7 (consumers) wait for a full stage, merge its IPT outputs per thread
//    (co-rank inside shared memory, then a serial stable merge), write them with 128-bit
//    stores, and release the stage on its "empty" mbarrier.
// A child that is a large strictly descending run (a leaf of even depth, flagged in the node
// item's 4th field: bit 0 left child, bit 1 right child) is still in its original order in the
// source buffer; the pass reads it backwards: its sorted element i is the element at the end of
// its range minus i, for the co-rank probes, the copied ranges and the consumers' reads.
// A ring of NS stages: the copies of the next NS-1 tiles overlap the merge of the current one.
// All waits are bounded; a timeout posts kDevTimeout and the CTA drains its copies and exits.
// ---------------------------------------------------------------------------------------
constexpr int kLevelThreads = kMergeThreads + 64;  // 8 consumer warps + issuer + searcher
constexpr int kQueue = 8;                          // searched tiles the searcher may run ahead
constexpr int kSearchBatch = 4;                    // tiles searched together (8 lanes each)

// A searched tile: its node, outputs [g0, g1) (element positions), left-child elements [i0, i1).
struct QueuedTile {
  NodeItem nd;
  pos_t g0, g1, i0, i1;
};

// A staged tile as the consumers see it: outputs [g0, g0 + len), la of them from the left child.
struct StageDesc {
  pos_t g0;
  int32_t len, la;
  int32_t aoff, boff, vaoff, vboff;  // smem element offsets of the tile's first left / right element
  int32_t rev;                       // bit 0: the left child is read backwards, bit 1: the right child
  int32_t pad[8];
};

// Position of sorted element i of a node's left / right child: lo + i (mid + i) for a child in
// order, mid - 1 - i (hi - 1 - i) for a descending run read backwards.  Computed from the node
// item itself, so the searches keep no extra pointers live.
__device__ __forceinline__ pos_t left_at(const NodeItem& nd, pos_t i) { return (nd.rev & 1) ? nd.mid - 1 - i : nd.lo + i; }
__device__ __forceinline__ pos_t right_at(const NodeItem& nd, pos_t j) { return (nd.rev & 2) ? nd.hi - 1 - j : nd.mid + j; }

// Output range of tile k of a node: tiles start at the node's lo and then at the multiples of
// kTile inside it (the products in 64 bits: a tile's end can pass 2^32 before the min).
template <int kTile>
__device__ __forceinline__ pos_t tile_start(const NodeItem& nd, uint32_t k) {
  return k == 0 ? nd.lo : (pos_t)(((uint64_t)(nd.lo / kTile) + k) * kTile);
}
template <int kTile>
__device__ __forceinline__ pos_t tile_end(const NodeItem& nd, uint32_t k) {
  return (pos_t)min((uint64_t)nd.hi, ((uint64_t)(nd.lo / kTile) + k + 1) * kTile);
}

template <class K, bool V, int NS, int IPT>
struct PassLayout {
  typedef typename K::T T;
  static constexpr int kStages = NS;
  static constexpr int kTile = IPT * kMergeThreads;
  static constexpr int KU = 16 / (int)sizeof(T);
  static constexpr int KCAP = kTile + 4 * KU;
  static constexpr int VCAP = kTile + 16;
  static constexpr size_t kKeyBytes = ((size_t)KCAP * sizeof(T) + 127) & ~(size_t)127;
  static constexpr size_t kValBytes = V ? (((size_t)VCAP * 4 + 127) & ~(size_t)127) : 0;
  static constexpr size_t kStageBytes = kKeyBytes + kValBytes;
  static constexpr size_t kBarOff = 0;  // full[NS], empty[NS]
  static constexpr size_t kDescOff = (2 * NS * 8 + 63) & ~(size_t)63;  // StageDesc[NS]
  static constexpr size_t kQBarOff = kDescOff + NS * sizeof(StageDesc);  // qfull[kQueue], qempty[kQueue]
  static constexpr size_t kQueueOff = (kQBarOff + 2 * kQueue * 8 + 63) & ~(size_t)63;  // QueuedTile[kQueue]
  static constexpr size_t kFlagOff = kQueueOff + kQueue * sizeof(QueuedTile);
  static constexpr size_t kStageOff = (kFlagOff + 16 + 127) & ~(size_t)127;
  static constexpr size_t kBytes = kStageOff + NS * kStageBytes;
};

// smallest i in [a, b] with i == b or A[i] > B[diag-1-i] (A, B: the node's children in sorted
// order), by a 32-way warp search in global memory
template <class K>
__device__ __forceinline__ pos_t warp_corank(const typename K::T* __restrict__ src, const NodeItem& nd, pos_t diag,
                                             pos_t a, pos_t b) {
  const int lane = threadIdx.x & 31;
  while (a < b) {
    const pos_t span = b - a;
    const pos_t x = a + (pos_t)(((uint64_t)span * lane) >> 5);  // probes in [a, b)
    const bool gt = !key_le<K>(src[left_at(nd, x)], src[right_at(nd, diag - 1 - x)]);
    const uint32_t mask = __ballot_sync(0xffffffffu, gt);
    if (mask) {
      const int fl = __ffs(mask) - 1;
      const pos_t xf = __shfl_sync(0xffffffffu, x, fl);
      const pos_t xp = __shfl_sync(0xffffffffu, x, fl > 0 ? fl - 1 : 0);
      b = xf;
      if (fl > 0) a = xp + 1;
    } else {
      a = __shfl_sync(0xffffffffu, x, 31) + 1;
    }
  }
  return a;
}

// AND of a predicate over the kMergeThreads consumer threads (also a barrier among them)
__device__ __forceinline__ bool consumer_all(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.and.pred b, 1, %2, a;\n selp.u32 %0, 1, 0, b;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "n"(kMergeThreads)
      : "memory");
  return r != 0;
}

// Element range [e0, e1) of base widened to whole 16-byte blocks: [c0, c1) (element indices,
// possibly c0 < 0 by a few elements when base itself is not 16-byte aligned).  Empty ranges give
// an empty chunk.  Needs base aligned to sizeof(E).
template <class E>
__device__ __forceinline__ void chunk16(const E* base, int64_t e0, int64_t e1, int64_t& c0, int64_t& c1) {
  constexpr int kPer = 16 / (int)sizeof(E);
  const int64_t phase = (int64_t)(((uintptr_t)base & 15u) / sizeof(E));  // elements before base in its block
  c0 = ((e0 + phase) & ~(int64_t)(kPer - 1)) - phase;
  c1 = (e1 > e0) ? (((e1 + phase + kPer - 1) & ~(int64_t)(kPer - 1)) - phase) : c0;
}

__device__ __forceinline__ bool bounded_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  uint32_t tries = 0;
  while (!mbar_try_wait(bar, parity))
    if (++tries > limit) return false;
  return true;
}

// Reverse the staged elements [off, off + len) of a tile's keys (and payloads at voff) in place,
// spread over the kMergeThreads consumers: a child read backwards is staged in memory order,
// and this puts its sorted elements in order before the merge.
template <class T, bool V, int KCAP, int VCAP>
__device__ __forceinline__ void reverse_staged(T* sk, uint32_t* sv, int32_t off, int32_t voff, int32_t len, int tid) {
  for (int32_t k = tid; k < len / 2; k += kMergeThreads) {
    const int32_t x = off + k, y = off + len - 1 - k;
    if (PS_IN_RANGE(x, KCAP) && PS_IN_RANGE(y, KCAP)) {
      const T t = sk[x];
      sk[x] = sk[y];
      sk[y] = t;
    }
    if (V) {
      const int32_t vx = voff + k, vy = voff + len - 1 - k;
      if (PS_IN_RANGE(vx, VCAP) && PS_IN_RANGE(vy, VCAP)) {
        const uint32_t u = sv[vx];
        sv[vx] = sv[vy];
        sv[vy] = u;
      }
    }
  }
}

// One consumer thread's share of a staged tile: the co-rank of its first output inside shared
// memory, a serial stable merge of up to IPT outputs (the heads of both inputs kept in
// registers: one shared-memory key read per output), and 16-byte stores (8-byte ones where a
// thread's share of keys or payloads is an odd multiple of 8 bytes).
template <class K, bool V, int IPT, class Lay>
__device__ __forceinline__ void consume_tile(const StageDesc& d, const uint8_t* stage, typename K::T* __restrict__ dstk,
                                             uint32_t* __restrict__ dstv, int tid) {
  typedef typename K::T T;
  constexpr int KU = Lay::KU;
  const T* A = (const T*)stage + d.aoff;
  const T* B = (const T*)stage + d.boff;
  const uint32_t* sv = (const uint32_t*)(stage + Lay::kKeyBytes);
  const int32_t len = d.len, la = d.la, lb = len - la;
  const int32_t diag = tid * IPT;
  if (diag >= len) return;
  int32_t i = corank_serial<K>(A, B, la, lb, diag);
  int32_t j = diag - i;
  const int32_t cnt = min(IPT, len - diag);
  T key[IPT];
  uint32_t val[IPT];
  T a = A[min(i, la - 1 >= 0 ? la - 1 : 0)], b = B[min(j, lb - 1 >= 0 ? lb - 1 : 0)];
  auto step = [&](int q) {
    const bool takeA = (j >= lb) || (i < la && key_le<K>(a, b));
    key[q] = takeA ? a : b;
    if (V) {
      const int32_t vi = takeA ? d.vaoff + i : d.vboff + j;
      val[q] = PS_IN_RANGE(vi, Lay::VCAP) ? sv[vi] : 0u;
    }
    i += takeA ? 1 : 0;
    j += takeA ? 0 : 1;
    if (takeA) {
      if (i < la && PS_IN_RANGE(d.aoff + i, Lay::KCAP)) a = A[i];
    } else {
      if (j < lb && PS_IN_RANGE(d.boff + j, Lay::KCAP)) b = B[j];
    }
  };
  if (cnt == IPT) {  // a whole share: no per-output guard
#pragma unroll
    for (int q = 0; q < IPT; ++q) step(q);
  } else {
#pragma unroll
    for (int q = 0; q < IPT; ++q)
      if (q < cnt) step(q);
  }
  const int64_t g = d.g0 + diag;
  bool stored = false;
  if constexpr (IPT % KU == 0) {  // a thread's keys fill whole 16-byte stores
    if (cnt == IPT && ((uintptr_t)(dstk + g) & 15u) == 0) {
      uint4* o = (uint4*)(dstk + g);
#pragma unroll
      for (int q = 0; q < IPT / KU; ++q) {
        uint4 w;
        T* wt = (T*)&w;
#pragma unroll
        for (int u = 0; u < KU; ++u) wt[u] = key[q * KU + u];
        o[q] = w;
      }
      stored = true;
    }
  } else {  // 4-byte keys, 6 or 10 items: 8-byte stores
    static_assert(IPT % 2 == 0 && sizeof(T) == 4, "a thread's keys fill whole 8-byte stores");
    if (cnt == IPT && ((uintptr_t)(dstk + g) & 7u) == 0) {
      uint2* o = (uint2*)(dstk + g);
#pragma unroll
      for (int q = 0; q < IPT / 2; ++q) {
        uint2 w;
        T* wt = (T*)&w;
        wt[0] = key[2 * q];
        wt[1] = key[2 * q + 1];
        o[q] = w;
      }
      stored = true;
    }
  }
  if (!stored) {
#pragma unroll
    for (int q = 0; q < IPT; ++q)
      if (q < cnt) dstk[g + q] = key[q];
  }
  if (V) {
    if (IPT % 4 == 0 && cnt == IPT && ((uintptr_t)(dstv + g) & 15u) == 0) {
      uint4* o = (uint4*)(dstv + g);
#pragma unroll
      for (int q = 0; q < IPT / 4; ++q) o[q] = make_uint4(val[4 * q], val[4 * q + 1], val[4 * q + 2], val[4 * q + 3]);
    } else if (IPT % 4 == 2 && cnt == IPT && ((uintptr_t)(dstv + g) & 7u) == 0) {  // 6 or 10 items
      uint2* o = (uint2*)(dstv + g);
#pragma unroll
      for (int q = 0; q < IPT / 2; ++q) o[q] = make_uint2(val[2 * q], val[2 * q + 1]);
    } else {
#pragma unroll
      for (int q = 0; q < IPT; ++q)
        if (q < cnt) dstv[g + q] = val[q];
    }
  }
}

// CTAs per SM the register budget is sized for (16 items per thread need more registers).
__host__ __device__ constexpr int pass_min_blocks(int ipt) { return ipt <= 12 ? 4 : 3; }

template <class K, bool V, int NS, int IPT>
__global__ void __launch_bounds__(kLevelThreads, pass_min_blocks(IPT))
level_pass_kernel(const typename K::T* __restrict__ srck, const uint32_t* __restrict__ srcv,
                  typename K::T* __restrict__ dstk, uint32_t* __restrict__ dstv,
                  const NodeItem* __restrict__ nodes, const uint32_t* __restrict__ tile_off, uint32_t nitems,
                  uint32_t ntiles, const unsigned long long* __restrict__ ctr, uint32_t cap,
                  PlanHeader* __restrict__ hdr, uint32_t* lib_status, uint32_t polls, int withhold) {
  // polls: the bound of every wait of the pass (the library default unless a failure self-test
  // sets a smaller one).  withhold (self-test only): CTA 0's issuer never issues its first tile's
  // copies, so that stage's "full" barrier is never completed and the waits on it run out.
  typedef typename K::T T;
  typedef PassLayout<K, V, NS, IPT> Lay;
  constexpr int kTile = Lay::kTile;
  if (ctr != nullptr) {  // counts from the plan on the device (no host round trip)
    if (hdr->status & kDevBadOffsets) return;
    const unsigned long long v = *ctr;
    nitems = (uint32_t)(v >> 32);
    ntiles = (uint32_t)(v & 0xffffffffull);
    if (nitems > cap) return;  // the plan posted an internal error already
  }
  constexpr int kPassStages = NS;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = (uint64_t*)(smem + Lay::kBarOff);
  uint64_t* empty = full + kPassStages;
  StageDesc* sdesc = (StageDesc*)(smem + Lay::kDescOff);
  volatile int32_t* abort_flag = (volatile int32_t*)(smem + Lay::kFlagOff);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t t_begin = (uint32_t)(((uint64_t)blockIdx.x * ntiles) / gridDim.x);
  const uint32_t t_end = (uint32_t)(((uint64_t)(blockIdx.x + 1) * ntiles) / gridDim.x);
  if (t_begin >= t_end) return;  // no tile for this CTA (uniform over the CTA)
  uint64_t* qfull = (uint64_t*)(smem + Lay::kQBarOff);
  uint64_t* qempty = qfull + kQueue;
  QueuedTile* queue = (QueuedTile*)(smem + Lay::kQueueOff);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPassStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kMergeThreads / 32);
    }
    for (int q = 0; q < kQueue; ++q) {
      mbar_init(&qfull[q], 1);
      mbar_init(&qempty[q], 1);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kMergeThreads / 32 + 1) {
    // ------------------------------ searcher ------------------------------
    int32_t slot = 0;
    if (lane == 0) slot = slot_of_tile(tile_off, nitems, t_begin);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    NodeItem nd = nodes[slot];
    pos_t g0 = tile_start<kTile>(nd, t_begin - tile_off[slot]);
    pos_t i0 = 0;
    if (g0 > nd.lo) {
      const pos_t diag = g0 - nd.lo, lb0 = nd.hi - nd.mid;
      i0 = warp_corank<K>(srck, nd, diag, diag > lb0 ? diag - lb0 : 0, min(diag, nd.mid - nd.lo));
    }
    // Batches of kSearchBatch tiles: lane group m (8 lanes) finds the end co-rank of the batch's
    // tile m with an 8-way search, all groups at once.  Each window is anchored at the last
    // co-rank known in the same node (the batch start, or 0 at a node's first tile), so it is at
    // most kSearchBatch tiles wide.
    const int grp = lane >> 3, gl = lane & 7;
    const uint32_t gmask = 0xFFu << (grp * 8);
    uint32_t published = 0;
    bool ok = true;
    uint32_t t = t_begin;
    while (t < t_end && ok) {
      const int nb = (int)min((uint32_t)kSearchBatch, t_end - t);
      NodeItem m_nd[kSearchBatch];
      pos_t m_g0[kSearchBatch], m_g1[kSearchBatch], m_a[kSearchBatch], m_b[kSearchBatch];
      int32_t m_slot[kSearchBatch];
      bool m_new[kSearchBatch];
      {
        int32_t cs = slot;
        pos_t cg0 = g0, ag = g0, ai = i0;
        NodeItem cnd = nd;
#pragma unroll
        for (int m = 0; m < kSearchBatch; ++m) {
          m_new[m] = false;
          if (m < nb) {
            const uint32_t tt = t + m;
            if (cs + 1 < (int32_t)nitems && tile_off[cs + 1] <= tt) {
              while (cs + 1 < (int32_t)nitems && tile_off[cs + 1] <= tt) ++cs;
              cnd = nodes[cs];
              cg0 = cnd.lo;
              ag = cnd.lo;
              ai = 0;
              m_new[m] = true;
            }
            const pos_t g1 = (pos_t)min((uint64_t)cnd.hi, ((uint64_t)(cg0 / kTile) + 1) * kTile);
            const pos_t cla = cnd.mid - cnd.lo, clb = cnd.hi - cnd.mid, diag = g1 - cnd.lo;
            m_nd[m] = cnd;
            m_slot[m] = cs;
            m_g0[m] = cg0;
            m_g1[m] = g1;
            // window of the end co-rank (empty window when the tile ends at the node's end)
            m_a[m] = (g1 < cnd.hi) ? max(ai, diag > clb ? diag - clb : 0) : cla;
            m_b[m] = (g1 < cnd.hi) ? (pos_t)min((uint64_t)ai + (g1 - ag), (uint64_t)cla) : cla;
            cg0 = g1;
          }
        }
      }
      // group grp searches tile grp (8-way probes)
      pos_t res = 0;
      {
        NodeItem snd = m_nd[0];
        pos_t sa = m_a[0], sb = m_b[0], sg1 = m_g1[0];
#pragma unroll
        for (int m = 1; m < kSearchBatch; ++m)
          if (grp == m) {
            snd = m_nd[m];
            sa = m_a[m];
            sb = m_b[m];
            sg1 = m_g1[m];
          }
        if (grp < nb) {
          const pos_t diag = sg1 - snd.lo;
          pos_t ga = sa, gb = sb;
          while (ga < gb) {
            const pos_t span = gb - ga;
            const pos_t x = ga + (pos_t)(((uint64_t)span * gl) >> 3);
            const bool gt = !key_le<K>(srck[left_at(snd, x)], srck[right_at(snd, diag - 1 - x)]);
            const uint32_t msk = (__ballot_sync(gmask, gt) >> (grp * 8)) & 0xFFu;
            if (msk) {
              const int fl = __ffs(msk) - 1;
              const pos_t xf = __shfl_sync(gmask, x, grp * 8 + fl);
              const pos_t xp = __shfl_sync(gmask, x, grp * 8 + (fl > 0 ? fl - 1 : 0));
              gb = xf;
              if (fl > 0) ga = xp + 1;
            } else {
              ga = __shfl_sync(gmask, x, grp * 8 + 7) + 1;
            }
          }
          res = ga;
        }
      }
      pos_t m_i1[kSearchBatch];
#pragma unroll
      for (int m = 0; m < kSearchBatch; ++m) m_i1[m] = __shfl_sync(0xffffffffu, res, m * 8);
      // wait for the batch's queue slots, publish the searched tiles
#pragma unroll
      for (int m = 0; m < kSearchBatch; ++m) {
        if (m < nb && ok) {
          const uint32_t idx = published + m;
          int good = 1;
          if (lane == 0) {
            good = 0;
            for (uint32_t tries = 0; tries < polls; ++tries) {
              if (mbar_try_wait(&qempty[idx % kQueue], ((idx / kQueue) & 1u) ^ 1u)) { good = 1; break; }
              if (*abort_flag) break;
            }
          }
          good = __shfl_sync(0xffffffffu, good, 0);
          if (!good) { ok = false; break; }
          if (lane == 0) {
            const NodeItem cnd = m_nd[m];
            QueuedTile q;
            q.nd = cnd;
            q.g0 = m_g0[m];
            q.g1 = m_g1[m];
            q.i0 = m_new[m] ? 0 : (m == 0 ? i0 : m_i1[m - 1]);
            q.i1 = (m_g1[m] < cnd.hi) ? m_i1[m] : (cnd.mid - cnd.lo);
            queue[idx % kQueue] = q;
            mbar_arrive(&qfull[idx % kQueue]);
          }
          __syncwarp();
        }
      }
      published += nb;
      // carry the state to the next batch: next tile starts where the batch's last tile ended
      slot = m_slot[0];
      nd = m_nd[0];
      g0 = m_g1[0];
      i0 = m_i1[0];
#pragma unroll
      for (int m = 1; m < kSearchBatch; ++m)
        if (m < nb) {
          slot = m_slot[m];
          nd = m_nd[m];
          g0 = m_g1[m];
          i0 = (m_g1[m] < m_nd[m].hi) ? m_i1[m] : (m_nd[m].mid - m_nd[m].lo);
        }
      if (nb == 1) i0 = (m_g1[0] < m_nd[0].hi) ? m_i1[0] : (m_nd[0].mid - m_nd[0].lo);
      t += nb;
    }
    if (!ok && lane == 0) {
      if (!*abort_flag) post_status(&hdr->status, lib_status, kDevTimeout);
      *abort_flag = 1;
    }
  } else if (warp == kMergeThreads / 32) {
    // ------------------------------ issuer ------------------------------
    if (lane != 0) return;  // one thread issues; the others have nothing to do
    const uint32_t total = t_end - t_begin;
    uint32_t issued = 0;
    bool ok = true;
    for (; issued < total; ++issued) {
      const uint32_t q = issued % kQueue;
      bool good = false;
      for (uint32_t tries = 0; tries < polls; ++tries) {
        if (mbar_try_wait(&qfull[q], (issued / kQueue) & 1u)) { good = true; break; }
        if (*abort_flag) break;
      }
      if (!good) { ok = false; break; }
      const QueuedTile qt = queue[q];
      mbar_arrive(&qempty[q]);
      const int s = (int)(issued % kPassStages);
      const uint32_t use = issued / kPassStages;
      if (!bounded_wait(&empty[s], (use & 1u) ^ 1u, polls)) { ok = false; break; }
      const NodeItem& cnd = qt.nd;
      const pos_t tj0 = qt.g0 - cnd.lo - qt.i0, tj1 = qt.g1 - cnd.lo - qt.i1;  // right-child elements [tj0, tj1)
      const bool ra = (cnd.rev & 1) != 0, rb = (cnd.rev & 2) != 0;
      // memory ranges of the tile's sorted elements (a child read backwards has them mirrored
      // at the end of its range)
      const int64_t a0 = ra ? cnd.mid - qt.i1 : cnd.lo + qt.i0, a1 = ra ? cnd.mid - qt.i0 : cnd.lo + qt.i1;
      const int64_t b0 = rb ? cnd.hi - tj1 : cnd.mid + tj0, b1 = rb ? cnd.hi - tj0 : cnd.mid + tj1;
      // 16-byte aligned enclosing chunks, computed on absolute addresses (the arrays only need
      // natural alignment; a chunk may start up to 15 bytes before a range and end up to 15
      // bytes after it, always inside 16-byte blocks holding range elements)
      int64_t ka0, ka1, kb0, kb1, va0, va1, vb0, vb1;
      chunk16(srck, a0, a1, ka0, ka1);
      chunk16(srck, b0, b1, kb0, kb1);
      chunk16(srcv, a0, a1, va0, va1);
      chunk16(srcv, b0, b1, vb0, vb1);
      StageDesc d;
      d.g0 = qt.g0;
      d.len = (int32_t)(qt.g1 - qt.g0);
      d.la = (int32_t)(qt.i1 - qt.i0);
      d.aoff = (int32_t)(a0 - ka0);
      d.boff = (int32_t)((ka1 - ka0) + (b0 - kb0));
      d.vaoff = (int32_t)(a0 - va0);
      d.vboff = (int32_t)((va1 - va0) + (b0 - vb0));
      d.rev = cnd.rev & 3;  // the consumers reverse these staged ranges before merging
      sdesc[s] = d;
      uint8_t* stage = smem + Lay::kStageOff + (size_t)s * Lay::kStageBytes;
      T* sk = (T*)stage;
      uint32_t* sv = (uint32_t*)(stage + Lay::kKeyBytes);
      const uint32_t kba = (uint32_t)(ka1 - ka0) * sizeof(T), kbb = (uint32_t)(kb1 - kb0) * sizeof(T);
      const uint32_t vba = V ? (uint32_t)(va1 - va0) * 4u : 0u, vbb = V ? (uint32_t)(vb1 - vb0) * 4u : 0u;
      if (withhold && blockIdx.x == 0 && issued == 0) continue;  // self-test: this stage never fills
      mbar_arrive_expect_tx(&full[s], kba + kbb + vba + vbb);
      if (kba) bulk_g2s(sk, srck + ka0, kba, &full[s]);
      if (kbb) bulk_g2s(sk + (ka1 - ka0), srck + kb0, kbb, &full[s]);
      if (V) {
        if (vba) bulk_g2s(sv, srcv + va0, vba, &full[s]);
        if (vbb) bulk_g2s(sv + (va1 - va0), srcv + vb0, vbb, &full[s]);
      }
    }
    if (!ok) {
      post_status(&hdr->status, lib_status, kDevTimeout);
      *abort_flag = 1;
    }
    // drain: every copy issued into a stage must have landed before the CTA exits
    for (uint32_t q = (issued > kPassStages ? issued - kPassStages : 0); q < issued; ++q) {
      const int s = (int)(q % kPassStages);
      bounded_wait(&full[s], (q / kPassStages) & 1u, polls);
    }
  } else {
    // ------------------------------ consumers ------------------------------
    const int tid = threadIdx.x;
    uint32_t it = 0;
    for (uint32_t t = t_begin; t < t_end; ++t, ++it) {
      const int s = (int)(it % kPassStages);
      const uint32_t use = it / kPassStages;
      bool ready = false;
      for (uint32_t tries = 0; tries < polls; ++tries) {
        if (mbar_try_wait(&full[s], use & 1u)) {
          ready = true;
          break;
        }
        if (*abort_flag) break;
      }
      // all consumers take the same branch (they meet at named barriers below)
      if (!consumer_all(ready)) {
        if (tid == 0 && !*abort_flag) post_status(&hdr->status, lib_status, kDevTimeout);
        break;
      }
      const StageDesc d = sdesc[s];
      const uint8_t* stage = smem + Lay::kStageOff + (size_t)s * Lay::kStageBytes;
      if (d.rev) {  // uniform over the consumers: they all work on the same tile
        uint8_t* wstage = smem + Lay::kStageOff + (size_t)s * Lay::kStageBytes;
        T* sk = (T*)wstage;
        uint32_t* svw = (uint32_t*)(wstage + Lay::kKeyBytes);
        if (d.rev & 1) reverse_staged<T, V, Lay::KCAP, Lay::VCAP>(sk, svw, d.aoff, d.vaoff, d.la, tid);
        if (d.rev & 2) reverse_staged<T, V, Lay::KCAP, Lay::VCAP>(sk, svw, d.boff, d.vboff, d.len - d.la, tid);
        consumer_all(true);  // barrier among the consumers: the staged tile is in sorted order
      }
      consume_tile<K, V, IPT, Lay>(d, stage, dstk, dstv, tid);
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(&empty[s]);
    }
  }
}

}  // namespace ps
