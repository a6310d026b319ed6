// Stage 4: the merges of the powersort tree (Alg. 2's Merge calls), scheduled level by level.
//
// Every merge is the stable merge of two adjacent sorted ranges [lo, mid) and [mid, hi) in which
// an element of the left range goes first when keys are equal (the tie rule of the paper's
// merge routine, Appendix B), so the output is the unique stable order.  Work is split by merge
// path: output position g of a merge is produced from the first i elements of the left range and
// the first g - i of the right one, where i (the co-rank) is the smallest index whose left
// element is greater than the right element it would be compared with.
//
//  * subtree_kernel      a whole subtree of at most sub_tile elements, merged in shared memory
//                        level by level (leaves placed by depth parity, descending runs
//                        reversed on the way in), written once.
//  * leaf_place_kernel   large leaves whose depth maps to the scratch buffer -> copied there;
//                        descending -> reversed.
//  * level_pass_kernel   (ps_level.cuh) the large merges of one depth in one persistent launch.
#pragma once

#include "ps_common.cuh"
#include "ps_debug.cuh"
#include "ps_mergeutil.cuh"

namespace ps {

// ---------------------------------------------------------------------------------------
// Whole subtree in shared memory.
//
// The task's elements stay in one shared-memory array from the leaves to the subtree root.
// Each level's merges are computed into registers (thread t produces the outputs at positions
// [t*IPT, t*IPT + IPT)), the block synchronises, and the outputs overwrite their positions, so
// one array suffices and buffer parity plays no role inside the task.  Every element carries
// its position inside the task; as all elements of a left child sit before all elements of the
// right child, "the left element goes first on equal keys" is the order of (key, position):
//  * 4-byte keys: one 64-bit word (order-mapped key << 32 | position) compared as an integer;
//  * 8-byte keys: the key and a 32-bit position side by side, keys compared with the tie rule.
// The payload does not move during the merges: it is staged once at the end and gathered
// through the positions.  The array has one padding slot per IPT elements, so the IPT-strided
// accesses of a warp fall into distinct banks.
// ---------------------------------------------------------------------------------------
template <class K, int KB = (int)sizeof(typename K::T)>
struct SubElem;

template <class K>
struct SubElem<K, 4> {
  typedef uint64_t R;
  static constexpr int TS = sub_tile(4);
  static constexpr int IPT = TS / kSubThreads;
  static constexpr int kPadded = TS + TS / IPT;
  static constexpr size_t kDataBytes = (size_t)kPadded * 8;
  struct Arr {
    uint64_t* w;
  };
  __device__ __forceinline__ static Arr arr(uint8_t* base) { return Arr{(uint64_t*)base}; }
  __device__ __forceinline__ static R ld(const Arr& a, int32_t i) { return PS_IN_RANGE(i, kPadded) ? a.w[i] : R(0); }
  __device__ __forceinline__ static void st(const Arr& a, int32_t i, R x) {
    if (PS_IN_RANGE(i, kPadded)) a.w[i] = x;
  }
  __device__ __forceinline__ static R make(uint32_t key, int32_t pos) {
    return ((uint64_t)K::ord(key) << 32) | (uint32_t)pos;
  }
  __device__ __forceinline__ static R max_elem() { return ~(R)0; }  // above every element (positions < 2^16)
  // positions differ, so two elements never compare equal
  __device__ __forceinline__ static bool before(R a, R b) { return a < b; }
  __device__ __forceinline__ static bool less(R a, R b) { return a < b; }
  __device__ __forceinline__ static uint32_t key(R x) { return K::unord((uint32_t)(x >> 32)); }
  __device__ __forceinline__ static int32_t pos(R x) { return (int32_t)(uint32_t)x; }
};

template <class K>
struct SubElem<K, 8> {
  struct R {
    uint64_t k;
    uint32_t p;
  };
  static constexpr int TS = sub_tile(8);
  static constexpr int IPT = TS / kSubThreads;
  static constexpr int kPadded = TS + TS / IPT;
  static constexpr size_t kDataBytes = (size_t)kPadded * 12;
  struct Arr {
    uint64_t* k;
    uint32_t* p;
  };
  __device__ __forceinline__ static Arr arr(uint8_t* base) {
    return Arr{(uint64_t*)base, (uint32_t*)(base + (size_t)kPadded * 8)};
  }
  __device__ __forceinline__ static R ld(const Arr& a, int32_t i) {
    return PS_IN_RANGE(i, kPadded) ? R{a.k[i], a.p[i]} : R{0, 0};
  }
  __device__ __forceinline__ static void st(const Arr& a, int32_t i, R x) {
    if (!PS_IN_RANGE(i, kPadded)) return;
    a.k[i] = x.k;
    a.p[i] = x.p;
  }
  __device__ __forceinline__ static R make(uint64_t key, int32_t pos) { return R{key, (uint32_t)pos}; }
  __device__ __forceinline__ static R max_elem() { return R{~0ull, ~0u}; }  // above every element
  // a comes from the left child: it goes first unless its key is greater
  __device__ __forceinline__ static bool before(const R& a, const R& b) { return K::le(a.k, b.k); }
  // the order of (key, position), for elements of one run
  __device__ __forceinline__ static bool less(const R& a, const R& b) {
    return a.k != b.k ? K::le(a.k, b.k) : a.p < b.p;
  }
  __device__ __forceinline__ static uint64_t key(const R& x) { return x.k; }
  __device__ __forceinline__ static int32_t pos(const R& x) { return (int32_t)x.p; }
};

// padded slot of position p
template <class E>
__device__ __forceinline__ int32_t sub_slot(int32_t p) {
  return p + p / E::IPT;
}

// Batcher's odd-even merge sort network on N registers (N = 8 or 16): the compare-exchanges of
// the order of (key, position), listed by the non-recursive form of the construction (for
// p = 1, 2, 4, ..: for k = p, p/2, .., 1: for j = k mod p, j + 3k, ..: for i < k: compare
// i + j with i + j + k when both lie in the same block of 2p).  The pairs are compile-time
// constants, so the values stay in registers.  The network sorts every input: by the 0-1
// principle it suffices that it sorts all 2^N sequences of zeros and ones, which holds for both
// sizes (19 and 63 comparators).
template <int N>
struct MicroNet;
template <>
struct MicroNet<8> {
  static constexpr int kPairs = 19;
  __host__ __device__ static constexpr int lo(int c) {
    constexpr uint8_t t[kPairs] = {0, 2, 4, 6, 0, 1, 4, 5, 1, 5, 0, 1, 2, 3, 2, 3, 1, 3, 5};
    return t[c];
  }
  __host__ __device__ static constexpr int hi(int c) {
    constexpr uint8_t t[kPairs] = {1, 3, 5, 7, 2, 3, 6, 7, 2, 6, 4, 5, 6, 7, 4, 5, 2, 4, 6};
    return t[c];
  }
};
template <>
struct MicroNet<16> {
  static constexpr int kPairs = 63;
  __host__ __device__ static constexpr int lo(int c) {
    constexpr uint8_t t[kPairs] = {0, 2, 4, 6, 8, 10, 12, 14, 0, 1, 4, 5, 8, 9, 12, 13, 1, 5, 9, 13, 0, 1, 2, 3, 8, 9, 10, 11, 2, 3, 10, 11, 1, 3, 5, 9, 11, 13, 0, 1, 2, 3, 4, 5, 6, 7, 4, 5, 6, 7, 2, 3, 6, 7, 10, 11, 1, 3, 5, 7, 9, 11, 13};
    return t[c];
  }
  __host__ __device__ static constexpr int hi(int c) {
    constexpr uint8_t t[kPairs] = {1, 3, 5, 7, 9, 11, 13, 15, 2, 3, 6, 7, 10, 11, 14, 15, 2, 6, 10, 14, 4, 5, 6, 7, 12, 13, 14, 15, 4, 5, 12, 13, 2, 4, 6, 10, 12, 14, 8, 9, 10, 11, 12, 13, 14, 15, 8, 9, 10, 11, 4, 5, 8, 9, 12, 13, 2, 4, 6, 8, 10, 12, 14};
    return t[c];
  }
};

template <class E, int N>
__device__ __forceinline__ void micro_sort(typename E::R (&v)[N]) {
  typedef MicroNet<N> Net;
#pragma unroll
  for (int c = 0; c < Net::kPairs; ++c) {
    const typename E::R a = v[Net::lo(c)], b = v[Net::hi(c)];
    const bool sw = E::less(b, a);
    v[Net::lo(c)] = sw ? b : a;
    v[Net::hi(c)] = sw ? a : b;
  }
}

template <class K, bool V>
struct SubLayout {
  typedef SubElem<K> E;
  static constexpr int TS = E::TS;
  static constexpr int RC = TS / 2 + 2;  // runs in a task: all but a segment's last have length >= 2
  // The region after the element array holds in turn: run starts and directions (leaf
  // placement), the level-sorted node list (merges), the staged payload (write-out).
  static constexpr size_t kRuns = (size_t)RC * 3;
  static constexpr size_t kNodes = (size_t)RC * 8;
  static constexpr size_t kPay = V ? (size_t)TS * 4 : 0;
  static constexpr size_t kMeta = kNodes > kPay ? kNodes : kPay;
  static_assert(kRuns <= kMeta, "run metadata fits the shared region");
  static_assert(kRuns + (size_t)TS * 2 <= kMeta, "run metadata and the extended-run sources fit");
  static constexpr size_t kBytes = E::kDataBytes + kMeta;
};

// co-rank of output diag in the merge of positions [l, mm) and [mm, h) of the task array
template <class E>
__device__ __forceinline__ int32_t sub_corank(const typename E::Arr& X, int32_t l, int32_t mm, int32_t h,
                                              int32_t diag) {
  int32_t lo = max(0, diag - (h - mm)), hi = min(diag, mm - l);
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (E::before(E::ld(X, sub_slot<E>(l + mid)), E::ld(X, sub_slot<E>(mm + diag - 1 - mid)))) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <class K, bool V>
__device__ __forceinline__ void subtree_task(Bufs buf, const pos_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
                                             const int32_t* __restrict__ nodeL, const int32_t* __restrict__ nodeR,
                                             const uint8_t* __restrict__ ndepth, const uint8_t* __restrict__ ldepth,
                                             const uint8_t* __restrict__ micro, const int32_t task,
                                             PlanHeader* __restrict__ hdr,
                                             uint32_t* lib_status) {
  typedef typename K::T T;
  typedef SubElem<K> E;
  typedef typename E::R R;
  typedef SubLayout<K, V> Lay;
  constexpr int TS = E::TS, IPT = E::IPT, RC = Lay::RC, NW = kSubThreads / 32;
  static_assert(kMaxLevels * NW == kSubThreads, "one thread per (depth, warp) pair");
  static_assert(IPT <= 32, "valid-output mask is 32 bits");
  extern __shared__ __align__(128) uint8_t smem[];
  const typename E::Arr X = E::arr(smem);
  uint8_t* meta = smem + E::kDataBytes;
  __shared__ int32_t s_cnt[NW][kMaxLevels];  // boundaries per (warp, relative depth), then offsets
  __shared__ int32_t s_lvl[kMaxLevels + 1];  // nodes of relative depth d: entries [s_lvl[d], s_lvl[d+1])
  __shared__ int32_t s_wsum[NW];
  __shared__ int32_t s_maxrd;
  __shared__ int32_t s_nmicro;
  constexpr int kMicro = micro_tile((int)sizeof(T));

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t runs = hdr->runs;
  if (task >= runs || (task < 0 && ~task >= runs)) {  // never for a consistent plan
    if (tid == 0) post_status(&hdr->status, lib_status, kDevInternal);
    return;
  }
  int32_t L, R_, droot;
  if (task >= 0) {
    L = nodeL[task];
    R_ = nodeR[task];
    droot = ndepth[task];
  } else {
    L = ~task;
    R_ = L + 1;
    droot = ldepth[L];
  }
  if (L < 0 || R_ > runs || L >= R_) {
    if (tid == 0) post_status(&hdr->status, lib_status, kDevInternal);
    return;
  }
  const int64_t lo = S[L];
  const int64_t m64 = (int64_t)S[R_] - lo;
  const int32_t nr = R_ - L;
  if (m64 > TS || nr + 1 > RC) {  // cannot happen for a greedy run partition; never overrun SMEM
    if (tid == 0) post_status(&hdr->status, lib_status, kDevInternal);
    return;
  }
  const int32_t m = (int32_t)m64;  // the task's elements (at most TS)

  // 1. run starts and directions; the keys, tagged with their positions
  int16_t* rs = (int16_t*)meta;
  uint8_t* rdsc = (uint8_t*)(rs + RC);
  bool any_desc = false, any_ext = false;
  for (int32_t k = tid; k <= nr; k += kSubThreads) {
    rs[k] = (int16_t)((int64_t)S[L + k] - lo);
    if (k < nr) {
      rdsc[k] = run_desc[L + k];
      any_desc |= rdsc[k] == 1;
      any_ext |= (rdsc[k] & 2) != 0;
    }
  }
  const T* __restrict__ gk = (const T*)buf.k[0];
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    const int32_t p = tid + u * kSubThreads;
    if (p < m) E::st(X, sub_slot<E>(p), E::make(gk[lo + p], p));
  }
  for (int t = tid; t < NW * kMaxLevels; t += kSubThreads) (&s_cnt[0][0])[t] = 0;
  if (tid == 0) {
    s_maxrd = -1;
    s_nmicro = 0;
  }
  const int anyd = __syncthreads_or(any_desc);
  const int anyx = __syncthreads_or(any_ext);
  const int32_t cs = tid * IPT;

  // 2a. runs extended to the minimal run length: the element at p goes to its stable rank inside
  //     its run (the order of key, then position); src[rank] = p records where each output
  //     position takes its element from
  int16_t* src = (int16_t*)(meta + Lay::kRuns);
  if (anyx) {
    if (cs < m) {
      int32_t a = 0, b = nr;  // run containing cs
      while (b - a > 1) {
        const int32_t mid = (a + b) >> 1;
        if (rs[mid] <= cs) a = mid;
        else b = mid;
      }
      int32_t k = a;
      for (int q = 0; q < IPT; ++q) {
        const int32_t p = cs + q;
        if (p >= m) break;
        while (p >= rs[k + 1]) ++k;
        if (rdsc[k] & 2) {
          const R x = E::ld(X, sub_slot<E>(p));
          int32_t rank = rs[k];
          for (int32_t j = rs[k]; j < rs[k + 1]; ++j) rank += E::less(E::ld(X, sub_slot<E>(j)), x) ? 1 : 0;
          if (PS_IN_RANGE(rank, TS)) src[rank] = (int16_t)p;
        }
      }
    }
    __syncthreads();
  }

  // 2b. descending runs reversed and extended runs permuted in place, through registers
  if (anyd | anyx) {
    R v[IPT];
    uint32_t mv = 0;
    if (cs < m) {
      int32_t a = 0, b = nr;  // run containing cs: largest k with rs[k] <= cs
      while (b - a > 1) {
        const int32_t mid = (a + b) >> 1;
        if (rs[mid] <= cs) a = mid;
        else b = mid;
      }
      int32_t k = a;
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        const int32_t p = cs + q;
        if (p < m) {
          while (p >= rs[k + 1]) ++k;
          if (rdsc[k] != 0) {
            const int32_t from = (rdsc[k] & 2) ? (PS_IN_RANGE(p, TS) ? (int32_t)src[p] : p)
                                               : (int32_t)rs[k] + rs[k + 1] - 1 - p;
            if (from != p) {
              v[q] = E::ld(X, sub_slot<E>(from));
              mv |= 1u << q;
            }
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < IPT; ++q)
      if ((mv >> q) & 1u) E::st(X, sub_slot<E>(cs + q), v[q]);
  }

  // 3. the nodes (boundaries 1..nr-1) larger than kMicro, sorted by relative depth and by
  //    position inside a depth: a counting sort over warp chunks (match_any groups a warp's equal
  //    depths).  Nodes of at most kMicro elements lie inside a micro root's subtree (the largest
  //    such ancestor) and are merged by that root's register sort instead.
  const int32_t chunk = (nr - 1 + NW - 1) / NW;
  const int32_t w0 = 1 + warp * chunk, w1 = min(1 + (warp + 1) * chunk, nr);
  bool bad = false;
  int my_max = -1;
  for (int32_t k0 = w0; k0 < w1; k0 += 32) {
    const int32_t k = k0 + lane;
    int rd = kMaxLevels;  // lanes past the chunk and small nodes form their own group
    if (k < w1 && (int64_t)S[nodeR[L + k]] - (int64_t)S[nodeL[L + k]] > kMicro) {
      rd = (int)ndepth[L + k] - droot;
      if (rd < 0 || rd >= kMaxLevels) {
        bad = true;
        rd = 0;
      }
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, rd);
    if (rd < kMaxLevels) {
      my_max = max(my_max, rd);
      if (lane == __ffs(peers) - 1) s_cnt[warp][rd] += __popc(peers);
    }
  }
  if (bad) post_status(&hdr->status, lib_status, kDevInternal);
  my_max = __reduce_max_sync(0xffffffffu, my_max);
  if (lane == 0) atomicMax(&s_maxrd, my_max);
  __syncthreads();
  {
    // exclusive scan in (depth, warp) order: thread t holds depth t / NW, warp t % NW
    const int rd = tid / NW, w = tid % NW;
    const int32_t c = s_cnt[w][rd];
    int32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t o = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += o;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    int32_t off = inc - c;
    for (int x = 0; x < warp; ++x) off += s_wsum[x];
    s_cnt[w][rd] = off;
    if (w == 0) s_lvl[rd] = off;
    if (tid == kSubThreads - 1) s_lvl[kMaxLevels] = off + c;
  }
  __syncthreads();
  // ent[0 .. ) holds the level nodes: lo | mid << 16 | hi << 32 (task-relative); the micro roots
  // fill it from the top, lo | hi << 32 (level nodes and micro roots are distinct boundaries)
  uint64_t* ent = (uint64_t*)meta;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int32_t k0 = w0; k0 < w1; k0 += 32) {
    const int32_t k = k0 + lane;
    int rd = kMaxLevels;
    uint32_t nlo = 0, nhi = 0;
    if (k < w1) {
      const int32_t j = L + k;
      nlo = (uint32_t)((int64_t)S[nodeL[j]] - lo);
      nhi = (uint32_t)((int64_t)S[nodeR[j]] - lo);
      if ((int32_t)(nhi - nlo) > kMicro) {
        rd = min(max((int)ndepth[j] - droot, 0), kMaxLevels - 1);
      } else if (micro[j]) {
        const int32_t at = RC - 1 - atomicAdd(&s_nmicro, 1);
        if (PS_IN_RANGE(at, RC)) ent[at] = (uint64_t)nlo | ((uint64_t)nhi << 32);
      }
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, rd);
    if (rd < kMaxLevels) {
      const int32_t j = L + k;
      const int32_t at = s_cnt[warp][rd] + __popc(peers & lt_mask);
      const uint32_t nmid = (uint32_t)((int64_t)S[j] - lo);
      if (PS_IN_RANGE(at, RC)) ent[at] = (uint64_t)(nlo | (nmid << 16)) | ((uint64_t)nhi << 32);
    }
    __syncwarp();
    if (rd < kMaxLevels && lane == __ffs(peers) - 1) s_cnt[warp][rd] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // 3b. every micro root's subtree sorted by one thread in registers: its elements in the order of
  //     (key, position) are exactly the result of its stable merges (left elements first on ties)
  {
    const int32_t nmicro = s_nmicro;
    for (int32_t q = tid; q < nmicro; q += kSubThreads) {
      const uint64_t e = PS_IN_RANGE(RC - 1 - q, RC) ? ent[RC - 1 - q] : 0ull;
      const int32_t ml = (int32_t)(e & 0xFFFFu), len = (int32_t)(e >> 32) - ml;
      R v[kMicro];
#pragma unroll
      for (int i = 0; i < kMicro; ++i) v[i] = (i < len) ? E::ld(X, sub_slot<E>(ml + i)) : E::max_elem();
      micro_sort<E, kMicro>(v);
#pragma unroll
      for (int i = 0; i < kMicro; ++i)
        if (i < len) E::st(X, sub_slot<E>(ml + i), v[i]);
    }
    if (nmicro > 0) __syncthreads();  // uniform: s_nmicro is read after a barrier
  }

  // 4. the levels, deepest first
  for (int rd = s_maxrd; rd >= 0; --rd) {
    const int32_t e0 = s_lvl[rd], e1 = s_lvl[rd + 1];
    if (e0 == e1) continue;  // uniform over the block
    R out[IPT];
    uint32_t valid = 0;
    if (cs < m) {
      int32_t a = e0, b = e1;  // first node of the level with hi > cs
      while (a < b) {
        const int32_t mid = (a + b) >> 1;
        if ((int32_t)(ent[mid] >> 32) <= cs) a = mid + 1;
        else b = mid;
      }
      constexpr int32_t kNone = 1 << 30;
      int32_t l = kNone, mm = kNone, h = kNone, ia = kNone, ib = kNone;
      R va, vb;
      if (a < e1) {
        const uint64_t e = ent[a];
        l = (int32_t)(e & 0xFFFFu);
        mm = (int32_t)((e >> 16) & 0xFFFFu);
        h = (int32_t)(e >> 32);
        ia = l;
        ib = mm;
        if (l < cs) {
          const int32_t diag = cs - l;
          const int32_t i = sub_corank<E>(X, l, mm, h, diag);
          ia = l + i;
          ib = mm + diag - i;
        }
        if (ia < mm) va = E::ld(X, sub_slot<E>(ia));
        if (ib < h) vb = E::ld(X, sub_slot<E>(ib));
      }
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        const int32_t p = cs + q;
        if (p >= h) {  // this node is done; the level's next node starts at or after p
          ++a;
          if (a < e1) {
            const uint64_t e = ent[a];
            l = (int32_t)(e & 0xFFFFu);
            mm = (int32_t)((e >> 16) & 0xFFFFu);
            h = (int32_t)(e >> 32);
            ia = l;
            ib = mm;
            va = E::ld(X, sub_slot<E>(l));
            vb = E::ld(X, sub_slot<E>(mm));
          } else {
            l = mm = h = kNone;
          }
        }
        if (p >= l) {
          const bool take = ia < mm && (ib >= h || E::before(va, vb));
          out[q] = take ? va : vb;
          valid |= 1u << q;
          if (take) {
            if (++ia < mm) va = E::ld(X, sub_slot<E>(ia));
          } else {
            if (++ib < h) vb = E::ld(X, sub_slot<E>(ib));
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < IPT; ++q)
      if ((valid >> q) & 1u) E::st(X, sub_slot<E>(cs + q), out[q]);
    __syncthreads();
  }

  // 5. write-out into the buffer that holds the subtree root's output (out_buffer)
  const bool odd = out_buffer(droot) == 1;  // selects, not an indexed parameter array
  T* __restrict__ ok = (T*)(odd ? buf.k[1] : buf.k[0]);
  if (V) {
    uint32_t* pay = (uint32_t*)meta;  // the node list is no longer needed
    const uint32_t* __restrict__ gv = buf.v[0];
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      const int32_t p = tid + u * kSubThreads;
      if (p < m) pay[p] = gv[lo + p];
    }
    __syncthreads();
    uint32_t* __restrict__ ov = odd ? buf.v[1] : buf.v[0];
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      const int32_t p = tid + u * kSubThreads;
      if (p < m) {
        const R x = E::ld(X, sub_slot<E>(p));
        ok[lo + p] = E::key(x);
        ov[lo + p] = PS_IN_RANGE(E::pos(x), m) ? pay[E::pos(x)] : 0u;
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      const int32_t p = tid + u * kSubThreads;
      if (p < m) ok[lo + p] = E::key(E::ld(X, sub_slot<E>(p)));
    }
  }
}

// CTAs per SM the one-task kernel's register budget is sized for: 4 for 4-byte keys (shared
// memory holds no more); 5 for 8-byte keys, whose tasks need 37 KB (measured 2.3% faster on the
// uint64 Pareto sort than 4, and than 6, where the 40-register budget spills).
template <class K>
__host__ __device__ constexpr int sub_min_blocks() { return sizeof(typename K::T) == 8 ? 5 : 4; }

// One CTA per task.  cap != 0: the grid covers the tasks up to a bound that the host computed
// without the plan (device-driven calls); CTAs past the plan's count return at once.
template <class K, bool V>
__global__ void __launch_bounds__(kSubThreads, sub_min_blocks<K>())
subtree_kernel(Bufs buf, const pos_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
               const int32_t* __restrict__ nodeL, const int32_t* __restrict__ nodeR,
               const uint8_t* __restrict__ ndepth, const uint8_t* __restrict__ ldepth,
               const uint8_t* __restrict__ micro, const int32_t* __restrict__ tasks, uint32_t cap,
               PlanHeader* __restrict__ hdr, uint32_t* lib_status) {
  if (cap != 0) {  // both header words read at once: a surplus CTA returns after one load latency
    const uint32_t n_small = hdr->n_small, status = hdr->status;
    if (blockIdx.x >= min(n_small, cap) || (status & kDevBadOffsets)) return;
  }
  subtree_task<K, V>(buf, S, run_desc, nodeL, nodeR, ndepth, ldepth, micro, tasks[blockIdx.x], hdr, lib_status);
}

// The tasks past the one-task grid of a device-driven call (tasks first, .. of the plan's count;
// none for the inputs the grid's bound covers): a persistent grid whose CTAs take tasks from a
// counter in the plan header.  Its task loop needs far more registers than the one-task kernel
// (it spills), which is why it only takes what the one-task grid cannot.
template <class K, bool V>
__global__ void __launch_bounds__(kSubThreads, 4)
subtree_persistent_kernel(Bufs buf, const pos_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
                          const int32_t* __restrict__ nodeL, const int32_t* __restrict__ nodeR,
                          const uint8_t* __restrict__ ndepth, const uint8_t* __restrict__ ldepth,
                          const uint8_t* __restrict__ micro, const int32_t* __restrict__ tasks, uint32_t first,
                          uint32_t cap, PlanHeader* __restrict__ hdr,
                          uint32_t* lib_status) {
  if (hdr->status & kDevBadOffsets) return;  // nothing moves when the offsets were rejected
  const uint32_t ntasks = min(hdr->n_small, cap);
  __shared__ uint32_t s_task;
  for (;;) {
    if (threadIdx.x == 0) s_task = first + atomicAdd(&hdr->small_next, 1u);
    __syncthreads();
    const uint32_t tb = s_task;
    if (tb >= ntasks) break;  // uniform over the CTA
    subtree_task<K, V>(buf, S, run_desc, nodeL, nodeR, ndepth, ldepth, micro, tasks[tb], hdr, lib_status);
    __syncthreads();  // the next task reuses the shared arrays (and s_task)
  }
}

// ---------------------------------------------------------------------------------------
// Large leaves whose depth maps to the scratch buffer -> copied there (reversed if
// descending); the others, if descending -> reversed in place.  Work is cut into tiles of
// kMergeTile outputs (or pairs); a CTA owns a contiguous range of tiles, finds the leaf of its
// first tile once and walks the leaf list from there.
// ---------------------------------------------------------------------------------------
template <class K, bool V>
__device__ __forceinline__ void leaf_place_one(Bufs buf, const pos_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
                                               const uint8_t* __restrict__ ldepth, int32_t i, uint32_t k) {
  typedef typename K::T T;
  constexpr int kPer = kMergeTile / 256;  // elements (or pairs) per thread
  const int64_t s = S[i], e = S[i + 1];
  const bool desc = (run_desc[i] & 1) != 0;  // extended runs (bit 1) are short: never placed here
  const T* __restrict__ k0 = (const T*)buf.k[0];
  const uint32_t* __restrict__ v0 = buf.v[0];
  // all loads of the thread first (independent, coalesced even when reversed), then the stores;
  // 64-bit tile bases, 32-bit offsets inside the tile
  T kx[kPer], ky[kPer];
  uint32_t vx[kPer], vy[kPer];
  const int64_t base = s + (int64_t)k * kMergeTile;
  if (out_buffer(ldepth[i]) == 1) {
    // copy to the scratch buffer; element off of the tile comes from base + off, or from its
    // mirror s + e - 1 - (base + off) when the run is descending
    T* __restrict__ k1 = (T*)buf.k[1] + base;
    uint32_t* __restrict__ v1 = buf.v[1] + base;
    const int32_t cnt = (int32_t)min((int64_t)kMergeTile, e - base);
    const int64_t from = desc ? s + e - 1 - base : base;
    const T* __restrict__ ks = k0 + from;
    const uint32_t* __restrict__ vs = v0 + from;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int32_t off = (int32_t)threadIdx.x + u * 256;
      if (off < cnt) {
        const int32_t src = desc ? -off : off;
        kx[u] = ks[src];
        if (V) vx[u] = vs[src];
      }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int32_t off = (int32_t)threadIdx.x + u * 256;
      if (off < cnt) {
        k1[off] = kx[u];
        if (V) v1[off] = vx[u];
      }
    }
  } else {
    // a descending run that is a whole segment: reversed in place, pairs (p, s + e - 1 - p) for p
    // in the first half; the tile holds p = base + off, its partner is mirror - off
    T* __restrict__ kk = (T*)buf.k[0];
    uint32_t* __restrict__ vv = buf.v[0];
    const int32_t cnt = (int32_t)min((int64_t)kMergeTile, s + (e - s) / 2 - base);
    T* __restrict__ klo = kk + base;
    T* __restrict__ khi = kk + (s + e - 1 - base);
    uint32_t* __restrict__ vlo = vv + base;
    uint32_t* __restrict__ vhi = vv + (s + e - 1 - base);
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int32_t off = (int32_t)threadIdx.x + u * 256;
      if (off < cnt) {
        kx[u] = klo[off];
        ky[u] = khi[-off];
        if (V) {
          vx[u] = vlo[off];
          vy[u] = vhi[-off];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int32_t off = (int32_t)threadIdx.x + u * 256;
      if (off < cnt) {
        klo[off] = ky[u];
        khi[-off] = kx[u];
        if (V) {
          vlo[off] = vy[u];
          vhi[-off] = vx[u];
        }
      }
    }
  }
}

// Tiles [t_begin, t_end) of the leaf list (items[slot] = leaf, its first tile tile_off[slot]).
// Tiles touch disjoint elements, so the threads need no barrier between tiles.
template <class K, bool V>
__device__ __forceinline__ void leaf_place_range(Bufs buf, const pos_t* __restrict__ S,
                                                 const uint8_t* __restrict__ run_desc,
                                                 const uint8_t* __restrict__ ldepth, const int32_t* __restrict__ items,
                                                 const uint32_t* __restrict__ tile_off, uint32_t nitems,
                                                 uint32_t t_begin, uint32_t t_end, int32_t runs) {
  __shared__ int32_t s_slot;
  if (t_begin >= t_end || nitems == 0) return;  // uniform over the CTA
  if (threadIdx.x == 0) s_slot = slot_of_tile(tile_off, nitems, t_begin);
  __syncthreads();
  int32_t slot = s_slot;
  for (uint32_t tile = t_begin; tile < t_end; ++tile) {
    while (slot + 1 < (int32_t)nitems && tile_off[slot + 1] <= tile) ++slot;
    const int32_t i = items[slot];
    if (i < 0 || i >= runs) return;  // never for a consistent plan (uniform over the CTA)
    leaf_place_one<K, V>(buf, S, run_desc, ldepth, i, tile - tile_off[slot]);
  }
}

// CTAs per SM the placement kernels keep resident (their registers hold a thread's whole share
// of a tile: 12 keys and payloads, or pairs of them).
template <class K>
__host__ __device__ constexpr int leaf_place_min_blocks() { return sizeof(typename K::T) == 4 ? 3 : 2; }

// Grid over the counts known on the host: CTA b owns tiles [b*T/G, (b+1)*T/G).
template <class K, bool V>
__global__ void __launch_bounds__(256, leaf_place_min_blocks<K>())
leaf_place_kernel(Bufs buf, const pos_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
                  const uint8_t* __restrict__ ldepth, const int32_t* __restrict__ items,
                  const uint32_t* __restrict__ tile_off, uint32_t nitems, uint32_t ntiles,
                  const PlanHeader* __restrict__ hdr) {
  const uint32_t t0 = (uint32_t)(((uint64_t)blockIdx.x * ntiles) / gridDim.x);
  const uint32_t t1 = (uint32_t)(((uint64_t)(blockIdx.x + 1) * ntiles) / gridDim.x);
  leaf_place_range<K, V>(buf, S, run_desc, ldepth, items, tile_off, nitems, t0, t1, hdr->runs);
}

// The same over the counts the plan left on the device (no host round trip).
template <class K, bool V>
__global__ void __launch_bounds__(256, leaf_place_min_blocks<K>())
leaf_place_persistent_kernel(Bufs buf, const pos_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
                             const uint8_t* __restrict__ ldepth, const int32_t* __restrict__ items,
                             const uint32_t* __restrict__ tile_off, uint32_t cap,
                             const PlanHeader* __restrict__ hdr) {
  if (hdr->status & kDevBadOffsets) return;
  const unsigned long long v = hdr->leaf_ctr;
  const uint32_t nitems = min((uint32_t)(v >> 32), cap);
  const uint32_t ntiles = (uint32_t)(v & 0xffffffffull);
  const uint32_t t0 = (uint32_t)(((uint64_t)blockIdx.x * ntiles) / gridDim.x);
  const uint32_t t1 = (uint32_t)(((uint64_t)(blockIdx.x + 1) * ntiles) / gridDim.x);
  leaf_place_range<K, V>(buf, S, run_desc, ldepth, items, tile_off, nitems, t0, t1, hdr->runs);
}

}  // namespace ps
