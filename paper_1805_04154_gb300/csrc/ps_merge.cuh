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
//  * leaf_place_kernel   large leaves: odd depth -> copy to the scratch buffer, descending ->
//                        reversed.
//  * level_pass_kernel   persistent, warp-specialized level pass: a producer warp finds each
//                        tile's co-rank and stages both input ranges into shared memory with bulk
//                        (TMA) copies on mbarriers; consumer warps merge IPT outputs per
//                        thread and write them with 128-bit stores.
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
  __device__ __forceinline__ static R ld(const Arr& a, int32_t i) { return a.w[i]; }
  __device__ __forceinline__ static void st(const Arr& a, int32_t i, R x) { a.w[i] = x; }
  __device__ __forceinline__ static R make(uint32_t key, int32_t pos) {
    return ((uint64_t)K::ord(key) << 32) | (uint32_t)pos;
  }
  // positions differ, so two elements never compare equal
  __device__ __forceinline__ static bool before(R a, R b) { return a < b; }
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
  __device__ __forceinline__ static R ld(const Arr& a, int32_t i) { return R{a.k[i], a.p[i]}; }
  __device__ __forceinline__ static void st(const Arr& a, int32_t i, R x) {
    a.k[i] = x.k;
    a.p[i] = x.p;
  }
  __device__ __forceinline__ static R make(uint64_t key, int32_t pos) { return R{key, (uint32_t)pos}; }
  // a comes from the left child: it goes first unless its key is greater
  __device__ __forceinline__ static bool before(const R& a, const R& b) { return K::le(a.k, b.k); }
  __device__ __forceinline__ static uint64_t key(const R& x) { return x.k; }
  __device__ __forceinline__ static int32_t pos(const R& x) { return (int32_t)x.p; }
};

// padded slot of position p
template <class E>
__device__ __forceinline__ int32_t sub_slot(int32_t p) {
  return p + p / E::IPT;
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
__device__ __forceinline__ void subtree_task(Bufs buf, const int32_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
                                             const int32_t* __restrict__ nodeL, const int32_t* __restrict__ nodeR,
                                             const uint8_t* __restrict__ ndepth, const uint8_t* __restrict__ ldepth,
                                             const int32_t task, int fused, PlanHeader* __restrict__ hdr,
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
  const int32_t lo = S[L], m = S[R_] - lo, nr = R_ - L;
  if (m > TS || nr + 1 > RC) {  // cannot happen for a greedy run partition; never overrun SMEM
    if (tid == 0) post_status(&hdr->status, lib_status, kDevInternal);
    return;
  }

  // 1. run starts and directions; the keys, tagged with their positions
  int16_t* rs = (int16_t*)meta;
  uint8_t* rdsc = (uint8_t*)(rs + RC);
  bool any_desc = false;
  for (int32_t k = tid; k <= nr; k += kSubThreads) {
    rs[k] = (int16_t)(S[L + k] - lo);
    if (k < nr) {
      rdsc[k] = run_desc[L + k];
      any_desc |= rdsc[k] != 0;
    }
  }
  const T* __restrict__ gk = (const T*)buf.k[0];
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    const int32_t p = tid + u * kSubThreads;
    if (p < m) E::st(X, sub_slot<E>(p), E::make(gk[lo + p], p));
  }
  for (int t = tid; t < NW * kMaxLevels; t += kSubThreads) (&s_cnt[0][0])[t] = 0;
  if (tid == 0) s_maxrd = -1;
  const int anyd = __syncthreads_or(any_desc);

  // 2. descending runs reversed in place, through registers
  const int32_t cs = tid * IPT;
  if (anyd) {
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
          if (rdsc[k]) {
            const int32_t src = (int32_t)rs[k] + rs[k + 1] - 1 - p;
            if (src != p) {
              v[q] = E::ld(X, sub_slot<E>(src));
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

  // 3. the nodes (boundaries 1..nr-1), sorted by relative depth and by position inside a depth:
  //    a counting sort over warp chunks (match_any groups a warp's equal depths)
  const int32_t chunk = (nr - 1 + NW - 1) / NW;
  const int32_t w0 = 1 + warp * chunk, w1 = min(1 + (warp + 1) * chunk, nr);
  bool bad = false;
  int my_max = -1;
  for (int32_t k0 = w0; k0 < w1; k0 += 32) {
    const int32_t k = k0 + lane;
    int rd = kMaxLevels;  // lanes past the chunk form their own group
    if (k < w1) {
      rd = (int)ndepth[L + k] - droot;
      if (rd < 0 || rd >= kMaxLevels) {
        bad = true;
        rd = 0;
      }
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, rd);
    if (k < w1) {
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
  uint64_t* ent = (uint64_t*)meta;  // node: lo | mid << 16 | hi << 32 (task-relative)
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int32_t k0 = w0; k0 < w1; k0 += 32) {
    const int32_t k = k0 + lane;
    int rd = kMaxLevels;
    if (k < w1) rd = min(max((int)ndepth[L + k] - droot, 0), kMaxLevels - 1);
    const uint32_t peers = __match_any_sync(0xffffffffu, rd);
    if (k < w1) {
      const int32_t j = L + k;
      const int32_t at = s_cnt[warp][rd] + __popc(peers & lt_mask);
      const uint32_t nlo = (uint32_t)(S[nodeL[j]] - lo), nmid = (uint32_t)(S[j] - lo);
      const uint32_t nhi = (uint32_t)(S[nodeR[j]] - lo);
      ent[at] = (uint64_t)(nlo | (nmid << 16)) | ((uint64_t)nhi << 32);
    }
    __syncwarp();
    if (k < w1 && lane == __ffs(peers) - 1) s_cnt[warp][rd] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();

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
  const bool odd = out_buffer(droot, fused != 0) == 1;  // selects, not an indexed parameter array
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
        ov[lo + p] = pay[E::pos(x)];
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

// One CTA per task, or (ntasks == kCountOnDevice) a persistent grid over the plan's task count.
template <class K, bool V>
__global__ void __launch_bounds__(kSubThreads, 4)
subtree_kernel(Bufs buf, const int32_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
               const int32_t* __restrict__ nodeL, const int32_t* __restrict__ nodeR,
               const uint8_t* __restrict__ ndepth, const uint8_t* __restrict__ ldepth,
               const int32_t* __restrict__ tasks, uint32_t ntasks, uint32_t cap, int fused,
               PlanHeader* __restrict__ hdr, uint32_t* lib_status) {
  if (ntasks == kCountOnDevice) {
    if (hdr->status & kDevBadOffsets) return;  // nothing moves when the offsets were rejected
    ntasks = min(hdr->n_small, cap);
  }
  for (uint32_t tb = blockIdx.x; tb < ntasks; tb += gridDim.x) {
    subtree_task<K, V>(buf, S, run_desc, nodeL, nodeR, ndepth, ldepth, tasks[tb], fused, hdr, lib_status);
    __syncthreads();  // the next task reuses the shared arrays
  }
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

// ---------------------------------------------------------------------------------------
// Large leaves whose depth maps to the scratch buffer -> copied there (reversed if
// descending); the others, if descending -> reversed in place.  One CTA per kMergeTile outputs
// (or pairs).
// ---------------------------------------------------------------------------------------
template <class K, bool V>
__device__ __forceinline__ void leaf_place_tile(Bufs buf, const int32_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
                                                const uint8_t* __restrict__ ldepth, const int32_t* __restrict__ items,
                                                const uint32_t* __restrict__ tile_off, uint32_t nitems, uint32_t tile,
                                                int fused, int32_t runs) {
  typedef typename K::T T;
  constexpr int kPer = kMergeTile / 256;  // elements (or pairs) per thread
  __shared__ int32_t s_slot;
  if (threadIdx.x == 0) s_slot = slot_of_tile(tile_off, nitems, tile);
  __syncthreads();
  const int32_t slot = s_slot;
  const int32_t i = items[slot];
  if (i < 0 || i >= runs) return;  // never for a consistent plan (uniform over the CTA)
  const int32_t k = (int32_t)(tile - tile_off[slot]);
  const int32_t s = S[i], e = S[i + 1];
  const bool desc = run_desc[i] != 0;
  const T* __restrict__ k0 = (const T*)buf.k[0];
  const uint32_t* __restrict__ v0 = buf.v[0];
  // all loads of the thread first (independent, coalesced even when reversed), then the stores
  T kx[kPer], ky[kPer];
  uint32_t vx[kPer], vy[kPer];
  if (out_buffer(ldepth[i], fused != 0) == 1) {
    T* __restrict__ k1 = (T*)buf.k[1];
    uint32_t* __restrict__ v1 = buf.v[1];
    const int32_t q0 = s + k * kMergeTile + threadIdx.x, q1 = min(e, s + (k + 1) * kMergeTile);
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int32_t q = q0 + u * 256;
      if (q < q1) {
        const int32_t src = desc ? s + e - 1 - q : q;
        kx[u] = k0[src];
        if (V) vx[u] = v0[src];
      }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int32_t q = q0 + u * 256;
      if (q < q1) {
        k1[q] = kx[u];
        if (V) v1[q] = vx[u];
      }
    }
  } else {
    T* kk = (T*)buf.k[0];
    uint32_t* vv = buf.v[0];
    const int32_t half = (e - s) / 2;
    const int32_t p0 = s + k * kMergeTile + threadIdx.x, p1 = min(s + half, s + (k + 1) * kMergeTile);
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int32_t p = p0 + u * 256;
      if (p < p1) {
        const int32_t q = s + e - 1 - p;
        kx[u] = kk[p];
        ky[u] = kk[q];
        if (V) {
          vx[u] = vv[p];
          vy[u] = vv[q];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int32_t p = p0 + u * 256;
      if (p < p1) {
        const int32_t q = s + e - 1 - p;
        kk[p] = ky[u];
        kk[q] = kx[u];
        if (V) {
          vv[p] = vy[u];
          vv[q] = vx[u];
        }
      }
    }
  }
}

// One CTA per tile, or (ntiles == kCountOnDevice) a persistent grid over the plan's counts.
template <class K, bool V>
__global__ void __launch_bounds__(256)
leaf_place_kernel(Bufs buf, const int32_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
                  const uint8_t* __restrict__ ldepth, const int32_t* __restrict__ items,
                  const uint32_t* __restrict__ tile_off, uint32_t nitems, uint32_t ntiles, uint32_t cap, int fused,
                  const PlanHeader* __restrict__ hdr) {
  if (ntiles == kCountOnDevice) {
    if (hdr->status & kDevBadOffsets) return;
    const unsigned long long v = hdr->leaf_ctr;
    nitems = min((uint32_t)(v >> 32), cap);
    ntiles = (uint32_t)(v & 0xffffffffull);
    if (nitems == 0) return;
  }
  const int32_t runs = hdr->runs;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    leaf_place_tile<K, V>(buf, S, run_desc, ldepth, items, tile_off, nitems, tile, fused, runs);
    __syncthreads();  // s_slot is rewritten by the next tile
  }
}

// ---------------------------------------------------------------------------------------
// One level pass: all merges of the tree nodes at one depth whose ranges exceed the subtree
// limit, split into output tiles that start at the node's lo and then at the multiples of the
// tile size (IPT outputs per consumer thread x 256 threads) inside it.  Persistent and warp-specialized:
//  * CTA b owns the contiguous tile range [b*T/G, (b+1)*T/G) of the pass (T tiles, G CTAs), so
//    the co-rank at the end of one tile is the co-rank at the start of the next;
//  * warp 8 (producer) walks the CTA's tiles: it finds each tile's end co-rank with a 32-way
//    warp search inside the window the start co-rank allows (at most one tile wide; its
//    probes touch the lines the tile's copy then reads), waits for a free stage, and issues the
//    tile's four bulk copies (left/right keys and payloads, 16-byte aligned chunks) on that
//    stage's "full" mbarrier;
//  * warps 0-7 (consumers) wait for a full stage, merge its IPT outputs per thread
//    (co-rank inside shared memory, then a serial stable merge), write them with 128-bit
//    stores, and release the stage on its "empty" mbarrier.
// A ring of NS stages: the copies of the next NS-1 tiles overlap the merge of the current one.
// All waits are bounded; a timeout posts kDevTimeout and the CTA drains its copies and exits.
// ---------------------------------------------------------------------------------------
constexpr int kPassThreads = kMergeThreads + 32;  // 8 consumer warps + 1 producer warp

struct StageDesc {
  int32_t g0, g1, i0, i1;   // outputs [g0, g1); left elements [i0, i1) of the node
  int32_t lo, mid, la, lb;  // node [lo, mid) + [mid, hi)
  int32_t aoff, boff, vaoff, vboff;  // smem element offsets of A[i0], B[j0] (keys / payloads)
  int32_t pad[4];
};

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
  static constexpr size_t kFlagOff = kDescOff + NS * sizeof(StageDesc);
  static constexpr size_t kStageOff = (kFlagOff + 16 + 127) & ~(size_t)127;
  static constexpr size_t kBytes = kStageOff + NS * kStageBytes;
};

// smallest i in [a, b] with i == b or A[i] > B[diag-1-i], by a 32-way warp search in global memory
template <class K>
__device__ __forceinline__ int32_t warp_corank(const typename K::T* __restrict__ A, const typename K::T* __restrict__ B,
                                               int32_t diag, int32_t a, int32_t b) {
  const int lane = threadIdx.x & 31;
  while (a < b) {
    const int32_t span = b - a;
    const int32_t x = a + (int32_t)(((int64_t)span * lane) >> 5);  // probes in [a, b)
    const bool gt = !key_le<K>(A[x], B[diag - 1 - x]);
    const uint32_t mask = __ballot_sync(0xffffffffu, gt);
    if (mask) {
      const int fl = __ffs(mask) - 1;
      const int32_t xf = __shfl_sync(0xffffffffu, x, fl);
      const int32_t xp = __shfl_sync(0xffffffffu, x, fl > 0 ? fl - 1 : 0);
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
__device__ __forceinline__ void chunk16(const E* base, int32_t e0, int32_t e1, int32_t& c0, int32_t& c1) {
  constexpr int kPer = 16 / (int)sizeof(E);
  const int32_t phase = (int32_t)(((uintptr_t)base & 15u) / sizeof(E));  // elements before base in its block
  c0 = ((e0 + phase) & ~(kPer - 1)) - phase;
  c1 = (e1 > e0) ? (((e1 + phase + kPer - 1) & ~(kPer - 1)) - phase) : c0;
}

__device__ __forceinline__ bool bounded_wait(uint64_t* bar, uint32_t parity) {
  uint32_t tries = 0;
  while (!mbar_try_wait(bar, parity))
    if (++tries > kMbarTries) return false;
  return true;
}

// CTAs per SM the register budget is sized for (16 items per thread need more registers).
__host__ __device__ constexpr int pass_min_blocks(int ipt) { return ipt <= 12 ? 4 : 3; }

template <class K, bool V, int NS, int IPT>
__global__ void __launch_bounds__(kPassThreads, pass_min_blocks(IPT))
level_pass_kernel(const typename K::T* __restrict__ srck, const uint32_t* __restrict__ srcv,
                  typename K::T* __restrict__ dstk, uint32_t* __restrict__ dstv,
                  const int4* __restrict__ nodes, const uint32_t* __restrict__ tile_off, uint32_t nitems,
                  uint32_t ntiles, const unsigned long long* __restrict__ ctr, uint32_t cap,
                  PlanHeader* __restrict__ hdr, uint32_t* lib_status) {
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
  constexpr int KU = Lay::KU;
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
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPassStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kMergeThreads / 32);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kMergeThreads / 32) {
    // ------------------------------ producer ------------------------------
    int32_t slot = 0;
    if (lane == 0) slot = slot_of_tile(tile_off, nitems, t_begin);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    int4 nd = nodes[slot];  // lo, mid, hi, boundary
    int32_t la = nd.y - nd.x, lb = nd.z - nd.y;
    const T* A = srck + nd.x;
    const T* B = srck + nd.y;
    const int32_t k0 = (int32_t)(t_begin - tile_off[slot]);
    int32_t g0 = (k0 == 0) ? nd.x : (nd.x / kTile + k0) * kTile;
    int32_t i0 = 0;
    if (g0 > nd.x) {
      const int32_t diag = g0 - nd.x;
      i0 = warp_corank<K>(A, B, diag, max(0, diag - lb), min(diag, la));
    }
    // Tiles go out in batches of kSearchBatch: lane group m (8 lanes) finds the end co-rank of
    // the batch's tile m with an 8-way search, all groups at once.  Each window is anchored at
    // the last co-rank known in the same node (the batch start, or 0 at a node's first tile),
    // so it is at most kSearchBatch tiles wide.
    constexpr int kSearchBatch = 4;
    const int grp = lane >> 3, gl = lane & 7;
    const uint32_t gmask = 0xFFu << (grp * 8);
    uint32_t issued = 0;
    bool ok = true;
    uint32_t t = t_begin;
    while (t < t_end && ok) {
      const int nb = (int)min((uint32_t)kSearchBatch, t_end - t);
      int4 m_nd[kSearchBatch];
      int32_t m_g0[kSearchBatch], m_g1[kSearchBatch], m_slot[kSearchBatch], m_a[kSearchBatch], m_b[kSearchBatch];
      bool m_new[kSearchBatch];
      {
        int32_t cs = slot, cg0 = g0, ag = g0, ai = i0;
        int4 cnd = nd;
#pragma unroll
        for (int m = 0; m < kSearchBatch; ++m) {
          m_new[m] = false;
          if (m < nb) {
            const uint32_t tt = t + m;
            if (cs + 1 < (int32_t)nitems && tile_off[cs + 1] <= tt) {
              while (cs + 1 < (int32_t)nitems && tile_off[cs + 1] <= tt) ++cs;
              cnd = nodes[cs];
              cg0 = cnd.x;
              ag = cnd.x;
              ai = 0;
              m_new[m] = true;
            }
            const int32_t g1 = min(cnd.z, (cg0 / kTile + 1) * kTile);
            const int32_t cla = cnd.y - cnd.x, clb = cnd.z - cnd.y, diag = g1 - cnd.x;
            m_nd[m] = cnd;
            m_slot[m] = cs;
            m_g0[m] = cg0;
            m_g1[m] = g1;
            // window of the end co-rank (empty window when the tile ends at the node's end)
            m_a[m] = (g1 < cnd.z) ? max(ai, diag - clb) : cla;
            m_b[m] = (g1 < cnd.z) ? min(ai + (g1 - ag), cla) : cla;
            cg0 = g1;
          }
        }
      }
      // group grp searches tile grp (8-way probes)
      int32_t res = 0;
      {
        int4 snd = m_nd[0];
        int32_t sa = m_a[0], sb = m_b[0], sg1 = m_g1[0];
#pragma unroll
        for (int m = 1; m < kSearchBatch; ++m)
          if (grp == m) {
            snd = m_nd[m];
            sa = m_a[m];
            sb = m_b[m];
            sg1 = m_g1[m];
          }
        if (grp < nb) {
          const T* GA = srck + snd.x;
          const T* GB = srck + snd.y;
          const int32_t diag = sg1 - snd.x;
          int32_t ga = sa, gb = sb;
          while (ga < gb) {
            const int32_t span = gb - ga;
            const int32_t x = ga + (int32_t)(((int64_t)span * gl) >> 3);
            const bool gt = !key_le<K>(GA[x], GB[diag - 1 - x]);
            const uint32_t msk = (__ballot_sync(gmask, gt) >> (grp * 8)) & 0xFFu;
            if (msk) {
              const int fl = __ffs(msk) - 1;
              const int32_t xf = __shfl_sync(gmask, x, grp * 8 + fl);
              const int32_t xp = __shfl_sync(gmask, x, grp * 8 + (fl > 0 ? fl - 1 : 0));
              gb = xf;
              if (fl > 0) ga = xp + 1;
            } else {
              ga = __shfl_sync(gmask, x, grp * 8 + 7) + 1;
            }
          }
          res = ga;
        }
      }
      int32_t m_i1[kSearchBatch];
#pragma unroll
      for (int m = 0; m < kSearchBatch; ++m) m_i1[m] = __shfl_sync(0xffffffffu, res, m * 8);
      // issue the batch in order
#pragma unroll
      for (int m = 0; m < kSearchBatch; ++m) {
        if (m < nb && ok) {
          const int4 cnd = m_nd[m];
          const int32_t cla = cnd.y - cnd.x;
          const int32_t tg0 = m_g0[m], tg1 = m_g1[m];
          const int32_t ti0 = m_new[m] ? 0 : (m == 0 ? i0 : m_i1[m - 1]);
          const int32_t ti1 = (tg1 < cnd.z) ? m_i1[m] : cla;
          const int s = (int)(issued % kPassStages);
          const uint32_t use = issued / kPassStages;
          if (!__all_sync(0xffffffffu, bounded_wait(&empty[s], (use & 1u) ^ 1u))) {
            ok = false;
          } else {
            if (lane == 0) {
              const int32_t a0 = cnd.x + ti0, a1 = cnd.x + ti1;
              const int32_t b0 = cnd.y + (tg0 - cnd.x - ti0), b1 = cnd.y + (tg1 - cnd.x - ti1);
              // 16-byte aligned enclosing chunks, computed on absolute addresses (the arrays only
              // need natural alignment; a chunk may start up to 15 bytes before a range and end up
              // to 15 bytes after it, always inside 16-byte blocks holding range elements)
              int32_t ka0, ka1, kb0, kb1, va0, va1, vb0, vb1;
              chunk16(srck, a0, a1, ka0, ka1);
              chunk16(srck, b0, b1, kb0, kb1);
              chunk16(srcv, a0, a1, va0, va1);
              chunk16(srcv, b0, b1, vb0, vb1);
              StageDesc d;
              d.g0 = tg0;
              d.g1 = tg1;
              d.i0 = ti0;
              d.i1 = ti1;
              d.lo = cnd.x;
              d.mid = cnd.y;
              d.la = cla;
              d.lb = cnd.z - cnd.y;
              d.aoff = a0 - ka0;
              d.boff = (ka1 - ka0) + (b0 - kb0);
              d.vaoff = a0 - va0;
              d.vboff = (va1 - va0) + (b0 - vb0);
              sdesc[s] = d;
              uint8_t* stage = smem + Lay::kStageOff + (size_t)s * Lay::kStageBytes;
              T* sk = (T*)stage;
              uint32_t* sv = (uint32_t*)(stage + Lay::kKeyBytes);
              const uint32_t kba = (uint32_t)(ka1 - ka0) * sizeof(T), kbb = (uint32_t)(kb1 - kb0) * sizeof(T);
              const uint32_t vba = V ? (uint32_t)(va1 - va0) * 4u : 0u, vbb = V ? (uint32_t)(vb1 - vb0) * 4u : 0u;
              mbar_arrive_expect_tx(&full[s], kba + kbb + vba + vbb);
              if (kba) bulk_g2s(sk, srck + ka0, kba, &full[s]);
              if (kbb) bulk_g2s(sk + (ka1 - ka0), srck + kb0, kbb, &full[s]);
              if (V) {
                if (vba) bulk_g2s(sv, srcv + va0, vba, &full[s]);
                if (vbb) bulk_g2s(sv + (va1 - va0), srcv + vb0, vbb, &full[s]);
              }
            }
            __syncwarp();
            ++issued;
          }
        }
      }
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
          i0 = (m_g1[m] < m_nd[m].z) ? m_i1[m] : (m_nd[m].y - m_nd[m].x);
        }
      if (nb == 1) i0 = (m_g1[0] < m_nd[0].z) ? m_i1[0] : (m_nd[0].y - m_nd[0].x);
      t += nb;
    }
    if (!ok) {
      if (lane == 0) post_status(&hdr->status, lib_status, kDevTimeout);
      *abort_flag = 1;
    }
    // drain: every copy issued into a stage must have landed before the CTA exits
    if (lane == 0) {
      for (uint32_t q = (issued > kPassStages ? issued - kPassStages : 0); q < issued; ++q) {
        const int s = (int)(q % kPassStages);
        bounded_wait(&full[s], (q / kPassStages) & 1u);
      }
    }
  } else {
    // ------------------------------ consumers ------------------------------
    const int tid = threadIdx.x;
    uint32_t it = 0;
    for (uint32_t t = t_begin; t < t_end; ++t, ++it) {
      const int s = (int)(it % kPassStages);
      const uint32_t use = it / kPassStages;
      bool ready = false;
      for (uint32_t tries = 0; tries < kMbarTries; ++tries) {
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
      const T* A = (const T*)stage + d.aoff;
      const T* B = (const T*)stage + d.boff;
      const uint32_t* sv = (const uint32_t*)(stage + Lay::kKeyBytes);
      const int32_t len = d.g1 - d.g0, la = d.i1 - d.i0, lb = len - la;
      const int32_t diag = tid * IPT;
      if (diag < len) {
        int32_t i = corank_serial<K>(A, B, la, lb, diag);
        int32_t j = diag - i;
        const int32_t cnt = min(IPT, len - diag);
        T key[IPT];
        uint32_t val[IPT];
        // heads of both inputs stay in registers: one shared-memory key read per output
        T a = A[min(i, la - 1 >= 0 ? la - 1 : 0)], b = B[min(j, lb - 1 >= 0 ? lb - 1 : 0)];
        if (cnt == IPT) {
#pragma unroll
          for (int q = 0; q < IPT; ++q) {
            const bool takeA = (j >= lb) || (i < la && key_le<K>(a, b));
            key[q] = takeA ? a : b;
            if (V) val[q] = sv[takeA ? d.vaoff + i : d.vboff + j];
            i += takeA ? 1 : 0;
            j += takeA ? 0 : 1;
            if (takeA) {
              if (i < la) a = A[i];
            } else {
              if (j < lb) b = B[j];
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < IPT; ++q) {
            if (q < cnt) {
              const bool takeA = (j >= lb) || (i < la && key_le<K>(a, b));
              key[q] = takeA ? a : b;
              if (V) val[q] = sv[takeA ? d.vaoff + i : d.vboff + j];
              i += takeA ? 1 : 0;
              j += takeA ? 0 : 1;
              if (takeA) {
                if (i < la) a = A[i];
              } else {
                if (j < lb) b = B[j];
              }
            }
          }
        }
        const int32_t g = d.g0 + diag;
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
        } else {
#pragma unroll
          for (int q = 0; q < IPT; ++q)
            if (q < cnt) dstk[g + q] = key[q];
        }
        if (V) {
          if (cnt == IPT && ((uintptr_t)(dstv + g) & 15u) == 0) {
            uint4* o = (uint4*)(dstv + g);
#pragma unroll
            for (int q = 0; q < IPT / 4; ++q)
              o[q] = make_uint4(val[4 * q], val[4 * q + 1], val[4 * q + 2], val[4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < IPT; ++q)
              if (q < cnt) dstv[g + q] = val[q];
          }
        }
      }
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(&empty[s]);
    }
  }
}

}  // namespace ps
