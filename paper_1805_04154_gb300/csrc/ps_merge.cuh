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
//  * corank_kernel       one warp per output tile: 32-way co-rank search in global memory.
//  * merge_tile_kernel   one CTA per output tile: both input ranges staged into shared memory by
//                        bulk (TMA) copies on an mbarrier, per-thread co-rank + serial merge of
//                        kMergeItems outputs, 128-bit stores.
#pragma once

#include "ps_common.cuh"

namespace ps {

struct Bufs {
  void* k[2];      // key buffers: [0] the caller's array, [1] scratch
  uint32_t* v[2];  // payload buffers (null when there is no payload)
};

template <class K>
__device__ __forceinline__ bool key_le(typename K::T a, typename K::T b) {
  return K::ord(a) <= K::ord(b);
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
// ---------------------------------------------------------------------------------------
template <class K, bool V>
struct SubLayout {
  typedef typename K::T T;
  static constexpr int TS = sub_tile((int)sizeof(T));
  static constexpr int RC = TS / 2 + 2;  // runs in a task: all but a segment's last have length >= 2
  static constexpr int IPT = TS / kSubThreads;
  static constexpr size_t kKeys = 2 * (size_t)TS * sizeof(T);
  static constexpr size_t kVals = V ? 2 * (size_t)TS * 4 : 0;
  static constexpr size_t kMeta = (size_t)RC * (2 + 2 + 2 + 2 + 1 + 1);
  static constexpr size_t kBytes = kKeys + kVals + kMeta;
};

template <class K, bool V>
__global__ void __launch_bounds__(kSubThreads)
subtree_kernel(Bufs buf, const int32_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
               const int32_t* __restrict__ nodeL, const int32_t* __restrict__ nodeR,
               const uint8_t* __restrict__ ndepth, const uint8_t* __restrict__ ldepth,
               const int32_t* __restrict__ tasks, PlanHeader* __restrict__ hdr, uint32_t* lib_status) {
  typedef typename K::T T;
  typedef SubLayout<K, V> Lay;
  constexpr int TS = Lay::TS, RC = Lay::RC, IPT = Lay::IPT;
  extern __shared__ __align__(128) uint8_t smem[];
  T* sk[2] = {(T*)smem, (T*)smem + TS};
  uint32_t* sv[2] = {nullptr, nullptr};
  uint8_t* meta = smem + Lay::kKeys;
  if (V) {
    sv[0] = (uint32_t*)(smem + Lay::kKeys);
    sv[1] = sv[0] + TS;
    meta += Lay::kVals;
  }
  int16_t* rs = (int16_t*)meta;   // local run starts, rs[nr] = m
  int16_t* nlo = rs + RC;         // node b: local [nlo, rs[b], nhi)
  int16_t* nhi = nlo + RC;
  int16_t* lvl = nhi + RC;        // boundaries of the current level, by position
  uint8_t* rinfo = (uint8_t*)(lvl + RC);  // leaf: (relative depth << 1) | descending
  uint8_t* nrd = rinfo + RC;              // node relative depth
  __shared__ int32_t s_wsum[kSubThreads / 32];
  __shared__ int32_t s_maxrd;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t task = tasks[blockIdx.x];
  int32_t L, R, droot;
  if (task >= 0) {
    L = nodeL[task];
    R = nodeR[task];
    droot = ndepth[task];
  } else {
    L = ~task;
    R = L + 1;
    droot = ldepth[L];
  }
  const int32_t lo = S[L], m = S[R] - lo, nr = R - L;
  if (m > TS || nr + 1 > RC) {  // cannot happen for a greedy run partition; never overrun SMEM
    if (tid == 0) post_status(&hdr->status, lib_status, kDevInternal);
    return;
  }
  if (tid == 0) s_maxrd = 0;
  __syncthreads();
  int my_max = 0;
  for (int32_t k = tid; k <= nr; k += kSubThreads) {
    rs[k] = (int16_t)(S[L + k] - lo);
    if (k < nr) {
      const int rd = (int)ldepth[L + k] - droot;
      rinfo[k] = (uint8_t)((rd << 1) | (run_desc[L + k] ? 1 : 0));
      my_max = max(my_max, rd);
    }
    if (k >= 1 && k < nr) {
      const int32_t j = L + k;
      nlo[k] = (int16_t)(S[nodeL[j]] - lo);
      nhi[k] = (int16_t)(S[nodeR[j]] - lo);
      nrd[k] = (uint8_t)((int)ndepth[j] - droot);
    }
  }
  my_max = __reduce_max_sync(0xffffffffu, my_max);
  if (lane == 0) atomicMax(&s_maxrd, my_max);
  __syncthreads();

  // place the leaves: leaf at relative depth d goes to buffer d mod 2, reversed if descending
  const T* gk = (const T*)buf.k[0];
  const uint32_t* gv = buf.v[0];
  {
    const int32_t p0 = tid * IPT;
    if (p0 < m) {
      int32_t a = 0, b = nr;  // run containing p0: largest k with rs[k] <= p0
      while (b - a > 1) {
        const int32_t mid = (a + b) >> 1;
        if (rs[mid] <= p0) a = mid; else b = mid;
      }
      int32_t k = a;
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        const int32_t p = p0 + q;
        if (p < m) {
          while (p >= rs[k + 1]) ++k;
          const uint8_t info = rinfo[k];
          const int32_t tgt = (info & 1) ? (int32_t)rs[k] + rs[k + 1] - 1 - p : p;
          const int bsel = (info >> 1) & 1;
          sk[bsel][tgt] = gk[lo + p];
          if (V) sv[bsel][tgt] = gv[lo + p];
        }
      }
    }
  }
  __syncthreads();

  const int32_t nb = nr - 1;                              // boundaries 1..nr-1
  const int32_t bpt = (nb + kSubThreads - 1) / kSubThreads;  // boundaries per thread
  for (int rd = s_maxrd - 1; rd >= 0; --rd) {
    // compact the boundaries of this level (in position order)
    const int32_t b0 = 1 + tid * bpt, b1 = min(1 + (tid + 1) * bpt, nr);
    int32_t c = 0;
    for (int32_t bb = b0; bb < b1; ++bb) c += (nrd[bb] == rd);
    int32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t o = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += o;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    int32_t off = inc - c, total = 0;
    for (int w = 0; w < kSubThreads / 32; ++w) {
      if (w < warp) off += s_wsum[w];
      total += s_wsum[w];
    }
    for (int32_t bb = b0; bb < b1; ++bb)
      if (nrd[bb] == rd) lvl[off++] = (int16_t)bb;
    __syncthreads();
    if (total == 0) continue;

    const T* srck = sk[(rd + 1) & 1];
    T* dstk = sk[rd & 1];
    const uint32_t* srcv = sv[(rd + 1) & 1];
    uint32_t* dstv = sv[rd & 1];
    const int32_t cs = tid * IPT, ce = min(m, cs + IPT);
    if (cs < ce) {
      int32_t a = 0, b = total;  // first node of the level with nhi > cs
      while (a < b) {
        const int32_t mid = (a + b) >> 1;
        if (nhi[lvl[mid]] <= cs) a = mid + 1; else b = mid;
      }
      for (int32_t idx = a; idx < total; ++idx) {
        const int32_t bnd = lvl[idx];
        const int32_t l = nlo[bnd];
        if (l >= ce) break;
        const int32_t mm = rs[bnd], h = nhi[bnd];
        const int32_t ps = max(cs, l), pe = min(ce, h);
        if (ps >= pe) continue;
        const T* A = srck + l;
        const T* B = srck + mm;
        const int32_t la = mm - l, lb = h - mm;
        int32_t i = corank_serial<K>(A, B, la, lb, ps - l);
        int32_t j = (ps - l) - i;
        for (int32_t p = ps; p < pe; ++p) {
          const bool takeA = (j >= lb) || (i < la && key_le<K>(A[i], B[j]));
          if (takeA) {
            dstk[p] = A[i];
            if (V) dstv[p] = srcv[l + i];
            ++i;
          } else {
            dstk[p] = B[j];
            if (V) dstv[p] = srcv[mm + j];
            ++j;
          }
        }
      }
    }
    __syncthreads();
  }

  // the subtree root (relative depth 0) sits in buffer 0; it belongs in global buffer droot mod 2
  T* ok = (T*)buf.k[droot & 1];
  uint32_t* ov = buf.v[droot & 1];
  for (int32_t p = tid; p < m; p += kSubThreads) {
    ok[lo + p] = sk[0][p];
    if (V) ov[lo + p] = sv[0][p];
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
// Large leaves: odd depth -> scratch buffer (reversed if descending); even depth and
// descending -> reversed in place.  One CTA per kMergeTile outputs (or pairs).
// ---------------------------------------------------------------------------------------
template <class K, bool V>
__global__ void __launch_bounds__(256)
leaf_place_kernel(Bufs buf, const int32_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
                  const uint8_t* __restrict__ ldepth, const int32_t* __restrict__ items,
                  const uint32_t* __restrict__ tile_off, uint32_t nitems) {
  typedef typename K::T T;
  __shared__ int32_t s_slot;
  if (threadIdx.x == 0) s_slot = slot_of_tile(tile_off, nitems, blockIdx.x);
  __syncthreads();
  const int32_t slot = s_slot;
  const int32_t i = items[slot];
  const int32_t k = (int32_t)(blockIdx.x - tile_off[slot]);
  const int32_t s = S[i], e = S[i + 1];
  const bool desc = run_desc[i] != 0;
  T* k0 = (T*)buf.k[0];
  T* k1 = (T*)buf.k[1];
  if (ldepth[i] & 1) {
    const int32_t q1 = min(e, s + (k + 1) * kMergeTile);
    for (int32_t q = s + k * kMergeTile + threadIdx.x; q < q1; q += blockDim.x) {
      const int32_t src = desc ? s + e - 1 - q : q;
      k1[q] = k0[src];
      if (V) buf.v[1][q] = buf.v[0][src];
    }
  } else {
    const int32_t half = (e - s) / 2;
    const int32_t p1 = min(s + half, s + (k + 1) * kMergeTile);
    for (int32_t p = s + k * kMergeTile + threadIdx.x; p < p1; p += blockDim.x) {
      const int32_t q = s + e - 1 - p;
      const T a = k0[p], b = k0[q];
      k0[p] = b;
      k0[q] = a;
      if (V) {
        const uint32_t va = buf.v[0][p], vb = buf.v[0][q];
        buf.v[0][p] = vb;
        buf.v[0][q] = va;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Co-rank of every merge tile of one level: one warp per tile, 32 probes per round.
// Tiles of a node [lo, hi) start at lo and then at the multiples of kMergeTile inside it.
// ---------------------------------------------------------------------------------------
template <class K>
__global__ void __launch_bounds__(256)
corank_kernel(const typename K::T* __restrict__ src, const int32_t* __restrict__ S,
              const int32_t* __restrict__ nodeL, const int32_t* __restrict__ nodeR,
              const int32_t* __restrict__ items, const uint32_t* __restrict__ tile_off, uint32_t nitems,
              uint32_t ntiles, TileDesc* __restrict__ tiles) {
  const int lane = threadIdx.x & 31;
  const uint32_t t = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (t >= ntiles) return;
  int32_t slot = 0;
  if (lane == 0) slot = slot_of_tile(tile_off, nitems, t);
  slot = __shfl_sync(0xffffffffu, slot, 0);
  const int32_t j = items[slot];
  const int32_t k = (int32_t)(t - tile_off[slot]);
  const int32_t lo = S[nodeL[j]], mid = S[j], hi = S[nodeR[j]];
  const int32_t g0 = (k == 0) ? lo : (lo / kMergeTile + k) * kMergeTile;
  const int32_t diag = g0 - lo, la = mid - lo, lb = hi - mid;
  const typename K::T* A = src + lo;
  const typename K::T* B = src + mid;
  int32_t a = max(0, diag - lb), b = min(diag, la);  // answer in [a, b]
  while (a < b) {
    const int32_t span = b - a;
    const int32_t x = a + (int32_t)(((int64_t)span * lane) >> 5);  // probes in [a, b)
    const bool gt = !key_le<K>(A[x], B[diag - 1 - x]);           // A[x] not among the first diag
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
  if (lane == 0) {
    TileDesc d;
    d.lo = lo;
    d.mid = mid;
    d.hi = hi;
    d.g0 = g0;
    d.i0 = a;
    d.pad[0] = d.pad[1] = d.pad[2] = 0;
    tiles[t] = d;
  }
}

// ---------------------------------------------------------------------------------------
// One merge tile: outputs [g0, g1) of the merge described by tiles[t].
// ---------------------------------------------------------------------------------------
template <class K, bool V>
struct MergeLayout {
  typedef typename K::T T;
  static constexpr int KU = 16 / (int)sizeof(T);  // elements per 16-byte unit
  static constexpr int KCAP = kMergeTile + 4 * KU;
  static constexpr int VCAP = kMergeTile + 16;
  static constexpr size_t kKeyOff = 128;
  static constexpr size_t kValOff = kKeyOff + (size_t)KCAP * sizeof(T);
  static constexpr size_t kBytes = kValOff + (V ? (size_t)VCAP * 4 : 0);
};

template <class K, bool V>
__global__ void __launch_bounds__(kMergeThreads)
merge_tile_kernel(const typename K::T* __restrict__ srck, const uint32_t* __restrict__ srcv,
                  typename K::T* __restrict__ dstk, uint32_t* __restrict__ dstv,
                  const TileDesc* __restrict__ tiles, PlanHeader* __restrict__ hdr,
                  uint32_t* lib_status) {
  typedef typename K::T T;
  typedef MergeLayout<K, V> Lay;
  constexpr int KU = Lay::KU;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* bar = (uint64_t*)smem;
  T* sk = (T*)(smem + Lay::kKeyOff);
  uint32_t* sv = (uint32_t*)(smem + Lay::kValOff);
  const int tid = threadIdx.x;

  const TileDesc td = tiles[blockIdx.x];
  const int32_t lo = td.lo, mid = td.mid, hi = td.hi, g0 = td.g0, i0 = td.i0;
  const int32_t g1 = min(hi, (g0 / kMergeTile + 1) * kMergeTile);
  const int32_t i1 = (g1 == hi) ? (mid - lo) : tiles[blockIdx.x + 1].i0;
  const int32_t a0 = lo + i0, a1 = lo + i1;
  const int32_t b0 = mid + (g0 - lo - i0), b1 = mid + (g1 - lo - i1);
  // 16-byte aligned enclosing chunks (the buffers are 16-byte aligned)
  const int32_t ka0 = a0 & ~(KU - 1), ka1 = (a1 > a0) ? ((a1 + KU - 1) & ~(KU - 1)) : ka0;
  const int32_t kb0 = b0 & ~(KU - 1), kb1 = (b1 > b0) ? ((b1 + KU - 1) & ~(KU - 1)) : kb0;
  const int32_t KA = ka1 - ka0;
  const int32_t va0 = a0 & ~3, va1 = (a1 > a0) ? ((a1 + 3) & ~3) : va0;
  const int32_t vb0 = b0 & ~3, vb1 = (b1 > b0) ? ((b1 + 3) & ~3) : vb0;
  const int32_t VA = va1 - va0;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t kbytes_a = (uint32_t)KA * sizeof(T), kbytes_b = (uint32_t)(kb1 - kb0) * sizeof(T);
    const uint32_t vbytes_a = V ? (uint32_t)VA * 4u : 0u, vbytes_b = V ? (uint32_t)(vb1 - vb0) * 4u : 0u;
    mbar_arrive_expect_tx(bar, kbytes_a + kbytes_b + vbytes_a + vbytes_b);
    if (kbytes_a) bulk_g2s(sk, srck + ka0, kbytes_a, bar);
    if (kbytes_b) bulk_g2s(sk + KA, srck + kb0, kbytes_b, bar);
    if (V) {
      if (vbytes_a) bulk_g2s(sv, srcv + va0, vbytes_a, bar);
      if (vbytes_b) bulk_g2s(sv + VA, srcv + vb0, vbytes_b, bar);
    }
  }
  {
    uint32_t spins = 0;
    while (!mbar_try_wait(bar, 0)) {
      if (++spins > kMbarTries) {
        post_status(&hdr->status, lib_status, kDevTimeout);
        // let the copies in flight land before the CTA exits (bounded again)
        uint32_t more = 0;
        while (!mbar_try_wait(bar, 0) && ++more < kMbarTries) {
        }
        return;
      }
    }
  }

  const T* A = sk + (a0 - ka0);
  const T* B = sk + KA + (b0 - kb0);
  const int32_t vA = a0 - va0, vB = VA + (b0 - vb0);
  const int32_t len = g1 - g0, la = i1 - i0, lb = len - la;
  const int32_t diag = tid * kMergeItems;
  if (diag >= len) return;
  int32_t i = corank_serial<K>(A, B, la, lb, diag);
  int32_t j = diag - i;
  T key[kMergeItems];
  int32_t src[kMergeItems];
  const int32_t cnt = min(kMergeItems, len - diag);
#pragma unroll
  for (int q = 0; q < kMergeItems; ++q) {
    if (q < cnt) {
      const bool takeA = (j >= lb) || (i < la && key_le<K>(A[i], B[j]));
      key[q] = takeA ? A[i] : B[j];
      src[q] = takeA ? vA + i : vB + j;
      if (takeA) ++i; else ++j;
    }
  }
  const int32_t g = g0 + diag;
  if (cnt == kMergeItems && (g % KU) == 0) {
    uint4* o = (uint4*)(dstk + g);
#pragma unroll
    for (int q = 0; q < kMergeItems / KU; ++q) {
      uint4 w;
      T* wt = (T*)&w;
#pragma unroll
      for (int u = 0; u < KU; ++u) wt[u] = key[q * KU + u];
      o[q] = w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kMergeItems; ++q)
      if (q < cnt) dstk[g + q] = key[q];
  }
  if (V) {
    if (cnt == kMergeItems && (g % 4) == 0) {
      uint4* o = (uint4*)(dstv + g);
#pragma unroll
      for (int q = 0; q < kMergeItems / 4; ++q)
        o[q] = make_uint4(sv[src[4 * q]], sv[src[4 * q + 1]], sv[src[4 * q + 2]], sv[src[4 * q + 3]]);
    } else {
#pragma unroll
      for (int q = 0; q < kMergeItems; ++q)
        if (q < cnt) dstv[g + q] = sv[src[q]];
    }
  }
}

}  // namespace ps
