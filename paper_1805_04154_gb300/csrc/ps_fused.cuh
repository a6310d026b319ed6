// Stage 4, fused passes: two levels of the powersort tree per HBM pass.
//
// Only nodes of even depth are written by HBM passes.  A large node N of even depth merges the
// up to four sorted ranges X1 X2 X3 X4 directly below it: its left child if that is a leaf or
// a subtree merged in shared memory, else the child's two children (the child, of odd depth,
// is never materialised); the same on the right.  The ranges are consecutive, so N's output is
// the stable merge of X1..X4 in which, on equal keys, a lower range goes first -- exactly what
// the two levels of binary merges (Alg. 2's Merge calls for the child and for N) produce.
//
// Work split.  Every kChunkSpan-th element of each range (positions kChunkSpan, 2 kChunkSpan,
// ...) is a chunk boundary; with the node's start and end they cut N's output into chunks, and
// a chunk takes at most kChunkSpan elements from each range (no range has a boundary strictly
// inside it).  chunk_table_kernel computes, for every boundary element, how many elements of
// each range precede it (its exact 4-way split) and its place among the node's boundaries, by
// binary searches over the boundary elements of the other ranges and then inside one span.
// fused_pass_kernel then groups consecutive chunks into tiles of at most kFusedTile outputs:
//  * warp 8 (producer) reads the boundaries, stages the tile's four portions into shared
//    memory with bulk (TMA) copies on the stage's "full" mbarrier;
//  * warps 0-7 (consumers) merge the X1|X2 and X3|X4 portions into a second shared buffer
//    (C1 | C2), release the stage to the producer, then merge C1 and C2 into registers and
//    write them with 128-bit stores, each thread owning kMergeItems outputs aligned to 16-byte
//    boundaries of the destination.
// All waits are bounded; a timeout posts kDevTimeout and the CTA drains its copies and exits.
#pragma once

#include "ps_level.cuh"
#include "ps_merge.cuh"

namespace ps {

// ---------------------------------------------------------------------------------------
// Ranges of a fused merge: b[0] = lo, b[1] = split of the left child (or lo), b[2] = mid,
// b[3] = split of the right child (or mid), b[4] = hi.  A child is split when it is an
// internal node larger than the shared-memory subtree limit (it then has odd depth).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ bool fused_ranges(const int4 nd, const int32_t* __restrict__ nodeL,
                                             const int32_t* __restrict__ nodeR, const int32_t* __restrict__ lsplit,
                                             const int32_t* __restrict__ rsplit, int32_t sub_lim, int32_t b[5]) {
  const int32_t x = nd.w;
  b[0] = nd.x;
  b[2] = nd.y;
  b[4] = nd.z;
  b[1] = nd.x;
  b[3] = nd.y;
  bool ok = true;
  if (x - nodeL[x] >= 2 && nd.y - nd.x > sub_lim) {
    b[1] = lsplit[x];
    ok = ok && b[1] > nd.x && b[1] < nd.y;
  }
  if (nodeR[x] - x >= 2 && nd.z - nd.y > sub_lim) {
    b[3] = rsplit[x];
    ok = ok && b[3] > nd.y && b[3] < nd.z;
  }
  if (!ok) {  // never for a consistent plan; fall back to an unsplit (still ordered) layout
    b[1] = nd.x;
    b[3] = nd.y;
  }
  return ok;
}

// y (from range m) precedes x (from range k) in the merged order: on equal keys the lower
// range goes first.
template <class K>
__device__ __forceinline__ bool precedes(typename K::T y, typename K::T x, bool m_before_k) {
  return m_before_k ? K::le(y, x) : !K::le(x, y);
}

// Number of elements of X[0, len) that precede x, and (in samples) how many of X's chunk
// boundaries (positions kChunkSpan * q, q >= 1) precede x.
template <class K>
__device__ __forceinline__ int32_t rank_in_range(const typename K::T* __restrict__ X, int32_t len,
                                                 typename K::T x, bool m_before_k, int32_t& samples) {
  const int32_t ns = len > 0 ? (len - 1) / kChunkSpan : 0;
  int32_t a = 0, b = ns;  // largest q in [0, ns] whose boundary precedes x (q = 0: none)
  while (a < b) {
    const int32_t mid = (a + b + 1) >> 1;
    if (precedes<K>(X[(size_t)mid * kChunkSpan], x, m_before_k)) a = mid;
    else b = mid - 1;
  }
  samples = a;
  int32_t lo = a >= 1 ? a * kChunkSpan + 1 : 0;
  int32_t hi = a < ns ? (a + 1) * kChunkSpan : len;  // first non-preceding index is <= hi
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (precedes<K>(X[mid], x, m_before_k)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Four threads per boundary slot of the pass (thread m of the group ranks the boundary element
// in range m).  Item it owns slots [slot_off[it], slot_off[it+1]): slot 0 is the node's start
// (0,0,0,0), slots 1..ns the chunk boundaries in merged order, the rest the node's end
// (|X1|, |X2|, |X3|, |X4|).
template <class K>
__global__ void __launch_bounds__(256)
chunk_table_kernel(const typename K::T* __restrict__ src, const int4* __restrict__ items,
                   const uint32_t* __restrict__ slot_off, uint32_t nitems, uint32_t nslots,
                   const int32_t* __restrict__ nodeL, const int32_t* __restrict__ nodeR,
                   const int32_t* __restrict__ lsplit, const int32_t* __restrict__ rsplit, int32_t sub_lim,
                   int4* __restrict__ tab, int4* __restrict__ item_ext, PlanHeader* __restrict__ hdr,
                   uint32_t* lib_status) {
  typedef typename K::T T;
  const int m = threadIdx.x & 3;
  const int g0 = threadIdx.x & 28;  // first lane of this thread's group of four
  const unsigned gmask = 0xFu << g0;
  const uint32_t stride = (gridDim.x * blockDim.x) >> 2;
  for (uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 2; j < nslots; j += stride) {
    const int32_t it = slot_of_tile(slot_off, nitems, j);
    const uint32_t base = slot_off[it];
    const int32_t local = (int32_t)(j - base);
    const int4 nd = items[it];
    int32_t b[5];
    const bool consistent = fused_ranges(nd, nodeL, nodeR, lsplit, rsplit, sub_lim, b);
    if (!consistent && m == 0) post_status(&hdr->status, lib_status, kDevInternal);
    int32_t len[4], ns[4], total = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      len[r] = b[r + 1] - b[r];
      ns[r] = len[r] > 0 ? (len[r] - 1) / kChunkSpan : 0;
      total += ns[r];
    }
    if (local == 0) {
      if (m == 0) {
        tab[base] = make_int4(0, 0, 0, 0);
        item_ext[it] = make_int4(b[1], b[3], total, 0);
      }
    } else if (local > total) {
      if (m == 0) tab[base + local] = make_int4(len[0], len[1], len[2], len[3]);
    } else {
      // range k of this boundary and its position there (selects keep the arrays in registers)
      int32_t q = local - 1, k = 0, bk = b[0];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const bool past = (k == r) && q >= ns[r];
        q -= past ? ns[r] : 0;
        k += past ? 1 : 0;
        bk = past ? b[r + 1] : bk;
      }
      const int32_t p = (q + 1) * kChunkSpan;
      const T x = src[bk + p];
      const int32_t bm = m == 0 ? b[0] : m == 1 ? b[1] : m == 2 ? b[2] : b[3];
      const int32_t lm = m == 0 ? len[0] : m == 1 ? len[1] : m == 2 ? len[2] : len[3];
      int32_t cm, before;
      if (m == k) {
        cm = p;
        before = p / kChunkSpan - 1;
      } else {
        cm = rank_in_range<K>(src + bm, lm, x, m < k, before);
      }
      before += __shfl_xor_sync(gmask, before, 1);
      before += __shfl_xor_sync(gmask, before, 2);
      const int32_t c0 = __shfl_sync(gmask, cm, g0), c1 = __shfl_sync(gmask, cm, g0 + 1);
      const int32_t c2 = __shfl_sync(gmask, cm, g0 + 2), c3 = __shfl_sync(gmask, cm, g0 + 3);
      if (m == 0) tab[base + 1 + before] = make_int4(c0, c1, c2, c3);
    }
  }
}

struct FusedDesc {
  int32_t g0, g1;     // absolute output positions [g0, g1)
  int32_t n[4];       // portion lengths
  int32_t koff[4];    // shared-memory element offset of each portion's first key
  int32_t voff[4];    // ... and payload
  int32_t pad[2];
};

template <class K, bool V, int NS>
struct FusedLayout {
  typedef typename K::T T;
  static constexpr int KU = 16 / (int)sizeof(T);
  static constexpr int KCAP = kFusedTile + 8 * KU;  // four portions, each widened to 16-byte blocks
  static constexpr int VCAP = kFusedTile + 32;
  static constexpr size_t kKeyBytes = ((size_t)KCAP * sizeof(T) + 127) & ~(size_t)127;
  static constexpr size_t kValBytes = V ? (((size_t)VCAP * 4 + 127) & ~(size_t)127) : 0;
  static constexpr size_t kStageBytes = kKeyBytes + kValBytes;
  // merged halves C1 | C2 of the current tile (phase 1 output, phase 2 input)
  static constexpr size_t kTKeyBytes = ((size_t)kFusedTile * sizeof(T) + 127) & ~(size_t)127;
  static constexpr size_t kTValBytes = V ? (((size_t)kFusedTile * 4 + 127) & ~(size_t)127) : 0;
  static constexpr size_t kBarOff = 0;
  static constexpr size_t kDescOff = (2 * NS * 8 + 63) & ~(size_t)63;
  static constexpr size_t kFlagOff = kDescOff + NS * sizeof(FusedDesc);
  static constexpr size_t kTOff = (kFlagOff + 16 + 127) & ~(size_t)127;
  static constexpr size_t kStageOff = kTOff + kTKeyBytes + kTValBytes;
  static constexpr size_t kBytes = kStageOff + NS * kStageBytes;
};

// Stable merge of A[0, la) and B[0, lb) in shared memory: outputs [diag, diag + cnt) into
// registers (left wins ties).
template <class K, bool V, int N>
__device__ __forceinline__ void smem_merge_regs(const typename K::T* A, const typename K::T* B, const uint32_t* Av,
                                                const uint32_t* Bv, int32_t la, int32_t lb, int32_t diag, int32_t cnt,
                                                typename K::T (&key)[N], uint32_t (&val)[N]) {
  typedef typename K::T T;
  int32_t i = corank_serial<K>(A, B, la, lb, diag);
  int32_t j = diag - i;
  T a = A[min(i, max(la - 1, 0))], b = B[min(j, max(lb - 1, 0))];
#pragma unroll
  for (int q = 0; q < N; ++q) {
    if (q < cnt) {
      const bool takeA = (j >= lb) || (i < la && key_le<K>(a, b));
      key[q] = takeA ? a : b;
      if (V) val[q] = takeA ? Av[i] : Bv[j];
      if (takeA) {
        if (++i < la) a = A[i];
      } else {
        if (++j < lb) b = B[j];
      }
    }
  }
}

// Stable merge of A[0, la) and B[0, lb) in shared memory: outputs [diag, diag + cnt) written
// straight to O / Ov (shared memory).
template <class K, bool V, int N>
__device__ __forceinline__ void smem_merge_to(const typename K::T* A, const typename K::T* B, const uint32_t* Av,
                                              const uint32_t* Bv, int32_t la, int32_t lb, int32_t diag, int32_t cnt,
                                              typename K::T* O, uint32_t* Ov) {
  typedef typename K::T T;
  int32_t i = corank_serial<K>(A, B, la, lb, diag);
  int32_t j = diag - i;
  T a = A[min(i, max(la - 1, 0))], b = B[min(j, max(lb - 1, 0))];
#pragma unroll
  for (int q = 0; q < N; ++q) {
    if (q < cnt) {
      const bool takeA = (j >= lb) || (i < la && key_le<K>(a, b));
      O[diag + q] = takeA ? a : b;
      if (V) Ov[diag + q] = takeA ? Av[i] : Bv[j];
      if (takeA) {
        if (++i < la) a = A[i];
      } else {
        if (++j < lb) b = B[j];
      }
    }
  }
}

// Named barrier among the kMergeThreads consumer threads.
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kMergeThreads) : "memory");
}

template <class K, bool V, int NS>
__global__ void __launch_bounds__(kPassThreads, 3)
fused_pass_kernel(const typename K::T* __restrict__ srck, const uint32_t* __restrict__ srcv,
                  typename K::T* __restrict__ dstk, uint32_t* __restrict__ dstv, const int4* __restrict__ items,
                  const int4* __restrict__ item_ext, const uint32_t* __restrict__ slot_off, uint32_t nitems,
                  uint32_t nslots, const int4* __restrict__ tab, PlanHeader* __restrict__ hdr, uint32_t* lib_status) {
  typedef typename K::T T;
  typedef FusedLayout<K, V, NS> Lay;
  constexpr int KU = Lay::KU;
  constexpr int IPT = kMergeItems;
  static_assert(kMergeThreads * IPT >= kFusedTile + 2 * IPT, "phase-1 threads cover two ragged merges");
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = (uint64_t*)(smem + Lay::kBarOff);
  uint64_t* empty = full + NS;
  FusedDesc* sdesc = (FusedDesc*)(smem + Lay::kDescOff);
  volatile int32_t* abort_flag = (volatile int32_t*)(smem + Lay::kFlagOff);
  T* tk = (T*)(smem + Lay::kTOff);
  uint32_t* tv = (uint32_t*)(smem + Lay::kTOff + Lay::kTKeyBytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t j_begin = (uint32_t)(((uint64_t)blockIdx.x * nslots) / gridDim.x);
  const uint32_t j_end = (uint32_t)(((uint64_t)(blockIdx.x + 1) * nslots) / gridDim.x);
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kMergeThreads / 32);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kMergeThreads / 32) {
    // ------------------------------ producer ------------------------------
    uint32_t issued = 0;
    bool ok = true, corrupt = false;
    int32_t it = -1;
    uint32_t it_end = 0;  // first slot of the next item
    int32_t b[5] = {0, 0, 0, 0, 0};
    uint32_t j = j_begin;
    int4 e0 = make_int4(0, 0, 0, 0);
    bool have_e0 = false;
    while (j < j_end && ok) {
      if (it < 0 || j >= it_end) {  // enter the item owning slot j (items are consecutive)
        if (it >= 0 && it + 1 < (int32_t)nitems && j == it_end) {
          ++it;
        } else {
          if (lane == 0) it = slot_of_tile(slot_off, nitems, j);
          it = __shfl_sync(0xffffffffu, it, 0);
        }
        it_end = (it + 1 < (int32_t)nitems) ? slot_off[it + 1] : nslots;
        const int4 nd = items[it];
        const int4 ex = item_ext[it];
        b[0] = nd.x;
        b[1] = ex.x;
        b[2] = nd.y;
        b[3] = ex.y;
        b[4] = nd.z;
        have_e0 = false;
      }
      if (j + 1 >= it_end) {  // the item's last slot starts no chunk
        ++j;
        have_e0 = false;
        continue;
      }
      if (!have_e0) e0 = tab[j];
      // tile = chunks j .. j2-1: the longest run of whole chunks within kFusedTile outputs
      const int32_t gs = e0.x + e0.y + e0.z + e0.w;
      const uint32_t lim = min(it_end - 1, j_end);  // largest end slot allowed
      const uint32_t cand = j + 1 + lane;
      int4 e = make_int4(0, 0, 0, 0);
      bool fit = false;
      if (cand <= lim) {
        e = tab[cand];
        fit = (e.x + e.y + e.z + e.w) - gs <= kFusedTile;
      }
      const uint32_t fm = __ballot_sync(0xffffffffu, fit);
      if (!(fm & 1u)) {  // a single chunk never exceeds the tile; only a corrupt table does
        corrupt = true;
        ok = false;
        break;
      }
      const int src_lane = 31 - __clz(fm);  // fit is monotone in the end slot
      const uint32_t j2 = j + 1 + src_lane;
      int4 e1;
      e1.x = __shfl_sync(0xffffffffu, e.x, src_lane);
      e1.y = __shfl_sync(0xffffffffu, e.y, src_lane);
      e1.z = __shfl_sync(0xffffffffu, e.z, src_lane);
      e1.w = __shfl_sync(0xffffffffu, e.w, src_lane);
      const int32_t ge = e1.x + e1.y + e1.z + e1.w;
      if (ge != gs) {  // (padding chunks between end boundaries are empty)
        const int s = (int)(issued % NS);
        const uint32_t use = issued / NS;
        if (!__all_sync(0xffffffffu, bounded_wait(&empty[s], (use & 1u) ^ 1u))) {
          ok = false;
          break;
        }
        if (lane == 0) {
          const int32_t c0[4] = {e0.x, e0.y, e0.z, e0.w}, c1[4] = {e1.x, e1.y, e1.z, e1.w};
          FusedDesc d;
          d.g0 = b[0] + gs;
          d.g1 = b[0] + ge;
          uint8_t* stage = smem + Lay::kStageOff + (size_t)s * Lay::kStageBytes;
          T* sk = (T*)stage;
          uint32_t* sv = (uint32_t*)(stage + Lay::kKeyBytes);
          int32_t kcur = 0, vcur = 0;
          uint32_t kbytes[4], vbytes[4];
          int32_t kfrom[4], vfrom[4], kat[4], vat[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int32_t p0 = b[k] + c0[k], p1 = b[k] + c1[k];
            d.n[k] = p1 - p0;
            int32_t ka, kb, va, vb;
            chunk16(srck, p0, p1, ka, kb);
            kfrom[k] = ka;
            kat[k] = kcur;
            kbytes[k] = (uint32_t)(kb - ka) * sizeof(T);
            d.koff[k] = kcur + (p0 - ka);
            kcur += kb - ka;
            if (V) {
              chunk16(srcv, p0, p1, va, vb);
              vfrom[k] = va;
              vat[k] = vcur;
              vbytes[k] = (uint32_t)(vb - va) * 4u;
              d.voff[k] = vcur + (p0 - va);
              vcur += vb - va;
            } else {
              vfrom[k] = 0;
              vat[k] = 0;
              vbytes[k] = 0;
              d.voff[k] = 0;
            }
          }
          sdesc[s] = d;
          uint32_t tx = 0;
#pragma unroll
          for (int k = 0; k < 4; ++k) tx += kbytes[k] + vbytes[k];
          mbar_arrive_expect_tx(&full[s], tx);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (kbytes[k]) bulk_g2s(sk + kat[k], srck + kfrom[k], kbytes[k], &full[s]);
            if (V && vbytes[k]) bulk_g2s(sv + vat[k], srcv + vfrom[k], vbytes[k], &full[s]);
          }
        }
        __syncwarp();
        ++issued;
      }
      j = j2;
      e0 = e1;  // the next tile starts where this one ended
      have_e0 = true;
    }
    // end of work: a marker descriptor (g0 > g1) in the next stage; the consumers then have
    // waited for every issued stage, so all copies have landed before the CTA exits
    if (ok) {
      const int s = (int)(issued % NS);
      const uint32_t use = issued / NS;
      ok = __all_sync(0xffffffffu, bounded_wait(&empty[s], (use & 1u) ^ 1u));
      if (ok && lane == 0) {
        FusedDesc d;
        d.g0 = 1;
        d.g1 = 0;
        sdesc[s] = d;
        mbar_arrive(&full[s]);
      }
      __syncwarp();
    }
    if (!ok) {
      if (lane == 0) post_status(&hdr->status, lib_status, corrupt ? kDevInternal : kDevTimeout);
      *abort_flag = 1;
      // drain: every copy issued into a stage must land before the CTA exits
      if (lane == 0) {
        for (uint32_t q = (issued > NS ? issued - NS : 0); q < issued; ++q) bounded_wait(&full[q % NS], (q / NS) & 1u);
      }
    }
  } else {
    // ------------------------------ consumers ------------------------------
    const int tid = threadIdx.x;
    for (uint32_t itn = 0;; ++itn) {
      const int s = (int)(itn % NS);
      const uint32_t use = itn / NS;
      bool ready = false;
      for (uint32_t tries = 0; tries < kMbarTries; ++tries) {
        if (mbar_try_wait(&full[s], use & 1u)) {
          ready = true;
          break;
        }
        if (*abort_flag) break;
      }
      // (also the barrier after which the previous tile's phase 2 no longer reads C1 | C2)
      if (!consumer_all(ready)) {
        if (tid == 0 && !*abort_flag) post_status(&hdr->status, lib_status, kDevTimeout);
        break;
      }
      const FusedDesc& d = sdesc[s];  // read from shared memory where used (fewer live registers)
      if (d.g0 > d.g1) break;         // producer's end marker
      const int32_t L1 = d.n[0] + d.n[1], L2 = d.n[2] + d.n[3];
      {
        // phase 1: X1|X2 -> C1 = T[0, L1) and X3|X4 -> C2 = T[L1, L1 + L2); then the stage is free
        const uint8_t* stage = smem + Lay::kStageOff + (size_t)s * Lay::kStageBytes;
        const T* sk = (const T*)stage;
        const uint32_t* sv = (const uint32_t*)(stage + Lay::kKeyBytes);
        const int32_t T1 = (L1 + IPT - 1) / IPT;
        const int32_t T2 = (L2 + IPT - 1) / IPT;
        if (tid < T1) {
          const int32_t diag = tid * IPT;
          smem_merge_to<K, V, IPT>(sk + d.koff[0], sk + d.koff[1], sv + d.voff[0], sv + d.voff[1], d.n[0], d.n[1],
                                   diag, min(IPT, L1 - diag), tk, tv);
        } else if (tid - T1 < T2) {
          const int32_t diag = (tid - T1) * IPT;
          smem_merge_to<K, V, IPT>(sk + d.koff[2], sk + d.koff[3], sv + d.voff[2], sv + d.voff[3], d.n[2], d.n[3],
                                   diag, min(IPT, L2 - diag), tk + L1, tv + L1);
        }
      }
      const int32_t g0 = d.g0, g1 = d.g1;
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(&empty[s]);  // the producer may refill this stage now
      consumer_sync();
      // phase 2: C1 | C2 -> outputs; thread t owns [A0 + t*IPT, A0 + t*IPT + IPT) within [g0, g1)
      const int32_t A0 = g0 - (int32_t)(((uintptr_t)(dstk + g0) & 15u) / sizeof(T));
      const int32_t p0 = max(g0, A0 + tid * IPT), p1 = min(g1, A0 + tid * IPT + IPT);
      if (p0 < p1) {
        const int32_t cnt = p1 - p0;
        T key[IPT];
        uint32_t val[IPT];
        smem_merge_regs<K, V, IPT>(tk, tk + L1, tv, tv + L1, L1, L2, p0 - g0, cnt, key, val);
        if (cnt == IPT && ((uintptr_t)(dstk + p0) & 15u) == 0) {
          uint4* o = (uint4*)(dstk + p0);
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
            if (q < cnt) dstk[p0 + q] = key[q];
        }
        if (V) {
          if (cnt == IPT && ((uintptr_t)(dstv + p0) & 15u) == 0) {
            uint4* o = (uint4*)(dstv + p0);
#pragma unroll
            for (int q = 0; q < IPT / 4; ++q)
              o[q] = make_uint4(val[4 * q], val[4 * q + 1], val[4 * q + 2], val[4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < IPT; ++q)
              if (q < cnt) dstv[p0 + q] = val[q];
          }
        }
      }
    }
  }
}

}  // namespace ps
