// Stages 2-3 and planning: node powers, the merge tree as nearest smaller values of the powers,
// node/leaf depths, merge cost, and the work lists of stage 4.  Key-independent; O(r) work.
#include "ps_debug.cuh"
#include "ps_internal.h"
#include "ps_level.cuh"

namespace ps {

// ---------------------------------------------------------------------------------------
// Stage 2: node power of every boundary (Definition "Node Power"; NodePower of Alg. 2).
// Boundary j (1 <= j <= r-1) separates run j-1 = [S[j-1], S[j]) and run j = [S[j], S[j+1]).
// With positions relative to the segment start and ns the segment length, the normalised
// midpoints are a = (S[j-1]+S[j]) / (2 ns) and b = (S[j]+S[j+1]) / (2 ns); the power is the
// index of their first differing fractional bit.  The first 31 fractional bits decide it for
// every ns < 2^32: b - a = (L_{j-1} + L_j) / (2 ns), and a greedy run is at least two elements
// long unless it is its segment's last, so either L_{j-1} + L_j >= 4 (then b - a >= 2^-31) or the
// boundary is the segment's last one with lengths (>= 2, 1), where (a, b] = (1 - 5/(2 ns),
// 1 - 1/ns] contains 1 - 2^-31 whenever ns > 2^31.  So x = floor(a 2^31), y = floor(b 2^31)
// (< 2^31) differ and the power is the number of leading zeros of x ^ y in 32 bits (<= 31).
// Boundaries between segments and the sentinels j = 0, j = r get power 0 (smaller than every
// real power).
// ---------------------------------------------------------------------------------------
// floor(a / d) for a < 2^64 and 2 <= d < 2^33, given m = floor((2^64 - 1) / d): division by an
// invariant integer through a multiply-high (Granlund and Montgomery, PLDI 1994).  a m / 2^64
// lies in (a/d - 2, a/d], so the estimate is q, q - 1 or q - 2, fixed by remainder tests (the
// remainder below 3d < 2^35 is exact in 64-bit wrapping arithmetic).
__device__ __forceinline__ uint64_t div_invariant(uint64_t a, uint64_t d, uint64_t m) {
  uint64_t q = __umul64hi(a, m);
  if (a - q * d >= d) ++q;
  if (a - q * d >= d) ++q;
  return q;
}

// A thread computes the powers of four consecutive boundaries j0 .. j0+3 (one 32-bit word of P):
// with q_k = floor((S[k] + S[k+1] - 2 base) 2^31 / (2 ns)) the scaled midpoint of run k in its
// segment, boundary j has x = q_{j-1} and y = q_j, so five divisions serve the four powers.
__global__ void __launch_bounds__(256, 6) node_power_kernel(const pos_t* __restrict__ S, const int32_t* __restrict__ run_seg,
                                  const int64_t* __restrict__ offsets, int64_t n, uint8_t* __restrict__ P,
                                  PlanHeader* __restrict__ hdr) {
  const int32_t r = hdr->runs;
  const int32_t words = r / 4 + 1;  // P[0 .. r] as whole words (the allocation covers them)
  int32_t cached_seg = -1;
  int64_t base = 0, ns = n;
  uint64_t two_n = 2 * (uint64_t)n, m = ~0ull / (2 * (uint64_t)max(n, (int64_t)1));
  bool bad = false;
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < words; g += gridDim.x * blockDim.x) {
    const int32_t j0 = 4 * g;
    // S[j0 - 1 .. j0 + 4]: entries past r are never used
    pos_t s[6];
    s[0] = j0 >= 1 ? S[j0 - 1] : 0u;
    if (j0 + 4 <= r) {
      const uint4 w = *(const uint4*)(S + j0);  // S is 16-byte aligned and j0 a multiple of 4
      s[1] = w.x;
      s[2] = w.y;
      s[3] = w.z;
      s[4] = w.w;
      s[5] = S[j0 + 4];
    } else {
#pragma unroll
      for (int e = 1; e < 6; ++e) s[e] = (j0 - 1 + e <= r) ? S[j0 - 1 + e] : 0u;
    }
    uint32_t q[5];
    int32_t sg[5];
#pragma unroll
    for (int e = 0; e < 5; ++e) {  // run k = j0 - 1 + e, for 0 <= k < r
      const int32_t k = j0 - 1 + e;
      q[e] = 0;
      sg[e] = -1;
      if (k >= 0 && k < r) {
        if (run_seg != nullptr) {
          sg[e] = run_seg[k];
          if (sg[e] != cached_seg) {
            cached_seg = sg[e];
            base = offsets[sg[e]];
            ns = offsets[sg[e] + 1] - base;
            two_n = 2 * (uint64_t)(ns > 0 ? ns : 1);
            m = ~0ull / two_n;
          }
          if (ns <= 0) sg[e] = -2 - k;  // only with invalid offsets, which the host rejects
        } else {
          sg[e] = 0;
        }
        const uint64_t mid2 = (uint64_t)((int64_t)s[e] + s[e + 1] - 2 * base);
        q[e] = (uint32_t)div_invariant(mid2 << 31, two_n, m);
      }
    }
    uint32_t w = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int32_t j = j0 + e;
      if (j >= 1 && j < r && sg[e] >= 0 && sg[e] == sg[e + 1]) {
        bad |= q[e] == q[e + 1];  // excluded by the run-length argument above
        w |= (uint32_t)__clz(q[e] ^ q[e + 1]) << (8 * e);
      }
    }
    ((uint32_t*)P)[g] = w;
  }
  if (bad) post_status(&hdr->status, nullptr, kDevInternal);
}

// ---------------------------------------------------------------------------------------
// Stage 3: the merge tree (Corollary "Cartesian tree": the min-Cartesian tree of the powers).
// For node j: Lj = nearest i < j with P_i < P_j, Rj = nearest k > j with P_k < P_j (the
// power-0 sentinels and segment boundaries always qualify); node j merges [S[Lj], S[j]) with
// [S[j], S[Rj]).  Its ancestors are exactly the entries of the nearest-smaller-value stacks on
// either side, so depth(j) = (left stack entries of power >= 1) + (right ones).
//
// Left to right, the stack of nearest smaller values holds at most one entry per power value
// (powers increase from its bottom), and an entry of power v is always the last boundary of
// power v seen so far.  So a stack is a 32-bit occupancy mask plus the table last[v] = last
// index of power v, and from last[] alone the stack is recovered: v is on it iff last[v] is
// larger than last[w] for every w < v.  Thread-chunk and tile summaries are therefore last[]
// vectors, combined by element-wise max.
//
// Per direction three kernels: per-tile last[] summaries, an exclusive max-scan over tiles,
// and the apply pass in which each of kTreeThreads threads rebuilds the stack in front of its
// kTreeChunk consecutive indices and walks them.  Virtual index u maps to boundary j = u
// (forward) or j = r - u (backward).
// ---------------------------------------------------------------------------------------
template <bool kBackward>
__device__ __forceinline__ int32_t virt_to_j(int32_t u, int32_t r) {
  return kBackward ? r - u : u;
}

constexpr uint32_t kNoPower = 0xFFu;  // staged power of a virtual index past r

// Bytes P[b..b+3] as one little-endian word (bytes outside [0, r] read as kNoPower).  Reads
// only the aligned words overlapping [0, r], which the P allocation covers whole.
__device__ __forceinline__ uint32_t load_power_window(const uint8_t* __restrict__ P, int32_t r, int32_t b) {
  const uint32_t* __restrict__ Pw = (const uint32_t*)P;
  const int32_t wa = b >> 2;  // floor(b / 4), also for negative b
  const int32_t words = r / 4 + 1;  // words holding bytes 0..r
  const uint32_t lo = (wa >= 0 && 4 * wa <= r && PS_IN_RANGE(wa, words)) ? Pw[wa] : 0u;
  const uint32_t hi =
      ((b & 3) != 0 && wa + 1 >= 0 && 4 * (wa + 1) <= r && PS_IN_RANGE(wa + 1, words)) ? Pw[wa + 1] : 0u;
  uint32_t w = __funnelshift_r(lo, hi, (uint32_t)(b & 3) * 8u);
  if (b < 0 || b + 3 > r) {
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (b + e < 0 || b + e > r) w |= kNoPower << (8 * e);
  }
  return w;
}

// Stage the powers of virtual indices [u0, u0 + kTreeTile) into sp (word k of the tile holds
// virtual indices 4k..4k+3, stored at word k + k/8 so that a thread's chunk is 8 words and the
// threads of a warp read distinct banks).
template <bool kBackward>
__device__ __forceinline__ void stage_tile_powers(const uint8_t* __restrict__ P, int32_t r, int32_t u0,
                                                  uint32_t* __restrict__ sp) {
  for (int k = threadIdx.x; k < kTreeTile / 4; k += kTreeThreads) {
    uint32_t w;
    if (!kBackward) {
      w = load_power_window(P, r, u0 + 4 * k);
    } else {
      // virtual u0+4k+e is boundary r-u0-4k-e: the window starting 3 below, byte-reversed
      w = __byte_perm(load_power_window(P, r, r - u0 - 4 * k - 3), 0u, 0x0123);
    }
    sp[k + (k >> 3)] = w;
  }
}

// Thread chunk pass: s_last[v][t] = last virtual index of power v in the thread's chunk, minus
// base (or -1).  The summary stores virtual indices (base 0, 32-bit); the apply pass stores them
// relative to its tile (base u0, 16-bit: a tile holds kTreeTile = 8192 indices).
template <class L>
__device__ __forceinline__ void chunk_last(const uint32_t* __restrict__ sp, int32_t u0, int32_t base,
                                           L (*s_last)[kTreeThreads]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int v = 0; v < 32; ++v) s_last[v][t] = (L)-1;
  const int32_t ub = u0 + t * kTreeChunk;
#pragma unroll
  for (int k = 0; k < kTreeChunk / 4; ++k) {
    const uint32_t w = sp[t * 9 + k];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t p = (w >> (8 * e)) & 0xFFu;
      if (p != kNoPower) s_last[p & 31][t] = (L)(ub + 4 * k + e - base);
    }
  }
}

template <bool kBackward>
__global__ void __launch_bounds__(kTreeThreads)
tree_summary_kernel(const uint8_t* __restrict__ P, const PlanHeader* __restrict__ hdr, int32_t* __restrict__ summary,
                    int32_t stride) {
  extern __shared__ __align__(16) uint8_t tsm[];
  int32_t(*s_last)[kTreeThreads] = (int32_t(*)[kTreeThreads])tsm;
  uint32_t* sp = (uint32_t*)(tsm + 32 * kTreeThreads * 4);
  const int32_t r = hdr->runs;
  const int32_t ntiles = r / kTreeTile + 1;  // virtual indices 0..r
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int32_t u0 = tile * kTreeTile;
    stage_tile_powers<kBackward>(P, r, u0, sp);
    __syncthreads();
    chunk_last(sp, u0, 0, s_last);
    __syncthreads();
    // warp w reduces power values 4w..4w+3 over the tile's threads
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int v = warp * 4 + q;
      int32_t m = -1;
#pragma unroll
      for (int x = 0; x < kTreeThreads / 32; ++x) m = max(m, s_last[v][x * 32 + lane]);
      m = __reduce_max_sync(0xffffffffu, m);
      if (lane == 0) summary[v * stride + tile] = m;
    }
    __syncthreads();
  }
}

// exclusive max-scan over tiles, one CTA per power value (grid: 32 CTAs of kScanThreads); the
// summaries are stored power-major, so a CTA reads its power's tiles consecutively: thread k of a
// chunk takes kScanPer consecutive tiles, the chunk is scanned through the warps' totals, and a
// running maximum carries from chunk to chunk
constexpr int kScanThreads = 256, kScanPer = 8;
__global__ void __launch_bounds__(kScanThreads)
tree_scan_kernel(const PlanHeader* __restrict__ hdr, const int32_t* __restrict__ summary, int32_t* __restrict__ prefix,
                 int32_t stride) {
  __shared__ int32_t s_warp[kScanThreads / 32];
  const int32_t r = hdr->runs;
  const int32_t ntiles = r / kTreeTile + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, v = blockIdx.x;
  const int32_t* __restrict__ in = summary + (size_t)v * stride;
  int32_t* __restrict__ out = prefix + (size_t)v * stride;
  int32_t run = -1;  // maximum over the chunks before this one
  for (int32_t base = 0; base < ntiles; base += kScanThreads * kScanPer) {
    const int32_t t0 = base + tid * kScanPer;
    int32_t x[kScanPer];
    int32_t mine = -1;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
      x[q] = t0 + q < ntiles ? in[t0 + q] : -1;
      mine = max(mine, x[q]);
    }
    int32_t inc = mine;  // inclusive over the warp's threads
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t o = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc = max(inc, o);
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    int32_t before = __shfl_up_sync(0xffffffffu, inc, 1);  // exclusive over the warp's threads
    if (lane == 0) before = -1;
    int32_t chunk = -1;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
      if (w < warp) before = max(before, s_warp[w]);
      chunk = max(chunk, s_warp[w]);
    }
    before = max(before, run);
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
      if (t0 + q < ntiles) out[t0 + q] = before;
      before = max(before, x[q]);
    }
    run = max(run, chunk);
    __syncthreads();  // s_warp is reused by the next chunk
  }
}

constexpr size_t kTreeSummarySmem = 32 * kTreeThreads * 4 + (kTreeTile / 4 + kTreeTile / 32) * 4;
// apply: 16-bit last-index table and nearest-smaller list (tile-relative), the staged powers, and
// the tile prefix of every power: 42 KB, 5 CTAs per SM
constexpr size_t kApplyLastBytes = 32 * kTreeThreads * 2;
constexpr size_t kApplyStageBytes = (kTreeTile / 4 + kTreeTile / 32) * 4;
constexpr size_t kApplyNearBytes = (size_t)(kTreeTile + kTreeTile / 32) * 2;
constexpr size_t kTreeApplySmem = kApplyLastBytes + kApplyStageBytes + kApplyNearBytes + 32 * 4;
static_assert(kTreeTile <= 32768, "tile-relative indices fit 16 bits");

template <bool kBackward>
__global__ void __launch_bounds__(kTreeThreads, 5)
tree_apply_kernel(const uint8_t* __restrict__ P, PlanHeader* __restrict__ hdr, const int32_t* __restrict__ prefix,
                  int32_t stride, int32_t* __restrict__ near_out, uint8_t* __restrict__ depth_acc) {
  // Indices are kept relative to the tile start u0 in 16 bits: a last-index entry x >= 0 is the
  // virtual index u0 + x; -1 stands for the tile prefix of its power, s_carry[v] (itself -1 when
  // no index of that power precedes the tile).  A nearest-smaller entry that is a tile prefix is
  // stored as -(v + 2), v its power.
  extern __shared__ __align__(16) uint8_t tsm[];
  int16_t(*s_last)[kTreeThreads] = (int16_t(*)[kTreeThreads])tsm;
  uint32_t* sp = (uint32_t*)(tsm + kApplyLastBytes);
  int16_t* s_near = (int16_t*)(tsm + kApplyLastBytes + kApplyStageBytes);  // index i stored at i + i/32
  int32_t* s_carry = (int32_t*)(tsm + kApplyLastBytes + kApplyStageBytes + kApplyNearBytes);
  const int32_t r = hdr->runs;
  const int32_t ntiles = r / kTreeTile + 1;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  bool bad = false;
  for (int32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int32_t u0 = tile * kTreeTile;
    stage_tile_powers<kBackward>(P, r, u0, sp);
    if (t < 32) s_carry[t] = prefix[t * stride + tile];
    __syncthreads();
    chunk_last(sp, u0, u0, s_last);
    __syncthreads();
    // exclusive max-scan of the chunk vectors over the tile's threads (tile-relative; what no
    // thread before supplies is the tile prefix, -1)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int v = warp * 4 + q;
      int32_t carry = -1;
#pragma unroll
      for (int x = 0; x < kTreeThreads / 32; ++x) {
        int32_t inc = s_last[v][x * 32 + lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int32_t o = __shfl_up_sync(0xffffffffu, inc, d);
          if (lane >= d) inc = max(inc, o);
        }
        int32_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) exc = -1;
        s_last[v][x * 32 + lane] = (int16_t)max(carry, exc);
        carry = max(carry, __shfl_sync(0xffffffffu, inc, 31));
      }
    }
    __syncthreads();
    // the stack in front of this thread's chunk (virtual indices)
    uint32_t occ = 0;
    {
      int32_t M = -1;
#pragma unroll
      for (int v = 0; v < 32; ++v) {
        const int32_t x0 = s_last[v][t];
        const int32_t x = x0 >= 0 ? u0 + x0 : s_carry[v];
        if (x > M) {
          occ |= 1u << v;
          M = x;
        }
      }
    }
    // walk the chunk: nearest smaller on this side and the number of stack entries of power >= 1;
    // the count byte replaces the staged power (0xFF: no node here)
    const int32_t ub = t * kTreeChunk;  // tile-relative
#pragma unroll
    for (int k = 0; k < kTreeChunk / 4; ++k) {
      const uint32_t w = sp[t * 9 + k];
      uint32_t cw = 0;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const uint32_t p = (w >> (8 * e)) & 0xFFu;
        const int32_t u = ub + 4 * k + e;
        const int i = u;
        uint32_t cnt = 0xFFu;
        if (p == 0) {
          occ = 1u;
          s_last[0][t] = (int16_t)u;
        } else if (p != kNoPower) {
          const uint32_t pp = p & 31u;
          const uint32_t om = occ & ((1u << pp) - 1u);
          if (om == 0u) bad = true;  // the power-0 sentinel is always below
          const int top = om ? 31 - __clz(om) : 0;
          const int16_t x = s_last[top][t];
          s_near[i + (i >> 5)] = x >= 0 ? x : (int16_t)(-(top + 2));
          cnt = (uint32_t)__popc(om) - 1u;
          occ = om | (1u << pp);
          s_last[pp][t] = (int16_t)u;
        }
        cw |= cnt << (8 * e);
      }
      sp[t * 9 + k] = cw;
    }
    __syncthreads();
    // coalesced write-out, kGroup indices per thread at a time: the backward pass adds its counts
    // to the forward pass's, and loading the group's old counts before its stores keeps those
    // loads off a load-store chain (byte stores may alias any load)
    constexpr int kGroup = 8;
#pragma unroll 1
    for (int i0 = t; i0 < kTreeTile; i0 += kGroup * kTreeThreads) {
      uint32_t cnt[kGroup], old[kGroup];
      int32_t jj[kGroup];
#pragma unroll
      for (int q = 0; q < kGroup; ++q) {
        const int i = i0 + q * kTreeThreads;
        const int32_t u = u0 + i;
        cnt[q] = (u <= r) ? (sp[(i >> 2) + (i >> 5)] >> (8 * (i & 3))) & 0xFFu : 0xFFu;
        jj[q] = virt_to_j<kBackward>(u, r);
        if (cnt[q] != 0xFFu && !PS_IN_RANGE(jj[q], r + 1)) cnt[q] = 0xFFu;
        old[q] = (kBackward && cnt[q] != 0xFFu) ? depth_acc[jj[q]] : 0u;
      }
#pragma unroll
      for (int q = 0; q < kGroup; ++q) {
        const int i = i0 + q * kTreeThreads;
        if (cnt[q] != 0xFFu) {
          const int32_t x = s_near[i + (i >> 5)];
          const int32_t nv = x >= 0 ? u0 + x : s_carry[-x - 2];
          near_out[jj[q]] = virt_to_j<kBackward>(nv, r);
          depth_acc[jj[q]] = (uint8_t)(old[q] + cnt[q]);
        }
      }
    }
    __syncthreads();
  }
  if (bad) post_status(&hdr->status, nullptr, kDevInternal);
}

// ---------------------------------------------------------------------------------------
// Peeksort's merge tree (Alg. 1; the Peeksort theorem: Mehlhorn's Method 1 on the run lengths).
// A range of runs [a, b) with b - a >= 2, elements [l, r] (inclusive), is split at a run
// boundary near its middle m = l + floor((r - l) / 2): after the first run if m lies in it,
// before the last run if m lies in that, else at the nearer end of the run [i, j] containing m
// (its start i if m - i < j - m, else after its end).  The tree is built level by level: each
// range of the current level writes its node (the split boundary j: nodeL[j] = a,
// nodeR[j] = b, depth) and appends its two sub-ranges that hold more than one run.  For the
// plan, the boundary gets P[j] = depth + 1 (0 at sentinels and segment borders): a leaf's
// parent is then the larger-P of its two boundaries and a node's parent the larger-P of its
// range ends, the same rule as for node powers.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 8) peek_init_kernel(const pos_t* __restrict__ S, const int32_t* __restrict__ run_seg,
                                 const int64_t* __restrict__ offsets, uint8_t* __restrict__ P,
                                 int2* __restrict__ front0, uint32_t* __restrict__ count,
                                 const PlanHeader* __restrict__ hdr) {
  const int32_t r = hdr->runs;
  for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= r; j += gridDim.x * blockDim.x) {
    P[j] = 0;
    if (j == r) continue;
    // one root per segment: the range of the segment's runs
    if (run_seg == nullptr) {
      if (j == 0 && r >= 2) {
        front0[atomicAdd(&count[0], 1u)] = make_int2(0, r);
      }
    } else if (j == 0 || run_seg[j] != run_seg[j - 1]) {
      const int64_t end = offsets[run_seg[j] + 1];
      int32_t lo = j, hi = r;  // first run index at or past the segment's end
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (S[mid] < end) lo = mid + 1;
        else hi = mid;
      }
      if (lo - j >= 2) front0[atomicAdd(&count[0], 1u)] = make_int2(j, lo);
    }
  }
}

__global__ void __launch_bounds__(256, 8) peek_level_kernel(const pos_t* __restrict__ S, int level, const int2* __restrict__ cur,
                                  int2* __restrict__ next, uint32_t* __restrict__ count, int32_t cap,
                                  uint8_t* __restrict__ P, int32_t* __restrict__ nodeL, int32_t* __restrict__ nodeR,
                                  uint8_t* __restrict__ ndepth, PlanHeader* __restrict__ hdr) {
  const uint32_t m_cnt = count[level];
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < m_cnt; t += gridDim.x * blockDim.x) {
    if (level >= kMaxLevels) {  // deeper than the plan's per-depth lists
      post_status(&hdr->status, nullptr, kDevInternal);
      return;
    }
    const int2 rg = cur[t];
    const int32_t a = rg.x, b = rg.y;
    const int64_t l = S[a], rr = (int64_t)S[b] - 1;
    const int64_t e = (int64_t)S[a + 1] - 1, s = S[b - 1];
    const int64_t m = l + (rr - l) / 2;
    int32_t j;
    if (m <= e) {
      j = a + 1;
    } else if (m >= s) {
      j = b - 1;
    } else {
      int32_t lo = a + 1, hi = b - 1;  // run k containing m: largest k with S[k] <= m
      while (hi - lo > 0) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (S[mid] <= m) lo = mid;
        else hi = mid - 1;
      }
      const int64_t i = S[lo], jj = (int64_t)S[lo + 1] - 1;
      j = (m - i < jj - m) ? lo : lo + 1;
    }
    nodeL[j] = a;
    nodeR[j] = b;
    ndepth[j] = (uint8_t)level;
    P[j] = (uint8_t)(level + 1);
    if (j - a >= 2 || b - j >= 2) {
      const uint32_t add = (j - a >= 2 ? 1u : 0u) + (b - j >= 2 ? 1u : 0u);
      const uint32_t at = atomicAdd(&count[level + 1], add);
      if (at + add > (uint32_t)cap) {
        post_status(&hdr->status, nullptr, kDevInternal);
        continue;
      }
      uint32_t w = at;
      if (j - a >= 2) next[w++] = make_int2(a, j);
      if (b - j >= 2) next[w] = make_int2(j, b);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Planning.  Leaf i (run i) hangs below the adjacent boundary with the larger power (i or
// i+1); its depth is that node's depth + 1, or 0 when the run is a whole segment.  Stage 4 is
// organised around the element count sub_lim that one CTA can merge in shared memory:
//  * a node or leaf of size <= sub_lim whose parent is larger (or that is a root) is one
//    "small task": its whole subtree is merged in shared memory;
//  * larger leaves that must move (odd depth -> scratch buffer; descending and alone in their
//    segment -> reversed in place) get placement tiles; a larger descending leaf of even depth
//    >= 2 is read backwards by its parent's merge;
//  * larger internal nodes are merged by HBM passes, one pass per depth.
// Buffer parity (out_buffer): a node at depth d writes buffer d mod 2 (0 = the caller's arrays)
// and reads its children from buffer (d+1) mod 2, so every leaf starts in buffer (depth mod 2).
// M = sum over leaves of depth x length (Sec. 2.3).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 8) plan_kernel(const pos_t* __restrict__ S, const uint8_t* __restrict__ run_desc,
                            const uint8_t* __restrict__ P, const int32_t* __restrict__ nodeL,
                            const int32_t* __restrict__ nodeR, const uint8_t* __restrict__ ndepth,
                            uint8_t* __restrict__ ldepth, uint8_t* __restrict__ micro, int32_t sub_lim,
                            int32_t micro_lim, int32_t* __restrict__ small_tasks,
                            int32_t* __restrict__ leaf_items, uint32_t* __restrict__ leaf_tile_off,
                            NodeItem* __restrict__ level_items, uint32_t* __restrict__ level_tile_off,
                            int32_t level_cap, uint32_t small_cap, int32_t merge_tile,
                            PlanHeader* __restrict__ hdr) {
  const int32_t r = hdr->runs;
  unsigned long long cost = 0;
  int32_t maxd = 0;
  auto node_size = [&](int32_t j) -> pos_t { return S[nodeR[j]] - S[nodeL[j]]; };
  auto node_parent = [&](int32_t j) -> int32_t {
    const int32_t L = nodeL[j], R = nodeR[j];
    const int pl = P[L], pr = P[R];
    if (pl == 0 && pr == 0) return -1;
    return pl > pr ? L : R;
  };
  for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < r; x += gridDim.x * blockDim.x) {
    // leaf x
    {
      const int pl = P[x], pr = P[x + 1];
      const int32_t par = (pl == 0 && pr == 0) ? -1 : (pl > pr ? x : x + 1);
      const int32_t d = par < 0 ? 0 : ndepth[par] + 1;
      ldepth[x] = (uint8_t)d;
      maxd = max(maxd, d);
      const pos_t len = S[x + 1] - S[x];
      cost += (unsigned long long)d * (unsigned long long)len;
      if (len <= sub_lim) {
        if (par < 0 || node_size(par) > sub_lim) {
          const uint32_t slot = atomicAdd(&hdr->n_small, 1u);
          if (slot < small_cap) small_tasks[slot] = ~x;  // leaf task
          else post_status(&hdr->status, nullptr, kDevInternal);
          atomicAdd(&hdr->small_elems, (unsigned long long)len);
        }
      } else {
        const bool desc = (run_desc[x] & 1) != 0;
        if (run_desc[x] & 2) post_status(&hdr->status, nullptr, kDevInternal);  // extended runs are short
        // odd depth: copied to the scratch buffer (reversed on the way if descending); a
        // descending leaf of even depth >= 2 stays where it is and its parent's level pass reads
        // it backwards; only a descending leaf that is a whole segment (depth 0, no merge above
        // it) is reversed in place
        uint32_t tiles = 0;
        const bool odd_buf = out_buffer(d) == 1;
        if (odd_buf) tiles = len / kMergeTile + (len % kMergeTile != 0 ? 1u : 0u);
        else if (desc && d == 0) tiles = (len / 2) / kMergeTile + ((len / 2) % kMergeTile != 0 ? 1u : 0u);
        if (tiles) {
          const unsigned long long old = atomicAdd(&hdr->leaf_ctr, (1ull << 32) | tiles);
          const uint32_t slot = (uint32_t)(old >> 32);
          if (slot < (uint32_t)level_cap) {
            leaf_items[slot] = x;
            leaf_tile_off[slot] = (uint32_t)(old & 0xffffffffu);
            atomicAdd(&hdr->place_elems, (unsigned long long)(odd_buf ? len : 2 * (len / 2)));
          } else {
            post_status(&hdr->status, nullptr, kDevInternal);
          }
        }
      }
    }
    // node x (boundary between runs x-1 and x)
    if (x >= 1 && P[x] >= 1) {
      const pos_t lo = S[nodeL[x]], hi = S[nodeR[x]];
      const pos_t size = hi - lo;
      const int32_t par = node_parent(x);
      const pos_t psize = par < 0 ? ~(pos_t)0 : node_size(par);
      micro[x] = (size <= (pos_t)micro_lim && psize > (pos_t)micro_lim) ? 1 : 0;
      if (size <= sub_lim) {
        if (psize > (pos_t)sub_lim) {
          const uint32_t slot = atomicAdd(&hdr->n_small, 1u);
          if (slot < small_cap) small_tasks[slot] = x;
          else post_status(&hdr->status, nullptr, kDevInternal);
          atomicAdd(&hdr->small_elems, (unsigned long long)size);
        }
      } else {
        const int d = ndepth[x];
        // output tiles: from lo to the next multiple of merge_tile, then whole tiles
        const uint32_t tiles = (hi - 1) / (uint32_t)merge_tile - lo / (uint32_t)merge_tile + 1;
        if (d >= kMaxLevels) {
          post_status(&hdr->status, nullptr, kDevInternal);
        } else {
          // children that are large descending leaves of even depth are read backwards by the
          // level pass (bit 0: left child, bit 1: right child); only nodes of odd depth have them
          int32_t rev = 0;
          if (d & 1) {
            if (nodeL[x] == x - 1 && (run_desc[x - 1] & 1) && S[x] - S[x - 1] > sub_lim) rev |= 1;
            if (nodeR[x] == x + 1 && (run_desc[x] & 1) && S[x + 1] - S[x] > sub_lim) rev |= 2;
          }
          const unsigned long long old = atomicAdd(&hdr->level_ctr[d], (1ull << 32) | tiles);
          const uint32_t slot = (uint32_t)(old >> 32);
          if (slot < (uint32_t)level_cap) {
            level_items[(size_t)d * level_cap + slot] = NodeItem{lo, S[x], hi, rev};
            level_tile_off[(size_t)d * level_cap + slot] = (uint32_t)(old & 0xffffffffu);
            atomicAdd(&hdr->level_elems[d], (unsigned long long)size);
          } else {
            post_status(&hdr->status, nullptr, kDevInternal);
          }
        }
      }
    }
  }
  // block reductions of cost and max depth
  __shared__ unsigned long long s_cost;
  __shared__ int32_t s_maxd;
  if (threadIdx.x == 0) {
    s_cost = 0;
    s_maxd = 0;
  }
  __syncthreads();
  for (int d = 16; d >= 1; d >>= 1) {
    cost += __shfl_down_sync(0xffffffffu, cost, d);
    maxd = max(maxd, __shfl_down_sync(0xffffffffu, maxd, d));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s_cost, cost);
    atomicMax(&s_maxd, maxd);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&hdr->cost, s_cost);
    atomicMax(&hdr->max_leaf_depth, s_maxd);
  }
}

// Sum over runs of L * log2(L) and per-segment n * log2(n) pieces for the entropy statistic:
// n H = sum_segments n_s lg n_s - sum_runs L lg L.  (Statistic only; not on the sort path.)
__global__ void entropy_kernel(const pos_t* __restrict__ S, const PlanHeader* __restrict__ hdr, double* out) {
  const int32_t r = hdr->runs;
  double acc = 0.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < r; i += gridDim.x * blockDim.x) {
    const double L = (double)(S[i + 1] - S[i]);
    acc += L * (double)log2f((float)L);
  }
  for (int d = 16; d >= 1; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// Plan header to a mapped host buffer (zero-copy): the host reads it after an event, without a
// device-to-host copy that would queue behind large copies of other streams.
__global__ void header_out_kernel(const PlanHeader* __restrict__ hdr, PlanHeader* out) {
  static_assert(sizeof(PlanHeader) % 4 == 0, "header is whole words");
  const uint32_t* src = (const uint32_t*)hdr;
  volatile uint32_t* dst = (volatile uint32_t*)out;
  for (int i = threadIdx.x; i < (int)(sizeof(PlanHeader) / 4); i += blockDim.x) dst[i] = src[i];
  __threadfence_system();
}

// Segment offsets must start at 0, be non-decreasing and end at n (and, with a caller's bound,
// no segment may be longer than max_segment).
__global__ void check_offsets_kernel(const int64_t* __restrict__ offsets, int32_t count, int64_t n,
                                     int64_t max_segment, PlanHeader* __restrict__ hdr) {
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= count; k += gridDim.x * blockDim.x) {
    bool bad = false;
    if (k == 0) bad = offsets[0] != 0;
    else bad = offsets[k] < offsets[k - 1] || (max_segment > 0 && offsets[k] - offsets[k - 1] > max_segment);
    if (k == count) bad = bad || offsets[k] != n;
    if (bad) post_status(&hdr->status, nullptr, kDevBadOffsets);
  }
}

// ---------------------------------------------------------------------------------------
// Host launchers for the key-independent stages.
// ---------------------------------------------------------------------------------------
// Grid of per_sm resident CTAs per SM (each kernel's launch bounds allow the per_sm it is
// launched with, so all of its CTAs are resident at once).
static int persistent_blocks(int per_sm) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms * per_sm;
}

// Peeksort tree levels launched: one per node depth the plan can hold (0 .. kMaxLevels-1) plus
// one more, whose ranges (a tree deeper than the plan's per-depth lists) post an internal error.
// Launches past the tree's height find no ranges and return at once.
static int peek_levels(int64_t) { return kMaxLevels + 1; }

static cudaError_t launch_peek_tree(const Ctx& c) {
  const int grid = persistent_blocks(8);
  cudaError_t e = cudaMemsetAsync(c.peek_count, 0, (kMaxLevels + 1) * sizeof(uint32_t), c.stream);
  if (e != cudaSuccess) return e;
  peek_init_kernel<<<grid, 256, 0, c.stream>>>(c.S, c.run_seg, c.offsets, c.P, c.peek_front[0], c.peek_count, c.hdr);
  const int levels = peek_levels(c.n);
  for (int d = 0; d < levels; ++d)
    peek_level_kernel<<<grid, 256, 0, c.stream>>>(c.S, d, c.peek_front[d & 1], c.peek_front[(d + 1) & 1],
                                                  c.peek_count, c.peek_front_cap, c.P, c.nodeL, c.nodeR,
                                                  c.ndepth, c.hdr);
  return cudaGetLastError();
}

int meta_launches(const Ctx& c) { return c.tree == 1 ? 2 + peek_levels(c.n) : 8; }

cudaError_t launch_meta_stages(const Ctx& c) {
  const int grid = persistent_blocks(8);
  if (c.tree == 1) {
    cudaError_t e = launch_peek_tree(c);
    if (e != cudaSuccess) return e;
    plan_kernel<<<grid, 256, 0, c.stream>>>(c.S, c.run_desc, c.P, c.nodeL, c.nodeR, c.ndepth, c.ldepth, c.micro,
                                            c.sub_lim, micro_tile(c.key_bytes), c.small_tasks, c.leaf_items, c.leaf_tile_off,
                                            c.level_items, c.level_tile_off, c.level_cap, (uint32_t)std::min<int64_t>(c.run_cap, 0xffffffffll), c.merge_tile,
                                            c.hdr);
    return cudaGetLastError();
  }
  node_power_kernel<<<persistent_blocks(6), 256, 0, c.stream>>>(c.S, c.run_seg, c.offsets, c.n, c.P, c.hdr);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tree_apply_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTreeApplySmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tree_apply_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTreeApplySmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // both grids are what is resident at once (the apply kernel's 42 KB of shared memory and 48
  // registers allow 5 CTAs per SM), so no CTA waits for a second wave
  static int apply_per_sm = 0, summary_per_sm = 0;
  if (apply_per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&apply_per_sm, tree_apply_kernel<true>,
                                                                  kTreeThreads, kTreeApplySmem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&summary_per_sm, tree_summary_kernel<true>, kTreeThreads,
                                                        kTreeSummarySmem);
    if (e != cudaSuccess) return e;
    apply_per_sm = std::max(1, std::min(apply_per_sm, 8));
    summary_per_sm = std::max(1, std::min(summary_per_sm, 4));
  }
  const int tgrid = persistent_blocks(summary_per_sm), agrid = persistent_blocks(apply_per_sm);
  tree_summary_kernel<false><<<tgrid, kTreeThreads, kTreeSummarySmem, c.stream>>>(c.P, c.hdr, c.tree_sum, c.tree_stride);
  tree_scan_kernel<<<32, kScanThreads, 0, c.stream>>>(c.hdr, c.tree_sum, c.tree_pre, c.tree_stride);
  tree_apply_kernel<false><<<agrid, kTreeThreads, kTreeApplySmem, c.stream>>>(c.P, c.hdr, c.tree_pre, c.tree_stride, c.nodeL, c.ndepth);
  tree_summary_kernel<true><<<tgrid, kTreeThreads, kTreeSummarySmem, c.stream>>>(c.P, c.hdr, c.tree_sum, c.tree_stride);
  tree_scan_kernel<<<32, kScanThreads, 0, c.stream>>>(c.hdr, c.tree_sum, c.tree_pre, c.tree_stride);
  tree_apply_kernel<true><<<agrid, kTreeThreads, kTreeApplySmem, c.stream>>>(c.P, c.hdr, c.tree_pre, c.tree_stride, c.nodeR, c.ndepth);
  plan_kernel<<<grid, 256, 0, c.stream>>>(c.S, c.run_desc, c.P, c.nodeL, c.nodeR, c.ndepth, c.ldepth, c.micro,
                                          c.sub_lim, micro_tile(c.key_bytes), c.small_tasks, c.leaf_items, c.leaf_tile_off,
                                          c.level_items, c.level_tile_off, c.level_cap, (uint32_t)std::min<int64_t>(c.run_cap, 0xffffffffll), c.merge_tile,
                                          c.hdr);
  return cudaGetLastError();
}

cudaError_t launch_entropy(const Ctx& c, double* d_out) {
  entropy_kernel<<<persistent_blocks(4), 256, 0, c.stream>>>(c.S, c.hdr, d_out);
  return cudaGetLastError();
}

cudaError_t launch_header_out(const Ctx& c, PlanHeader* mapped) {
  header_out_kernel<<<1, 128, 0, c.stream>>>(c.hdr, mapped);
  return cudaGetLastError();
}

// Device-driven calls: status bits the plan posted in the header reach the library's status
// word (read by ps_stream_status) without a host round trip.
__global__ void status_out_kernel(const PlanHeader* __restrict__ hdr, uint32_t* lib_status) {
  if (threadIdx.x == 0 && lib_status != nullptr) {
    const uint32_t st = hdr->status;
    if (st) atomicOr(lib_status, st);
  }
}

cudaError_t launch_status_out(const Ctx& c) {
  status_out_kernel<<<1, 32, 0, c.stream>>>(c.hdr, c.lib_status);
  return cudaGetLastError();
}

// Failure-path self-test: one warp waits on a shared-memory mbarrier that nothing completes --
// what a level pass's consumers would see if a stage's copies never landed -- with the same
// bounded poll loop; it gives up after `polls` polls, posts kDevTimeout to the library's status
// word and returns, so the context stays usable.
__global__ void wait_timeout_probe_kernel(uint32_t polls, uint32_t* lib_status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  bool done = false;
  for (uint32_t t = 0; t < polls && !done; ++t) done = mbar_try_wait(&bar, 0);
  if (!__all_sync(0xffffffffu, done) && threadIdx.x == 0) post_status(nullptr, lib_status, kDevTimeout);
}

cudaError_t launch_wait_timeout_probe(uint32_t polls, uint32_t* lib_status, cudaStream_t s) {
  wait_timeout_probe_kernel<<<1, 32, 0, s>>>(polls, lib_status);
  return cudaGetLastError();
}

cudaError_t launch_check_offsets(const Ctx& c) {
  check_offsets_kernel<<<persistent_blocks(1), 256, 0, c.stream>>>(c.offsets, c.count, c.n, c.max_segment, c.hdr);
  return cudaGetLastError();
}

}  // namespace ps

namespace ps {
unsigned long long bounds_hits_meta() { return bounds_hits_here(); }
}  // namespace ps
