// Stage 1: run detection (Sec. 2 run convention; ExtendRunRight of Alg. 2) as one parallel scan.
//
// Greedy left-to-right run finding is a 3-state automaton over the adjacent pairs:
//   START --le--> ASC     START --gt--> DESC
//   ASC   --le--> ASC     ASC   --gt--> START
//   DESC  --le--> START   DESC  --gt--> DESC
// where the transition into position p reads the pair (p-1, p): le = key[p-1] <= key[p].  Position
// p starts a run exactly when the automaton is in START at p (a segment start forces START).  The
// transition functions compose associatively, so the state at every position is an exclusive
// scan of them; attaching to each function the number of run starts it produces (which depends on
// the entry state) makes the same scan count the runs, so run starts are written compacted in one
// pass.  Cross-tile carries use decoupled look-back with bounded waits.
#pragma once

#include "ps_common.cuh"

namespace ps {

// A transition function over {START=0, ASC=1, DESC=2} (2 bits per entry state) together with,
// per entry state, the number of run starts produced.
struct Fn {
  uint32_t map;          // bits [2x, 2x+1] = exit state for entry state x
  uint32_t c0, c1, c2;   // run starts produced for entry state 0, 1, 2
};

__device__ __forceinline__ uint32_t fn_exit(const Fn& f, uint32_t x) { return (f.map >> (2 * x)) & 3u; }
__device__ __forceinline__ uint32_t fn_cnt(const Fn& f, uint32_t x) {
  return x == 0 ? f.c0 : (x == 1 ? f.c1 : f.c2);
}
// a applied first, then b
__device__ __forceinline__ Fn fn_then(const Fn& a, const Fn& b) {
  const uint32_t a0 = a.map & 3u, a1 = (a.map >> 2) & 3u, a2 = (a.map >> 4) & 3u;
  Fn r;
  r.map = fn_exit(b, a0) | (fn_exit(b, a1) << 2) | (fn_exit(b, a2) << 4);
  r.c0 = a.c0 + fn_cnt(b, a0);
  r.c1 = a.c1 + fn_cnt(b, a1);
  r.c2 = a.c2 + fn_cnt(b, a2);
  return r;
}
__device__ __forceinline__ Fn fn_identity() { return Fn{0u | (1u << 2) | (2u << 4), 0, 0, 0}; }
// transition into a position: kind 0 = pair le, 1 = pair gt, 2 = forced START (segment start)
__device__ __forceinline__ Fn fn_of_kind(uint32_t kind) {
  if (kind == 0) return Fn{1u | (1u << 2) | (0u << 4), 0, 0, 1};  // S->A A->A D->S
  if (kind == 1) return Fn{2u | (0u << 2) | (2u << 4), 0, 1, 0};  // S->D A->S D->D
  return Fn{0u, 1, 1, 1};                                          // all -> START
}
__device__ __forceinline__ Fn fn_shfl_up(const Fn& f, int d) {
  Fn r;
  r.map = __shfl_up_sync(0xffffffffu, f.map, d);
  r.c0 = __shfl_up_sync(0xffffffffu, f.c0, d);
  r.c1 = __shfl_up_sync(0xffffffffu, f.c1, d);
  r.c2 = __shfl_up_sync(0xffffffffu, f.c2, d);
  return r;
}
__device__ __forceinline__ Fn fn_shfl_down(const Fn& f, int d) {
  Fn r;
  r.map = __shfl_down_sync(0xffffffffu, f.map, d);
  r.c0 = __shfl_down_sync(0xffffffffu, f.c0, d);
  r.c1 = __shfl_down_sync(0xffffffffu, f.c1, d);
  r.c2 = __shfl_down_sync(0xffffffffu, f.c2, d);
  return r;
}

// Tile descriptor word for the look-back: [63:62] flag (1 aggregate, 2 inclusive prefix).
// Aggregate: map in [5:0], c0/c1/c2 in 16-bit fields at 8, 24, 40 (tile counts <= 4096).
// Prefix: exit state in [1:0], inclusive run count in [33:2].
constexpr uint64_t kFlagAgg = 1ull << 62, kFlagPrefix = 2ull << 62, kFlagMask = 3ull << 62;

__device__ __forceinline__ uint64_t pack_agg(const Fn& f) {
  return kFlagAgg | (uint64_t)f.map | ((uint64_t)f.c0 << 8) | ((uint64_t)f.c1 << 24) | ((uint64_t)f.c2 << 40);
}
__device__ __forceinline__ Fn unpack_agg(uint64_t w) {
  return Fn{(uint32_t)(w & 63u), (uint32_t)((w >> 8) & 0xffffu), (uint32_t)((w >> 24) & 0xffffu),
            (uint32_t)((w >> 40) & 0xffffu)};
}
__device__ __forceinline__ uint64_t pack_prefix(uint32_t state, uint32_t count) {
  return kFlagPrefix | (uint64_t)state | ((uint64_t)count << 2);
}

__device__ __forceinline__ void store_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t load_acquire_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Largest k with offsets[k] <= p (the segment containing p when segments are non-empty).
__device__ __forceinline__ int32_t segment_of(const int64_t* offsets, int32_t count, int32_t p) {
  int32_t lo = 0, hi = count;  // offsets[0] = 0 <= p
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

// One CTA per tile, tiles taken in order from a ticket counter (so predecessors have started).
// Outputs: run starts S[0..r-1] (S[r] = n written by the last tile), run_desc[k], run_seg[k],
// hdr->runs = r.
template <class K>
__global__ void __launch_bounds__(kDetectThreads)
detect_runs_kernel(const typename K::T* __restrict__ keys, int32_t n, const int64_t* __restrict__ offsets,
                   int32_t count, int32_t* __restrict__ S, uint8_t* __restrict__ run_desc,
                   int32_t* __restrict__ run_seg, uint64_t* __restrict__ tile_state, PlanHeader* hdr,
                   uint32_t* lib_status) {
  typedef typename K::T T;
  __shared__ T sk[kDetectTile + 2];
  __shared__ Fn warp_tot[kDetectThreads / 32];
  __shared__ uint32_t s_tile, s_entry, s_base;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(&hdr->detect_ticket, 1u);
  __syncthreads();
  const int32_t tile = (int32_t)s_tile;
  const int32_t t0 = tile * kDetectTile;

  // keys [t0-1, t0+kDetectTile] into shared memory (coalesced)
  for (int i = tid; i < kDetectTile + 2; i += kDetectThreads) {
    const int64_t g = (int64_t)t0 - 1 + i;
    if (g >= 0 && g < n) sk[i] = keys[g];
  }
  __syncthreads();

  // this thread's positions p in [p0, p1); seg0 = segment holding p0, nxt0 = the first segment
  // start >= p0 (a position is a segment start iff it equals some offsets[k])
  const int32_t p0 = t0 + tid * kDetectItems;
  const int32_t p1 = min(p0 + kDetectItems, n);
  int32_t seg0 = 0, nxt0 = n;
  if (offsets != nullptr && p0 < n) {
    seg0 = segment_of(offsets, count, p0);
    nxt0 = ((int32_t)offsets[seg0] == p0) ? p0 : (int32_t)offsets[seg0 + 1];
  }
  // transition kind into position p: 2 = forced start (p = 0 or a segment start), else the pair
  auto kind_at = [&](int32_t p, bool seg_start) -> uint32_t {
    if (p == 0 || seg_start) return 2u;
    return K::ord(sk[p - t0]) <= K::ord(sk[p - t0 + 1]) ? 0u : 1u;
  };

  // thread aggregate
  Fn agg = fn_identity();
  {
    int32_t nxt = nxt0;
    for (int32_t p = p0; p < p1; ++p) {
      const bool st = (p == nxt);
      if (st) nxt = (int32_t)offsets[segment_of(offsets, count, p) + 1];
      agg = fn_then(agg, fn_of_kind(kind_at(p, st)));
    }
  }

  // block exclusive scan of the thread aggregates
  Fn incl = agg;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const Fn up = fn_shfl_up(incl, d);
    if (lane >= d) incl = fn_then(up, incl);
  }
  if (lane == 31) warp_tot[warp] = incl;
  Fn excl = fn_shfl_up(incl, 1);
  if (lane == 0) excl = fn_identity();
  __syncthreads();
  Fn warp_prefix = fn_identity();
  for (int w = 0; w < warp; ++w) warp_prefix = fn_then(warp_prefix, warp_tot[w]);
  excl = fn_then(warp_prefix, excl);

  // tile aggregate and look-back (warp 0)
  if (warp == 0) {
    Fn tile_agg = fn_identity();
    for (int w = 0; w < kDetectThreads / 32; ++w) tile_agg = fn_then(tile_agg, warp_tot[w]);
    uint32_t entry = 0, base = 0;
    if (tile == 0) {
      if (lane == 0) store_release_u64(&tile_state[0], pack_prefix(fn_exit(tile_agg, 0), fn_cnt(tile_agg, 0)));
    } else {
      if (lane == 0) store_release_u64(&tile_state[tile], pack_agg(tile_agg));
      Fn acc = fn_identity();  // composition of tiles (pos, tile)
      int32_t pos = tile - 1;
      bool done = false, timed_out = false;
      uint32_t spins = 0;
      while (!done) {
        const int32_t q = pos - lane;
        uint64_t w = (q >= 0) ? load_acquire_u64(&tile_state[q]) : kFlagPrefix;  // before tile 0: START, 0
        // wait until every descriptor in the window is published
        while (__any_sync(0xffffffffu, (w & kFlagMask) == 0)) {
          if (++spins > kSpinLimit) { timed_out = true; break; }
          __nanosleep(64);
          if ((w & kFlagMask) == 0) w = load_acquire_u64(&tile_state[q]);
        }
        if (__any_sync(0xffffffffu, timed_out)) { timed_out = true; break; }
        const uint32_t pmask = __ballot_sync(0xffffffffu, (w & kFlagMask) == kFlagPrefix);
        const int first_prefix = pmask ? (__ffs(pmask) - 1) : 32;
        // ordered product of the aggregates of lanes [0, first_prefix): higher lanes first
        Fn v = (lane < first_prefix) ? unpack_agg(w) : fn_identity();
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const Fn hi = fn_shfl_down(v, d);
          if (lane + d < 32) v = fn_then(hi, v);
        }
        // lane 0 holds product over lanes 31..0 (identity beyond first_prefix)
        v.map = __shfl_sync(0xffffffffu, v.map, 0);
        v.c0 = __shfl_sync(0xffffffffu, v.c0, 0);
        v.c1 = __shfl_sync(0xffffffffu, v.c1, 0);
        v.c2 = __shfl_sync(0xffffffffu, v.c2, 0);
        acc = fn_then(v, acc);
        if (pmask) {
          const uint64_t pw = __shfl_sync(0xffffffffu, w, first_prefix);
          const uint32_t st = (uint32_t)(pw & 3u);
          const uint32_t cnt = (uint32_t)((pw >> 2) & 0xffffffffu);
          entry = fn_exit(acc, st);
          base = cnt + fn_cnt(acc, st);
          done = true;
        } else {
          pos -= 32;
        }
      }
      if (timed_out) {
        if (lane == 0) post_status(&hdr->status, lib_status, kDevTimeout);
        entry = 0;
        base = 0;
      }
      if (lane == 0)
        store_release_u64(&tile_state[tile],
                          pack_prefix(fn_exit(tile_agg, entry), base + fn_cnt(tile_agg, entry)));
    }
    if (lane == 0) {
      s_entry = entry;
      s_base = base;
    }
  }
  __syncthreads();
  const uint32_t tile_entry = s_entry, tile_base = s_base;

  // emit the run starts of this thread's positions
  uint32_t state = fn_exit(excl, tile_entry);
  uint32_t idx = tile_base + fn_cnt(excl, tile_entry);
  int32_t nxt = nxt0, cur_seg = seg0;
  for (int32_t p = p0; p < p1; ++p) {
    const bool st = (p == nxt);
    if (st) {
      cur_seg = segment_of(offsets, count, p);
      nxt = (int32_t)offsets[cur_seg + 1];
    }
    state = fn_exit(fn_of_kind(kind_at(p, st)), state);
    if (state == 0) {
      // descending iff the pair (p, p+1) lies inside the segment and is strictly decreasing
      bool desc = false;
      if (p + 1 < n && p + 1 != nxt) desc = !(K::ord(sk[p + 1 - t0]) <= K::ord(sk[p + 2 - t0]));
      S[idx] = p;
      run_desc[idx] = desc ? 1 : 0;
      if (run_seg) run_seg[idx] = cur_seg;
      ++idx;
    }
  }
  // the thread holding the last position closes the run array
  if (p0 < n && p1 == n) {
    S[idx] = n;
    hdr->runs = (int32_t)idx;
  }
}

}  // namespace ps
