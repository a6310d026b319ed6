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
// the entry state) makes the same scan count the runs, so run starts are written compacted.  The
// scan runs as reduce (tile functions) -> one-CTA scan over tiles -> emit, reading the keys twice;
// no block waits on another.
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

// Tile function word: map in [5:0], c0/c1/c2 in 16-bit fields at 8, 24, 40 (tile counts <= 4096).
__device__ __forceinline__ uint64_t pack_agg(const Fn& f) {
  return (uint64_t)f.map | ((uint64_t)f.c0 << 8) | ((uint64_t)f.c1 << 24) | ((uint64_t)f.c2 << 40);
}
__device__ __forceinline__ Fn unpack_agg(uint64_t w) {
  return Fn{(uint32_t)(w & 63u), (uint32_t)((w >> 8) & 0xffffu), (uint32_t)((w >> 24) & 0xffffu),
            (uint32_t)((w >> 40) & 0xffffu)};
}

// Thread function word: map in [5:0], c0/c1/c2 in 6-bit fields at 6, 12, 18 (counts <= 32).
__device__ __forceinline__ uint32_t pack_thread_fn(const Fn& f) {
  return f.map | (f.c0 << 6) | (f.c1 << 12) | (f.c2 << 18);
}
__device__ __forceinline__ Fn unpack_thread_fn(uint32_t w) {
  return Fn{w & 63u, (w >> 6) & 63u, (w >> 12) & 63u, (w >> 18) & 63u};
}

// The same function inside one tile, packed for the block scans: entry state x in bits
// [16x, 16x + 16) holding the exit state (2 bits) and the run starts produced (14 bits; a tile
// produces at most kDetectTile of them).  Composing a then b maps entry x to b's entry for a's
// exit, with a's count added: one extract per entry state, and one 64-bit shuffle per scan step.
typedef uint64_t TFn;
__device__ __forceinline__ TFn tfn_identity() { return 0ull | (1ull << 16) | (2ull << 32); }
__device__ __forceinline__ TFn tfn_of(const Fn& f) {
  return (uint64_t)((f.map & 3u) | (f.c0 << 2)) | ((uint64_t)(((f.map >> 2) & 3u) | (f.c1 << 2)) << 16) |
         ((uint64_t)(((f.map >> 4) & 3u) | (f.c2 << 2)) << 32);
}
__device__ __forceinline__ Fn fn_of(TFn t) {
  Fn f;
  f.map = (uint32_t)(t & 3u) | ((uint32_t)((t >> 16) & 3u) << 2) | ((uint32_t)((t >> 32) & 3u) << 4);
  f.c0 = (uint32_t)(t & 0xFFFFu) >> 2;
  f.c1 = (uint32_t)((t >> 16) & 0xFFFFu) >> 2;
  f.c2 = (uint32_t)((t >> 32) & 0xFFFFu) >> 2;
  return f;
}
__device__ __forceinline__ TFn tfn_then(TFn a, TFn b) {
  TFn r = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const uint32_t ax = (uint32_t)(a >> (16 * x)) & 0xFFFFu;
    const uint32_t bx = (uint32_t)(b >> (16 * (ax & 3u))) & 0xFFFFu;
    r |= (uint64_t)(bx + (ax & 0xFFFCu)) << (16 * x);
  }
  return r;
}
__device__ __forceinline__ uint32_t tfn_exit(TFn t, uint32_t x) { return (uint32_t)(t >> (16 * x)) & 3u; }
__device__ __forceinline__ uint32_t tfn_cnt(TFn t, uint32_t x) { return ((uint32_t)(t >> (16 * x)) & 0xFFFFu) >> 2; }

// Largest k with offsets[k] <= p (the segment containing p when segments are non-empty).
__device__ __forceinline__ int32_t segment_of(const int64_t* offsets, int32_t count, int64_t p) {
  int32_t lo = 0, hi = count;  // offsets[0] = 0 <= p
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

// Key u of a 16-byte chunk (four 4-byte keys or two 8-byte keys, little-endian).
template <class T>
__device__ __forceinline__ T chunk_key(const uint4& w, int u) {
  if constexpr (sizeof(T) == 4) {
    return (T)(u == 0 ? w.x : u == 1 ? w.y : u == 2 ? w.z : w.w);
  } else {
    return u == 0 ? (T)(((uint64_t)w.y << 32) | w.x) : (T)(((uint64_t)w.w << 32) | w.z);
  }
}

// The thread's view of its kDetectItems = 32 consecutive positions p0 .. p0+31:
//   L  bit q (q = 0..32): key[p0+q-1] <= key[p0+q]  (the pair into position p0+q)
//   F  bit q (q = 0..32): position p0+q is forced to START (position 0 or a segment start)
// Runs are walked start to start with bit operations instead of one automaton step per position:
// a run that starts at position s has direction L[s+1] (weakly ascending if set) and the next
// run starts at the first q >= s+2 whose pair disagrees with that direction, or at the first
// forced q >= s+1.  A run already open when the thread begins, with direction e, ends at the
// first q >= 0 whose pair disagrees with e (or is forced); entering in START at position p0-1
// behaves like entering with direction L[0].
template <class K>
struct ThreadRuns {
  typedef typename K::T T;
  int64_t p0;          // first position
  int32_t nvalid;      // positions p0 .. p0+nvalid-1 exist
  uint64_t L, F, valid;

  __device__ __forceinline__ void load(const T* __restrict__ keys, int64_t n, const int64_t* __restrict__ offsets,
                                       int32_t count, int32_t tile, int tid) {
    p0 = (int64_t)tile * kDetectTile + tid * kDetectItems;
    nvalid = (int32_t)max((int64_t)0, min((int64_t)kDetectItems, n - p0));
    valid = (nvalid >= 64) ? ~0ull : ((1ull << nvalid) - 1ull);
    L = 0;
    F = 0;
    if (nvalid == 0) return;
    T prev = (p0 > 0) ? keys[p0 - 1] : (T)0;
    if (kDetectItems < n - p0 && ((uintptr_t)(keys + p0) & 15u) == 0) {
      constexpr int kPer = 16 / (int)sizeof(T);
      const uint4* src = reinterpret_cast<const uint4*>(keys + p0);
#pragma unroll
      for (int v = 0; v < kDetectItems / kPer; ++v) {
        const uint4 w = __ldg(src + v);
        const T* wt = reinterpret_cast<const T*>(&w);
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
          const T cur = wt[u];
          L |= (uint64_t)(K::ord(prev) <= K::ord(cur)) << (v * kPer + u);
          prev = cur;
        }
      }
      L |= (uint64_t)(K::ord(prev) <= K::ord(keys[p0 + kDetectItems])) << kDetectItems;
    } else {
      for (int q = 0; q < nvalid; ++q) {
        const T cur = keys[p0 + q];
        L |= (uint64_t)(K::ord(prev) <= K::ord(cur)) << q;
        prev = cur;
      }
      if (kDetectItems < n - p0) L |= (uint64_t)(K::ord(prev) <= K::ord(keys[p0 + kDetectItems])) << kDetectItems;
    }
    forced_starts(offsets, count);
  }
  // F from position 0 and the segment offsets
  __device__ __forceinline__ void forced_starts(const int64_t* __restrict__ offsets, int32_t count) {
    if (p0 == 0) F |= 1ull;
    if (offsets != nullptr) {
      // every offsets value in [p0, p0 + kDetectItems] marks a forced start
      int32_t k = segment_of(offsets, count, p0);
      while (k <= count) {
        const int64_t o = offsets[k];
        if (o > p0 + kDetectItems) break;
        if (o >= p0) F |= 1ull << (int)(o - p0);
        ++k;
      }
    }
  }
  // The same view with the warp's 32 x 32 keys staged through shared memory.  A lane's 32 keys
  // form a row of 16-byte chunks (8 for 4-byte keys, 16 for 8-byte keys), staged eight chunks
  // per lane at a time (4 KB per warp; 8-byte keys take two such halves): each lane issues
  // eight 16-byte cp.async copies at lane-consecutive addresses (eight lanes cover 128
  // contiguous bytes of one row, so every copy instruction reads whole 128-byte segments and no
  // registers are held while the copies are in flight), then reads its own eight chunks back.
  // Chunk c of lane l's staged row is stored at index c ^ (l & 7), so the copies of a quarter
  // warp (one row) and the row reads of a quarter warp (eight rows, one chunk index each) both
  // cover eight distinct 16-byte bank groups.  The pairs into the lane's first position and out
  // of its last one use the neighbouring lanes' keys.  A warp whose keys (with the look-ahead)
  // are not wholly inside the array, or whose keys are not 16-byte aligned, takes load().
  __device__ __forceinline__ void load_staged(const T* __restrict__ keys, int64_t n, const int64_t* __restrict__ offsets,
                                              int32_t count, int32_t tile, int tid, uint4* __restrict__ stage) {
    static_assert(kDetectItems == 32, "a lane row is 32 keys");
    constexpr int kPerChunk = 16 / (int)sizeof(T);         // keys per 16-byte chunk
    constexpr int kRowChunks = kDetectItems / kPerChunk;   // chunks per lane row: 8 or 16
    constexpr int kHalves = kRowChunks / 8;                // staged eight chunks per lane at a time
    constexpr int kWarpKeys = 32 * kDetectItems;
    const int lane = tid & 31;
    const int64_t wp0 = (int64_t)tile * kDetectTile + (tid - lane) * kDetectItems;
    if (!(kWarpKeys < n - wp0 && ((uintptr_t)keys & 15u) == 0)) {  // uniform over the warp
      load(keys, n, offsets, count, tile, tid);
      return;
    }
    const uint4* __restrict__ src = reinterpret_cast<const uint4*>(keys + wp0);
    p0 = wp0 + lane * kDetectItems;
    nvalid = kDetectItems;
    valid = (1ull << kDetectItems) - 1ull;
    L = 0;
    F = 0;
    T first = 0, last = 0;
#pragma unroll
    for (int h = 0; h < kHalves; ++h) {
      if (h > 0) __syncwarp();  // every lane has read the previous half
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int g = j * 32 + lane, row = g >> 3, c = g & 7;  // staged chunk g of the warp's 256
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(stage + row * 8 + (c ^ (row & 7)))),
                     "l"(src + row * kRowChunks + h * 8 + c)
                     : "memory");
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncwarp();
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const uint4 w = stage[lane * 8 + (v ^ (lane & 7))];
#pragma unroll
        for (int u = 0; u < kPerChunk; ++u) {
          const T x = chunk_key<T>(w, u);
          const int q = (h * 8 + v) * kPerChunk + u;
          if (q == 0) first = x;
          else L |= (uint64_t)(K::ord(last) <= K::ord(x)) << q;
          last = x;
        }
      }
    }
    T before = __shfl_up_sync(0xffffffffu, last, 1);
    T after = __shfl_down_sync(0xffffffffu, first, 1);
    if (lane == 0) before = (p0 > 0) ? keys[p0 - 1] : (T)0;
    if (lane == 31) after = keys[p0 + kDetectItems];  // p0 + 32 = wp0 + kWarpKeys < n
    L |= (uint64_t)(K::ord(before) <= K::ord(first));
    L |= (uint64_t)(K::ord(last) <= K::ord(after)) << kDetectItems;
    forced_starts(offsets, count);
  }
  // rebuild the view from the pair / forced-start masks the reduce pass saved
  __device__ __forceinline__ void restore(int64_t n, int32_t tile, int tid, uint64_t l, uint64_t f) {
    p0 = (int64_t)tile * kDetectTile + tid * kDetectItems;
    nvalid = (int32_t)max((int64_t)0, min((int64_t)kDetectItems, n - p0));
    valid = (nvalid >= 64) ? ~0ull : ((1ull << nvalid) - 1ull);
    L = l;
    F = f;
  }
  // first run start at or after position 0 for a run entered with direction e (1 = ascending)
  __device__ __forceinline__ int first_start(uint32_t e) const {
    const uint64_t c = (((e ? ~L : L)) | F) & valid;
    return c ? __ffsll((long long)c) - 1 : 64;
  }
  // next run start after a run that starts at pos (pos < nvalid), or 64
  __device__ __forceinline__ int next_start(int pos) const {
    const uint32_t d = (uint32_t)(L >> (pos + 1)) & 1u;
    const uint64_t ge2 = (pos + 2 >= 64) ? 0ull : (~0ull << (pos + 2));
    const uint64_t ge1 = ~0ull << (pos + 1);
    const uint64_t c = ((((d ? ~L : L)) & ge2) | (F & ge1)) & valid;
    return c ? __ffsll((long long)c) - 1 : 64;
  }
  // state after the thread's last position for a chain whose last run starts at pos
  __device__ __forceinline__ uint32_t open_state(int pos) const {
    if (pos + 1 >= kDetectItems) return 0u;  // the last position itself starts a run
    return ((L >> (pos + 1)) & 1ull) ? 1u : 2u;
  }
  // walk the chain from its first start; returns the number of starts and the exit state
  __device__ __forceinline__ void chain(int pos, uint32_t none_state, uint32_t& cnt, uint32_t& exit_state) const {
    if ((F >> 1) == 0) {  // no forced start past position 0: all starts at once
      const uint64_t m = chain_starts(pos);
      cnt = (uint32_t)__popcll(m);
      exit_state = m ? open_state(63 - __clzll((long long)m)) : none_state;
      return;
    }
    cnt = 0;
    exit_state = none_state;
    while (pos < nvalid) {
      ++cnt;
      exit_state = open_state(pos);
      pos = next_start(pos);
    }
  }
  // The run starts of the chain that begins at pos0, as a mask, for a view with no forced start
  // past position 0.  After a start s the next one is the first q >= s + 2 whose pair disagrees
  // with the run's direction L[s+1], which is the first change point (q with L[q] != L[q-1]) at
  // or after s + 2.  Inside a maximal block of consecutive change points the chain therefore takes
  // every other point from the block's first one, and it always takes a block's first point (the
  // position before it is no change point, so the previous start lies at least two below it).
  // With pos0 made the first point of its block, the starts are the even-offset points of every
  // block: the blocks that begin at even positions keep their even bits, the others their odd
  // bits (a block's bits are found by adding its first bit, whose carry runs through the block).
  __device__ __forceinline__ uint64_t chain_starts(int pos0) const {
    if (pos0 >= nvalid) return 0ull;
    const uint64_t c = ((L ^ (L << 1)) & (~0ull << (pos0 + 1))) | (1ull << pos0);
    constexpr uint64_t kEven = 0x5555555555555555ull;
    const uint64_t even_firsts = c & ~(c << 1) & kEven;
    const uint64_t even_blocks = ((c + even_firsts) ^ c) & c;
    return ((even_blocks & kEven) | (c & ~even_blocks & ~kEven)) & valid;
  }
  __device__ __forceinline__ Fn aggregate() const {
    if (nvalid == 0) return fn_identity();
    Fn f;
    if (F & 1ull) {
      uint32_t c, x;
      chain(0, 0u, c, x);
      f.map = x | (x << 2) | (x << 4);
      f.c0 = f.c1 = f.c2 = c;
      return f;
    }
    uint32_t c1, x1, c0, x0;
    chain(first_start(1u), 1u, c1, x1);  // entered ascending
    chain(first_start(0u), 2u, c0, x0);  // entered descending
    const bool l0 = (L & 1ull) != 0;    // entering at START behaves like direction L[0]
    f.map = (l0 ? x1 : x0) | (x1 << 2) | (x0 << 4);
    f.c0 = l0 ? c1 : c0;
    f.c1 = c1;
    f.c2 = c0;
    return f;
  }
};

// Pass 1: the composed transition function (with run-start counts) of every tile.
template <class K>
__global__ void __launch_bounds__(kDetectThreads)
detect_reduce_kernel(const typename K::T* __restrict__ keys, int64_t n, const int64_t* __restrict__ offsets,
                     int32_t count, uint64_t* __restrict__ tile_agg, uint64_t* __restrict__ thr_L,
                     uint64_t* __restrict__ thr_F, uint32_t* __restrict__ thr_fn) {
  __shared__ TFn warp_tot[kDetectThreads / 32];
  __shared__ uint4 stage[kDetectThreads / 32 * 256];  // 4 KB of staged keys per warp
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  ThreadRuns<K> tr;
  tr.load_staged(keys, n, offsets, count, blockIdx.x, tid, stage + warp * 256);
  const Fn mine = tr.aggregate();
  // the emit pass replays the runs from these instead of reading the keys again
  const size_t gt = (size_t)blockIdx.x * kDetectThreads + tid;
  thr_L[gt] = tr.L;
  if (offsets != nullptr) thr_F[gt] = tr.F;
  thr_fn[gt] = pack_thread_fn(mine);
  TFn incl = tfn_of(mine);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const TFn up = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl = tfn_then(up, incl);
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (tid == 0) {
    TFn t = tfn_identity();
    for (int w = 0; w < kDetectThreads / 32; ++w) t = tfn_then(t, warp_tot[w]);
    tile_agg[blockIdx.x] = pack_agg(fn_of(t));
  }
}

// Pass 2 (one CTA of 1024 threads): scan of the tile functions from the START state at
// position 0.  tile_pre[t] = (state entering tile t) | (run starts before tile t) << 2;
// hdr->runs = r and S[r] = n, or kDevTooManyRuns when r exceeds kMaxRuns (kDevInternal if the run
// arrays' capacity run_cap could not hold r + 1 entries, which the run-length bound excludes).
static __global__ void __launch_bounds__(1024)
detect_scan_kernel(const uint64_t* __restrict__ tile_agg, int32_t ntiles, int64_t n, int64_t run_cap,
                   uint64_t* __restrict__ tile_pre, pos_t* __restrict__ S, PlanHeader* __restrict__ hdr) {
  __shared__ Fn warp_tot[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t per = (ntiles + 1023) / 1024;
  const int32_t t0 = tid * per, t1 = min(t0 + per, ntiles);
  Fn mine = fn_identity();
  for (int32_t t = t0; t < t1; ++t) mine = fn_then(mine, unpack_agg(tile_agg[t]));
  Fn incl = mine;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const Fn up = fn_shfl_up(incl, d);
    if (lane >= d) incl = fn_then(up, incl);
  }
  if (lane == 31) warp_tot[warp] = incl;
  Fn excl = fn_shfl_up(incl, 1);
  if (lane == 0) excl = fn_identity();
  __syncthreads();
  Fn wp = fn_identity();
  for (int w = 0; w < warp; ++w) wp = fn_then(wp, warp_tot[w]);
  excl = fn_then(wp, excl);
  uint32_t state = fn_exit(excl, 0);
  uint64_t cnt = fn_cnt(excl, 0);  // run counts reach n < 2^32
  for (int32_t t = t0; t < t1; ++t) {
    tile_pre[t] = (uint64_t)state | (cnt << 2);
    const Fn f = unpack_agg(tile_agg[t]);
    cnt += fn_cnt(f, state);
    state = fn_exit(f, state);
  }
  if (t0 < ntiles && t1 == ntiles) {
    if (cnt > (uint64_t)kMaxRuns || cnt + 1 > (uint64_t)run_cap) {
      hdr->runs = 0;
      atomicOr(&hdr->status, (uint32_t)(cnt + 1 > (uint64_t)run_cap ? kDevInternal : kDevTooManyRuns));
    } else {
      hdr->runs = (int32_t)cnt;
      S[cnt] = (pos_t)n;
    }
  }
}

// Pass 3: every thread replays its positions from its entry state and writes its run starts
// S[k], directions run_desc[k] and segments run_seg[k] at their global ranks.  Without segments a
// tile's runs (at most kDetectTile / 2 of them: every greedy run but the array's last has two
// elements or more) are collected in shared memory and written out coalesced.
constexpr int kEmitStage = kDetectTile / 2 + 32;

template <class K>
__global__ void __launch_bounds__(kDetectThreads)
detect_emit_kernel(int64_t n, int64_t run_cap, const int64_t* __restrict__ offsets, int32_t count,
                   const uint64_t* __restrict__ tile_pre, const uint64_t* __restrict__ thr_L,
                   const uint64_t* __restrict__ thr_F, const uint32_t* __restrict__ thr_fn,
                   pos_t* __restrict__ S, uint8_t* __restrict__ run_desc, int32_t* __restrict__ run_seg) {
  __shared__ TFn warp_tot[kDetectThreads / 32];
  __shared__ pos_t s_start[kEmitStage];
  __shared__ uint8_t s_desc[kEmitStage];
  __shared__ uint32_t s_count;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t gt = (size_t)blockIdx.x * kDetectThreads + tid;
  ThreadRuns<K> tr;
  tr.restore(n, blockIdx.x, tid, thr_L[gt], offsets != nullptr ? thr_F[gt] : (blockIdx.x == 0 && tid == 0 ? 1ull : 0ull));
  TFn incl = tfn_of(unpack_thread_fn(thr_fn[gt]));
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const TFn up = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl = tfn_then(up, incl);
  }
  if (lane == 31) warp_tot[warp] = incl;
  TFn excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = tfn_identity();
  __syncthreads();
  TFn wp = tfn_identity();
  for (int w = 0; w < warp; ++w) wp = tfn_then(wp, warp_tot[w]);
  excl = tfn_then(wp, excl);
  const bool staged = offsets == nullptr;  // uniform over the grid
  const uint64_t pre = tile_pre[blockIdx.x];
  const uint32_t tile_entry = (uint32_t)(pre & 3u);
  const uint64_t tile_base = pre >> 2;
  const uint32_t entry = tfn_exit(excl, tile_entry);  // state at position p0 - 1
  uint64_t idx = tile_base + tfn_cnt(excl, tile_entry);
  auto emit = [&](int pos, int32_t seg) {
    const int64_t p = tr.p0 + pos;
    // descending iff the pair (p, p+1) lies inside the segment and is strictly decreasing
    const bool desc = (p + 1 < n) && !((tr.F >> (pos + 1)) & 1ull) && !((tr.L >> (pos + 1)) & 1ull);
    const uint64_t local = idx - tile_base;
    if (staged && local < (uint64_t)kEmitStage) {
      s_start[local] = (pos_t)p;
      s_desc[local] = desc ? 1 : 0;
    } else if (idx < (uint64_t)run_cap) {  // always true when the tile counts are consistent
      S[idx] = (pos_t)p;
      run_desc[idx] = desc ? 1 : 0;
      if (run_seg) run_seg[idx] = seg;
    }
    ++idx;
  };
  if (tr.nvalid > 0) {
    int pos;
    if (tr.F & 1ull) pos = 0;
    else if (entry == 0) pos = tr.first_start((uint32_t)(tr.L & 1ull));
    else pos = tr.first_start(entry == 1 ? 1u : 0u);
    if ((tr.F >> 1) == 0) {  // no segment start past the thread's first position
      const int32_t seg = (offsets != nullptr) ? segment_of(offsets, count, tr.p0) : 0;
      uint64_t m = tr.chain_starts(pos);
      while (m) {
        emit(__ffsll((long long)m) - 1, seg);
        m &= m - 1;
      }
    } else {
      int32_t seg = segment_of(offsets, count, tr.p0);
      while (pos < tr.nvalid) {
        if ((tr.F >> pos) & 1ull) seg = segment_of(offsets, count, tr.p0 + pos);
        emit(pos, seg);
        pos = tr.next_start(pos);
      }
    }
  }
  if (!staged) return;
  if (tid == kDetectThreads - 1) s_count = (uint32_t)min(idx - tile_base, (uint64_t)kEmitStage);
  __syncthreads();
  const uint32_t cnt = s_count;
  for (uint32_t i = tid; i < cnt; i += kDetectThreads) {
    if (tile_base + i < (uint64_t)run_cap) {
      S[tile_base + i] = s_start[i];
      run_desc[tile_base + i] = s_desc[i];
    }
  }
}

}  // namespace ps
