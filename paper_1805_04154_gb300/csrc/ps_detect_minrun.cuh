// Stage 1 with a minimal run length w (Sec. 5.1: the tuned implementations extend every run
// shorter than w = 24 to w elements by insertion sort, capped at the end of the array).
//
// The run partition is the chain s_0 = 0, s_{i+1} = next(s_i) with
//   next(s) = max(e, min(s + w, end))
// where [s, e) is the greedy run from s (weakly ascending or strictly descending, ExtendRunRight
// of Alg. 2) and `end` is the next forced start (a segment start or n).  A run is "extended"
// when e < min(s + w, end); its elements are sorted stably when it is placed (ps_merge.cuh).
// Every step advances by min(w, end - s) or more.
//
// As for w = 1 (ps_detect.cuh) the partition is found by a scan over transfer functions, now on
// w + 2 states that describe the chain at a boundary b between two groups of positions:
//   F(k), 0 <= k < w : the next run starts at b + k (or at an earlier forced start);
//   A / D             : an ascending / descending run of length >= w is open at b and ends at
//                       its first break at or after b.
// A thread owns 32 positions and reads the pair and forced bits of the next 32 as a window, so
// the end of any run it starts is either decided inside the window or the run is still open
// after it (then its length is >= w and the exit state is A or D).  Exits of the form F(k) only
// arise from extended runs or short natural runs, so k < w.
//
// Functions are kept as tables (exit state, run starts) per entry state; composition walks
// them.  Kernels: reduce (tile tables) -> group (256-tile group tables) -> top (one thread walks
// the groups) -> tile (entry state and run count of every tile) -> emit (threads replay their
// runs from their entry states and write them at their ranks).  No block waits on another.
#pragma once

#include "ps_common.cuh"
#include "ps_debug.cuh"
#include "ps_detect.cuh"
#include "ps_internal.h"

namespace ps {

// Table entries are exit state | run starts << 6: 16 bits for a thread (starts <= 32), 32 bits
// for a tile or a group (starts <= 2^21).

// Next run start after a run starting at window position pos (0 <= pos < 32).  Lw bit q: the
// pair (p0+q-1, p0+q) is in order; Fw bit q: p0+q is a forced start or lies at or past n.
// Returns the next start (64: the natural run is still open after the window) and the run's
// flags: bit 0 = its first pair is strictly descending, bit 1 = extended to the minimal length.
__device__ __forceinline__ int mr_next(uint64_t Lw, uint64_t Fw, int pos, int w, uint32_t& flags) {
  const uint64_t fa = Fw & (~0ull << (pos + 1));
  const int end = fa ? __ffsll((long long)fa) - 1 : 64;
  int e;
  uint32_t desc = 0;
  if (end == pos + 1) {
    e = pos + 1;  // the last position of a segment: a run of one element
  } else {
    const uint32_t asc = (uint32_t)(Lw >> (pos + 1)) & 1u;
    desc = asc ^ 1u;
    const uint64_t brk = ((asc ? ~Lw : Lw) | Fw) & (~0ull << (pos + 2));
    e = brk ? __ffsll((long long)brk) - 1 : 64;
  }
  const int t = min(pos + w, end);
  if (e >= t) {
    flags = desc;
    return e;
  }
  flags = 2u | desc;
  return t;
}

// Exit state of a chain whose last run in this window ends at window position nx >= 32.
__device__ __forceinline__ uint32_t mr_exit(int nx, uint32_t flags, int w) {
  const int k = nx - 32;
  if (k < w) return (uint32_t)k;  // the next start is fixed
  return (flags & 1u) ? (uint32_t)w + 1u : (uint32_t)w;  // a long natural run is still open
}

// First run start in the window for entry state x, or -1 if an open run covers all 32 positions.
__device__ __forceinline__ int mr_first(uint64_t Lw, uint64_t Fw, int w, uint32_t x) {
  if (x < (uint32_t)w) {
    const uint64_t fm = Fw & ((2ull << x) - 1ull);
    return fm ? __ffsll((long long)fm) - 1 : (int)x;
  }
  const uint64_t brk = (((x == (uint32_t)w) ? ~Lw : Lw) | Fw) & 0xffffffffull;
  return brk ? __ffsll((long long)brk) - 1 : -1;
}

// The thread's table entry for entry state x: exit state | run starts << 6.
__device__ __forceinline__ uint32_t mr_walk(uint64_t Lw, uint64_t Fw, int nvalid, int w, uint32_t x) {
  if (nvalid <= 0) return x;
  int pos = mr_first(Lw, Fw, w, x);
  if (pos < 0) return x;
  uint32_t cnt = 0, ex = 0;
  while (pos < nvalid) {
    ++cnt;
    uint32_t fl;
    const int nx = mr_next(Lw, Fw, pos, w, fl);
    if (nx >= 32) {
      ex = mr_exit(nx, fl, w);
      break;
    }
    pos = nx;
  }
  return ex | (cnt << 6);
}

// bit i = OR of the bits [i, i + width) of b
__device__ __forceinline__ uint64_t mr_smear(uint64_t b, int width) {
  if (width <= 0) return 0;
  uint64_t r = b;
  for (int c = 1; c < width;) {
    const int sh = min(c, width - c);
    r |= r >> sh;
    c += sh;
  }
  return r;
}

// A full window (32 positions owned, the next 32 visible).  A start q is "regular" when its run
// is extended to exactly q + w: no forced start in (q, q + w) and a break of its direction in
// [q + 2, q + w).  Bit q of the result (q < 32) marks the other starts.  From a regular start the
// chain steps by w, so a walk jumps over all regular starts of the progression pos, pos + w, ...
// at once.
__device__ __forceinline__ uint32_t mr_irregular(uint64_t Lw, uint64_t Fw, int w) {
  const uint64_t Ba = ~Lw | Fw, Bd = Lw | Fw;        // positions that end an ascending / descending run
  const uint64_t nfa = ~(Fw >> 1);                   // q + 1 is not forced
  const uint64_t longA = (Lw >> 1) & nfa & ~(mr_smear(Ba, w - 2) >> 2);
  const uint64_t longD = ~(Lw >> 1) & nfa & ~(mr_smear(Bd, w - 2) >> 2);
  return (uint32_t)(longA | longD | (mr_smear(Fw, w - 1) >> 1));
}

// Table entry of a full window for a chain whose first start is pos; prog = bits 0, w, 2w, ... < 32.
__device__ __forceinline__ uint32_t mr_walk_fast(uint64_t Lw, uint64_t Fw, uint32_t X, uint32_t prog, int w, int pos) {
  uint32_t cnt = 0;
  for (;;) {
    const uint32_t pr = prog << pos;
    const uint32_t hit = pr & X;
    if (!hit) {
      cnt += (uint32_t)__popc(pr);
      const int last = 31 - __clz(pr);
      return (uint32_t)(last + w - 32) | (cnt << 6);
    }
    const int h = __ffs(hit) - 1;
    cnt += (uint32_t)__popc(pr & ((1u << h) - 1u)) + 1u;
    uint32_t fl;
    const int nx = mr_next(Lw, Fw, h, w, fl);
    if (nx >= 32) return mr_exit(nx, fl, w) | (cnt << 6);
    pos = nx;
  }
}

// The thread's whole table (entries for states 0 .. w + 1) into row[].
__device__ __forceinline__ void mr_table(uint64_t Lw, uint64_t Fw, int nvalid, int w, uint16_t* row) {
  if (nvalid < 32) {
    for (int x = 0; x < w + 2; ++x) row[x] = (uint16_t)mr_walk(Lw, Fw, nvalid, w, (uint32_t)x);
    return;
  }
  const uint64_t Ba = ~Lw | Fw, Bd = Lw | Fw;
  row[w] = (uint16_t)mr_walk(Lw, Fw, nvalid, w, (uint32_t)w);
  row[w + 1] = (uint16_t)mr_walk(Lw, Fw, nvalid, w, (uint32_t)w + 1);
  if ((Ba >> 1) == 0 || (Bd >> 1) == 0) {
    // one ascending (descending) stretch covers positions 1..63: a run started at any q < 32 is
    // still open after the window
    const uint16_t open = (uint16_t)(((Ba >> 1) == 0 ? w : w + 1) | (1 << 6));
    for (int k = 0; k < w; ++k) row[k] = open;
    return;
  }
  const uint32_t X = mr_irregular(Lw, Fw, w);
  uint32_t prog = 0;
  for (int q = 0; q < 32; q += w) prog |= 1u << q;
  const uint32_t F32 = (uint32_t)Fw;
  const int f = F32 ? __ffs(F32) - 1 : 32;  // entry F(k) starts at min(k, f)
  for (int k = 0; k < w; ++k) {
    if (k > f) {
      row[k] = row[f];
    } else {
      row[k] = (uint16_t)mr_walk_fast(Lw, Fw, X, prog, w, k);
    }
  }
}

// The window of one detection thread: its own pair / forced bits (positions 0..32) and those
// of the next thread (positions 32..64); positions at or past n are marked forced (a stop).
__device__ __forceinline__ void mr_window(uint64_t L, uint64_t F, uint64_t Ln, uint64_t Fn, int64_t p0, int64_t n,
                                          uint64_t& Lw, uint64_t& Fw) {
  Lw = (L & 0xffffffffull) | (Ln << 32);
  Fw = (F & 0xffffffffull) | (Fn << 32);
  const int64_t left = n - p0;
  if (left < 64) Fw |= ~0ull << (left > 0 ? (int)left : 0);
}

// Compose one warp's 32 thread tables (shared memory, stride kMrStates) for entry states
// lane and lane + 32; writes the warp table.
__device__ __forceinline__ void mr_warp_compose(const uint16_t (*tab)[kMrStates], uint32_t* wtab, int lane, int S) {
  for (int x = lane; x < S; x += 32) {
    uint32_t st = (uint32_t)x, cnt = 0;
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
      const uint32_t e = PS_IN_RANGE(st, kMrStates) ? tab[i][st] : 0u;
      cnt += e >> 6;
      st = e & 63u;
    }
    wtab[x] = st | (cnt << 6);
  }
}

// Pass 1: each tile's table (kMrStates entries); the pair / forced bits are kept for pass 5.
template <class K>
__global__ void __launch_bounds__(kDetectThreads)
minrun_reduce_kernel(const typename K::T* __restrict__ keys, int64_t n, const int64_t* __restrict__ offsets,
                     int32_t count, int w, uint32_t* __restrict__ tile_tab, uint64_t* __restrict__ thr_L,
                     uint64_t* __restrict__ thr_F) {
  __shared__ uint64_t s_L[kDetectThreads], s_F[kDetectThreads];
  __shared__ uint16_t s_tab[kDetectThreads][kMrStates];
  __shared__ uint32_t s_wtab[kDetectThreads / 32][kMrStates];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int S = w + 2;
  ThreadRuns<K> tr;
  tr.load(keys, n, offsets, count, blockIdx.x, tid);
  const size_t gt = (size_t)blockIdx.x * kDetectThreads + tid;
  thr_L[gt] = tr.L;
  if (offsets != nullptr) thr_F[gt] = tr.F;
  s_L[tid] = tr.L;
  s_F[tid] = tr.F;
  __syncthreads();
  uint64_t Ln = 0, Fn = 0;
  if (tid + 1 < kDetectThreads) {
    Ln = s_L[tid + 1];
    Fn = s_F[tid + 1];
  } else if ((int64_t)(blockIdx.x + 1) * kDetectTile < n) {
    ThreadRuns<K> nx;
    nx.load(keys, n, offsets, count, blockIdx.x + 1, 0);
    Ln = nx.L;
    Fn = nx.F;
  }
  uint64_t Lw, Fw;
  mr_window(tr.L, tr.F, Ln, Fn, tr.p0, n, Lw, Fw);
  mr_table(Lw, Fw, tr.nvalid, w, s_tab[tid]);
  __syncthreads();
  mr_warp_compose(&s_tab[warp * 32], s_wtab[warp], lane, S);
  __syncthreads();
  if (warp == 0) {
    for (int x = lane; x < S; x += 32) {
      uint32_t st = (uint32_t)x, cnt = 0;
      for (int v = 0; v < kDetectThreads / 32; ++v) {
        const uint32_t e = s_wtab[v][st];
        cnt += e >> 6;
        st = e & 63u;
      }
      tile_tab[(size_t)blockIdx.x * kMrStates + x] = st | (cnt << 6);
    }
  }
}

// Pass 2: each group of kMrGroup tiles composed into one table (tables staged in shared memory).
static __global__ void __launch_bounds__(256)
minrun_group_kernel(const uint32_t* __restrict__ tile_tab, int32_t ntiles, int w, uint32_t* __restrict__ grp_tab) {
  __shared__ uint32_t s_t[kMrGroup * kMrStates];
  const int S = w + 2;
  const int32_t t0 = blockIdx.x * kMrGroup, nt = min(kMrGroup, ntiles - t0);
  for (int i = threadIdx.x; i < nt * kMrStates; i += blockDim.x) s_t[i] = tile_tab[(size_t)t0 * kMrStates + i];
  __syncthreads();
  if (threadIdx.x < S) {
    uint32_t st = threadIdx.x, cnt = 0;
    for (int t = 0; t < nt; ++t) {
      const uint32_t e = s_t[t * kMrStates + st];
      cnt += e >> 6;
      st = e & 63u;
    }
    grp_tab[(size_t)blockIdx.x * kMrStates + threadIdx.x] = st | (cnt << 6);
  }
}

// Pass 3 (one CTA): the groups walked from F(0) at position 0, their tables staged in shared
// memory kMrTopChunk groups at a time (one coalesced load per chunk instead of a dependent global
// load per group).  grp_pre[g] = entry state of group g | runs before it << 8; hdr->runs = r and
// S[r] = n, or kDevTooManyRuns when r exceeds kMaxRuns.
constexpr int kMrTopChunk = 64;
static __global__ void __launch_bounds__(256)
minrun_top_kernel(const uint32_t* __restrict__ grp_tab, int32_t ngroups, int64_t n, int64_t run_cap,
                  uint64_t* __restrict__ grp_pre, pos_t* __restrict__ S, PlanHeader* __restrict__ hdr) {
  __shared__ uint32_t s_t[kMrTopChunk * kMrStates];
  uint32_t st = 0;  // meaningful in thread 0
  uint64_t cnt = 0;
  for (int32_t g0 = 0; g0 < ngroups; g0 += kMrTopChunk) {
    const int32_t ng = min(kMrTopChunk, ngroups - g0);
    for (int i = threadIdx.x; i < ng * kMrStates; i += blockDim.x) s_t[i] = grp_tab[(size_t)g0 * kMrStates + i];
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int32_t g = 0; g < ng; ++g) {
        grp_pre[g0 + g] = (uint64_t)st | (cnt << 8);
        const uint32_t e = PS_IN_RANGE(st, kMrStates) ? s_t[g * kMrStates + st] : 0u;
        cnt += e >> 6;
        st = e & 63u;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (cnt > (uint64_t)kMaxRuns) {
      hdr->runs = 0;
      post_status(&hdr->status, nullptr, cnt > (uint64_t)n ? kDevInternal : kDevTooManyRuns);
    } else if (cnt <= (uint64_t)n && cnt + 1 <= (uint64_t)run_cap) {
      hdr->runs = (int32_t)cnt;
      S[cnt] = (pos_t)n;
    } else {
      hdr->runs = 0;
      post_status(&hdr->status, nullptr, kDevInternal);  // a run has at least one element
    }
  }
}

// Pass 4: the entry state and run count of every tile of a group.
static __global__ void __launch_bounds__(256)
minrun_tile_kernel(const uint32_t* __restrict__ tile_tab, int32_t ntiles, const uint64_t* __restrict__ grp_pre,
                   uint64_t* __restrict__ tile_pre) {
  __shared__ uint32_t s_t[kMrGroup * kMrStates];
  const int32_t t0 = blockIdx.x * kMrGroup, nt = min(kMrGroup, ntiles - t0);
  for (int i = threadIdx.x; i < nt * kMrStates; i += blockDim.x) s_t[i] = tile_tab[(size_t)t0 * kMrStates + i];
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t pre = grp_pre[blockIdx.x];
    uint32_t st = (uint32_t)(pre & 63u);
    uint64_t cnt = pre >> 8;
    for (int t = 0; t < nt; ++t) {
      tile_pre[t0 + t] = (uint64_t)st | (cnt << 8);
      const uint32_t e = s_t[t * kMrStates + st];
      cnt += e >> 6;
      st = e & 63u;
    }
  }
}

// Pass 5: every thread rebuilds its table from the saved bits, the block finds each thread's
// entry state and rank, and each thread writes its runs: S[k], flags run_desc[k] (bit 0 first
// pair strictly descending, bit 1 extended) and segments run_seg[k].
template <class K>
__global__ void __launch_bounds__(kDetectThreads)
minrun_emit_kernel(int64_t n, int64_t run_cap, const int64_t* __restrict__ offsets, int32_t count, int w,
                   const uint64_t* __restrict__ tile_pre, const uint64_t* __restrict__ thr_L,
                   const uint64_t* __restrict__ thr_F, size_t nthreads, pos_t* __restrict__ S,
                   uint8_t* __restrict__ run_desc, int32_t* __restrict__ run_seg) {
  __shared__ uint16_t s_tab[kDetectThreads][kMrStates];
  __shared__ uint32_t s_wtab[kDetectThreads / 32][kMrStates];
  __shared__ uint32_t s_entry[kDetectThreads], s_rank[kDetectThreads];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int S_ = w + 2;
  const size_t gt = (size_t)blockIdx.x * kDetectThreads + tid;
  const bool seg = offsets != nullptr;
  ThreadRuns<K> tr;
  tr.restore(n, blockIdx.x, tid, thr_L[gt], seg ? thr_F[gt] : (gt == 0 ? 1ull : 0ull));
  const uint64_t Ln = gt + 1 < nthreads ? thr_L[gt + 1] : 0ull;
  const uint64_t Fn = (seg && gt + 1 < nthreads) ? thr_F[gt + 1] : 0ull;
  uint64_t Lw, Fw;
  mr_window(tr.L, tr.F, Ln, Fn, tr.p0, n, Lw, Fw);
  mr_table(Lw, Fw, tr.nvalid, w, s_tab[tid]);
  __syncthreads();
  mr_warp_compose(&s_tab[warp * 32], s_wtab[warp], lane, S_);
  __syncthreads();
  if (lane == 0) {
    const uint64_t pre = tile_pre[blockIdx.x];
    uint32_t st = (uint32_t)(pre & 63u), cnt = (uint32_t)(pre >> 8);
    for (int v = 0; v < warp; ++v) {
      const uint32_t e = s_wtab[v][st];
      cnt += e >> 6;
      st = e & 63u;
    }
    for (int i = 0; i < 32; ++i) {
      const int t = warp * 32 + i;
      s_entry[t] = st;
      s_rank[t] = cnt;
      const uint32_t e = s_tab[t][st];
      cnt += e >> 6;
      st = e & 63u;
    }
  }
  __syncwarp();
  if (tr.nvalid == 0) return;
  int pos = mr_first(Lw, Fw, w, s_entry[tid]);
  if (pos < 0) return;
  uint32_t idx = s_rank[tid];
  int32_t sg = seg ? segment_of(offsets, count, tr.p0) : 0;
  while (pos < tr.nvalid) {
    uint32_t fl;
    const int nx = mr_next(Lw, Fw, pos, w, fl);
    const int64_t p = tr.p0 + pos;
    if (seg && ((tr.F >> pos) & 1ull)) sg = segment_of(offsets, count, p);
    if ((uint64_t)idx < (uint64_t)run_cap) {  // always true when the tables are consistent
      S[idx] = (pos_t)p;
      run_desc[idx] = (uint8_t)fl;
      if (run_seg) run_seg[idx] = sg;
    }
    ++idx;
    if (nx >= 32) break;
    pos = nx;
  }
}

}  // namespace ps
