// CPU oracle for powersort and peeksort (Munro & Wild, "Nearly-Optimal Mergesorts:
// Fast, Practical Sorting Methods That Optimally Adapt to Existing Runs", arXiv 1805.04154).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct statement of
// what the GPU path computes.  It is loaded by the tests, by the package's smoke check and
// by the benchmark's CPU-baseline leg, and by nothing else: the GPU library never links,
// loads or calls it, and the two share no code, header, table or helper.
//
// Every function follows a passage of the paper, cited as (section / algorithm / definition /
// theorem).  Plain sequential C++ with 64/128-bit integer arithmetic; no blocking, fusion or
// reordering beyond what the cited passage states.  Where the paper is silent the reading
// taken is stated beside the code.
//
// Parity pins (see tests/test_oracle_*.py): Fig. 1's printed node powers, the merge-cost
// bounds of the Powersort / Peeksort theorems, brute-force optimal merge trees (interval DP),
// std::stable_sort, closed forms for equal run lengths, and the paper's printed average
// merge cost on random-runs inputs (Sec. 5.3).

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------
// Key types.  The paper sorts Java ints (Sec. 5.1); the library it is checked against also
// sorts unsigned 32/64-bit keys and binary32 floats.  For floats the order is the IEEE 754
// totalOrder relation on the bit pattern: every value with the sign bit set precedes every
// value without it; among non-negative patterns a larger pattern is larger, among negative
// patterns a larger pattern is smaller.  (So -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN.)
// ---------------------------------------------------------------------------------------
struct KeyI32 {
  typedef int32_t T;
  static bool less(T a, T b) { return a < b; }
};
struct KeyU32 {
  typedef uint32_t T;
  static bool less(T a, T b) { return a < b; }
};
struct KeyU64 {
  typedef uint64_t T;
  static bool less(T a, T b) { return a < b; }
};
struct KeyF32 {  // binary32 stored as its bit pattern
  typedef uint32_t T;
  static bool less(T a, T b) {
    const bool neg_a = (a >> 31) != 0, neg_b = (b >> 31) != 0;
    if (neg_a != neg_b) return neg_a;  // negative side first
    if (!neg_a) return a < b;          // both non-negative
    return a > b;                      // both negative
  }
};

enum { KT_I32 = 0, KT_U32 = 1, KT_U64 = 2, KT_F32 = 3 };

// a <= b in the key order
template <class K>
inline bool key_le(typename K::T a, typename K::T b) {
  return !K::less(b, a);
}

// ---------------------------------------------------------------------------------------
// Runs (Sec. 2, "Preliminaries"): a run is a maximal weakly increasing region or a strictly
// decreasing region; decreasing runs are reversed right away.  ExtendRunRight (Alg. 2) scans
// greedily from a run start.  Reading: the direction of a run is fixed by its own first pair,
// so the element where the direction turns belongs to the earlier run, and a run of length 1
// can only be the last element of the array.
// Returns the exclusive end of the run that starts at s (0-based, half-open), and whether it
// is strictly decreasing.
// ---------------------------------------------------------------------------------------
template <class K>
int64_t extend_run_right(const typename K::T* a, int64_t s, int64_t n, bool* descending) {
  *descending = false;
  if (s + 1 >= n) return n;  // last element alone
  int64_t e = s + 1;         // a[s..e] is the run so far (inclusive e)
  if (key_le<K>(a[s], a[s + 1])) {
    while (e + 1 < n && key_le<K>(a[e], a[e + 1])) ++e;
  } else {
    *descending = true;
    while (e + 1 < n && K::less(a[e + 1], a[e])) ++e;
  }
  return e + 1;
}

template <class K>
void reverse_range(typename K::T* a, uint32_t* v, int64_t lo, int64_t hi) {
  std::reverse(a + lo, a + hi);
  if (v) std::reverse(v + lo, v + hi);
}

// ---------------------------------------------------------------------------------------
// Node power (Definition "Node Power", Sec. 3.2; procedure NodePower of Alg. 2).
// Runs A = [s1, e1) and B = [e1, e2) inside an array of length n (0-based, half-open).
// The normalised midpoints are a = (s1 + e1) / (2n) and b = (e1 + e2) / (2n); the power is
// the least l >= 0 with floor(a * 2^l) < floor(b * 2^l), i.e. the index of the first
// fractional bit in which a and b differ.  Exact rational arithmetic in 128-bit integers.
// ---------------------------------------------------------------------------------------
int node_power_exact(int64_t s1, int64_t e1, int64_t e2, int64_t n) {
  typedef unsigned __int128 u128;
  const u128 two_n = (u128)(2 * n);
  const u128 l2 = (u128)(s1 + e1), r2 = (u128)(e1 + e2);
  for (int l = 0; l < 126; ++l) {
    if ((l2 << l) / two_n < (r2 << l) / two_n) return l;
  }
  return -1;  // unreachable for a < b
}

// The same quantity from the first 31 fractional bits of a and b (the paper's implementation
// note in Appendix B computes the power this way for int-sized arrays).  Valid for n < 2^31:
// then b - a >= 1/n > 2^-31, so the first difference lies within those bits.
int node_power_bits(int64_t s1, int64_t e1, int64_t e2, int64_t n) {
  const uint64_t two_n = (uint64_t)(2 * n);
  const uint64_t fa = ((uint64_t)(s1 + e1) << 31) / two_n;  // floor(a * 2^31)
  const uint64_t fb = ((uint64_t)(e1 + e2) << 31) / two_n;  // floor(b * 2^31)
  const uint64_t diff = fa ^ fb;
  int l = 1;  // fractional bit 1 is bit 30 of the 31-bit numbers
  for (int bit = 30; bit >= 0; --bit, ++l) {
    if ((diff >> bit) & 1u) return l;
  }
  return -1;
}

// ---------------------------------------------------------------------------------------
// Stable merge of the adjacent sorted ranges [lo, mid) and [mid, hi) (the merge primitive of
// Appendix B, "Merging"): the left run is copied out, then the two are merged into [lo, hi);
// on equal keys the element of the left run is taken first, which makes the merge stable.
// ---------------------------------------------------------------------------------------
template <class K>
void merge_runs(typename K::T* a, uint32_t* v, int64_t lo, int64_t mid, int64_t hi,
                std::vector<typename K::T>& ka, std::vector<uint32_t>& va) {
  const int64_t nl = mid - lo;
  ka.assign(a + lo, a + mid);
  if (v) va.assign(v + lo, v + mid);
  int64_t i = 0, j = mid, k = lo;
  while (i < nl && j < hi) {
    if (key_le<K>(ka[i], a[j])) {  // left wins ties
      a[k] = ka[i];
      if (v) v[k] = va[i];
      ++i;
    } else {
      a[k] = a[j];
      if (v) v[k] = v[j];
      ++j;
    }
    ++k;
  }
  while (i < nl) {
    a[k] = ka[i];
    if (v) v[k] = va[i];
    ++i;
    ++k;
  }
  // the remainder of the right run is already in place
}

// Straight insertion sort of [lo, hi) whose prefix [lo, lo + sorted) is sorted (Appendix B,
// "Insertionsort to extend runs").  Only used by the minimal-run-length variant of Sec. 5.1.
template <class K>
void insertion_sort(typename K::T* a, uint32_t* v, int64_t lo, int64_t hi, int64_t sorted) {
  for (int64_t i = lo + sorted; i < hi; ++i) {
    typename K::T x = a[i];
    uint32_t xv = v ? v[i] : 0;
    int64_t j = i;
    while (j > lo && K::less(x, a[j - 1])) {
      a[j] = a[j - 1];
      if (v) v[j] = v[j - 1];
      --j;
    }
    a[j] = x;
    if (v) v[j] = xv;
  }
}

// ---------------------------------------------------------------------------------------
// PowerSort (Alg. 2) on data.  Run detection with ExtendRunRight, NodePower per boundary,
// and the stack loop that pops while the power on top of the stack exceeds the new power.
// The merge tree is recorded: internal node j is the boundary between run j-1 and run j
// (1 <= j <= r-1); leaf i is run i.
// ---------------------------------------------------------------------------------------
struct Trace {
  int64_t* starts;       // [r+1] run starts, starts[r] = n
  uint8_t* desc;         // [r]   run was strictly decreasing (and got reversed)
  int32_t* power;        // [r+1] power of boundary j; power[0] = power[r] = 0
  int64_t* node_parent;  // [r+1] parent boundary of boundary j, -1 for the root (index 0, r unused)
  int64_t* leaf_parent;  // [r]   parent boundary of leaf i, -1 if the array is one run
  int32_t* leaf_depth;   // [r]   number of edges from leaf i to the root
  int64_t* merges;       // [3*(r-1)] (lo, mid, hi) in execution order
  uint64_t cost;         // merge cost M = sum over merges of (hi - lo)
  int64_t n_merges;
};

struct StackItem {
  int64_t lo, hi;     // element range
  int64_t first_run;  // index of the leftmost run it covers
  int64_t id;         // >= 1: boundary (internal node); < 0: leaf -(i+1)
  int32_t power;      // power pushed with it (Alg. 2 keeps a parallel stack P)
};

template <class K>
int64_t powersort_impl(typename K::T* a, uint32_t* v, int64_t n, int64_t min_run, Trace* tr) {
  tr->cost = 0;
  tr->n_merges = 0;
  if (n <= 0) return 0;
  std::vector<typename K::T> ka;
  std::vector<uint32_t> va;
  std::vector<StackItem> stack;  // X and P of Alg. 2 in one stack
  int64_t r = 0;

  auto next_run = [&](int64_t s) -> int64_t {
    bool d = false;
    int64_t e = extend_run_right<K>(a, s, n, &d);
    if (d) reverse_range<K>(a, v, s, e);
    if (min_run > 1 && e - s < min_run) {  // Sec. 5.1 variant: extend short runs to w
      const int64_t e2 = std::min(n, s + min_run);
      insertion_sort<K>(a, v, s, e2, e - s);
      e = e2;
    }
    tr->starts[r] = s;
    tr->desc[r] = d ? 1 : 0;
    ++r;
    return e;
  };
  auto set_parent = [&](int64_t id, int64_t parent) {
    if (id < 0)
      tr->leaf_parent[-id - 1] = parent;
    else
      tr->node_parent[id] = parent;
  };
  auto do_merge = [&](const StackItem& left, const StackItem& right) -> StackItem {
    // the boundary between the two is the first run of the right operand
    const int64_t node = right.first_run;
    merge_runs<K>(a, v, left.lo, left.hi, right.hi, ka, va);
    tr->merges[3 * tr->n_merges + 0] = left.lo;
    tr->merges[3 * tr->n_merges + 1] = left.hi;
    tr->merges[3 * tr->n_merges + 2] = right.hi;
    tr->n_merges++;
    tr->cost += (uint64_t)(right.hi - left.lo);
    set_parent(left.id, node);
    set_parent(right.id, node);
    StackItem m;
    m.lo = left.lo;
    m.hi = right.hi;
    m.first_run = left.first_run;
    m.id = node;
    m.power = 0;
    return m;
  };

  StackItem cur;
  cur.lo = 0;
  cur.first_run = 0;
  cur.id = -1;
  cur.hi = next_run(0);
  cur.power = 0;
  while (cur.hi < n) {
    StackItem nxt;
    nxt.lo = cur.hi;
    nxt.first_run = r;
    nxt.id = -(r + 1);
    nxt.hi = next_run(nxt.lo);
    nxt.power = 0;
    // power of the boundary between the current run (ending at nxt.lo) and the next one;
    // the left operand of NodePower is the run just detected before, not the merged range.
    const int64_t prev_start = tr->starts[r - 2];
    const int p = node_power_exact(prev_start, nxt.lo, nxt.hi, n);
    tr->power[r - 1] = p;
    while (!stack.empty() && stack.back().power > p) {
      StackItem left = stack.back();
      stack.pop_back();
      cur = do_merge(left, cur);
    }
    cur.power = p;
    stack.push_back(cur);
    cur = nxt;
  }
  while (!stack.empty()) {
    StackItem left = stack.back();
    stack.pop_back();
    cur = do_merge(left, cur);
  }
  tr->starts[r] = n;
  tr->power[0] = 0;
  tr->power[r] = 0;
  tr->node_parent[0] = -1;
  tr->node_parent[r] = -1;
  set_parent(cur.id, -1);
  // Depths: walk the merges backwards (a parent is merged after both its children).
  std::vector<int32_t> node_depth(r + 1, 0);
  for (int64_t m = tr->n_merges - 1; m >= 0; --m) {
    // node of merge m is the boundary at position mid
    const int64_t mid = tr->merges[3 * m + 1];
    const int64_t node = std::lower_bound(tr->starts, tr->starts + r, mid) - tr->starts;
    const int64_t par = tr->node_parent[node];
    node_depth[node] = par < 0 ? 0 : node_depth[par] + 1;
  }
  for (int64_t i = 0; i < r; ++i) {
    const int64_t par = tr->leaf_parent[i];
    tr->leaf_depth[i] = par < 0 ? 0 : node_depth[par] + 1;
  }
  return r;
}

// PowerSort's merge tree and cost from run lengths alone (Alg. 2 uses the data only to find
// the runs, so with the runs given the stack loop can be simulated exactly).
uint64_t powersort_cost_from_lengths(const int64_t* len, int64_t r, int32_t* depth_out,
                                     int32_t* power_out) {
  if (r <= 0) return 0;
  std::vector<int64_t> st(r + 1, 0);
  for (int64_t i = 0; i < r; ++i) st[i + 1] = st[i] + len[i];
  const int64_t n = st[r];
  struct It {
    int64_t first_run, last_run;  // runs [first_run, last_run)
    int32_t power;
  };
  std::vector<It> stack;
  std::vector<int32_t> depth(r, 0);
  uint64_t cost = 0;
  auto merge = [&](const It& l, const It& rr) -> It {
    cost += (uint64_t)(st[rr.last_run] - st[l.first_run]);
    for (int64_t i = l.first_run; i < rr.last_run; ++i) depth[i] += 1;
    It m;
    m.first_run = l.first_run;
    m.last_run = rr.last_run;
    m.power = 0;
    return m;
  };
  if (power_out) power_out[0] = power_out[r] = 0;
  It cur{0, 1, 0};
  for (int64_t j = 1; j < r; ++j) {
    const int p = node_power_exact(st[j - 1], st[j], st[j + 1], n);
    if (power_out) power_out[j] = p;
    while (!stack.empty() && stack.back().power > p) {
      It l = stack.back();
      stack.pop_back();
      cur = merge(l, cur);
    }
    cur.power = p;
    stack.push_back(cur);
    cur = It{j, j + 1, 0};
  }
  while (!stack.empty()) {
    It l = stack.back();
    stack.pop_back();
    cur = merge(l, cur);
  }
  if (depth_out)
    for (int64_t i = 0; i < r; ++i) depth_out[i] = depth[i];
  return cost;
}

// ---------------------------------------------------------------------------------------
// PeekSort (Alg. 1).  Inclusive indices as in the paper.  Reading: Alg. 1 passes the prefix
// run A[l..e] and suffix run A[s..r] down the recursion, sometimes as one-element placeholders
// (e+1, s-1, i-1) of a longer run, and bounds the middle-run scans by l and r.  Taken
// literally, a placeholder inside a run turns that run into two and costs an extra merge, and
// a middle scan that crosses a real prefix run can reverse part of it.  The proof of the
// Peeksort theorem states the intended result: the recursion builds Mehlhorn's Method 1 tree
// on the run lengths L_1..L_r.  So here e and s are always the true ends of the runs that
// contain l and r, and the run containing the middle position m is the run of the partition
// that contains m; runs are found left to right with ExtendRunRight (Sec. 2 convention) and
// decreasing runs are reversed first.  The case analysis of Alg. 1 is then unchanged.
// ---------------------------------------------------------------------------------------
struct PeekTree {
  std::vector<int64_t> st;     // run starts, st[r] = n
  std::vector<int32_t> depth;  // leaf depths
  std::vector<int64_t> merges; // (lo, mid, hi) triples, half-open, in execution order
  uint64_t cost = 0;
  int64_t run_of(int64_t pos) const {  // index of the run containing pos
    return (int64_t)(std::upper_bound(st.begin(), st.end(), pos) - st.begin()) - 1;
  }
  void merge(int64_t l, int64_t mid, int64_t r) {  // A[l..mid-1] with A[mid..r]
    cost += (uint64_t)(r - l + 1);
    merges.push_back(l);
    merges.push_back(mid);
    merges.push_back(r + 1);
    for (int64_t k = run_of(l); k + 1 < (int64_t)st.size() && st[k] <= r; ++k) depth[k] += 1;
  }
  void sort(int64_t l, int64_t r) {  // [l..r] is a union of whole runs
    const int64_t e = st[run_of(l) + 1] - 1;  // prefix run A[l..e]
    const int64_t s = st[run_of(r)];          // suffix run A[s..r]
    if (e == r || s == l) return;
    const int64_t m = l + (r - l) / 2;
    if (m <= e) {
      sort(e + 1, r);
      merge(l, e + 1, r);
    } else if (m >= s) {
      sort(l, s - 1);
      merge(l, s, r);
    } else {
      const int64_t k = run_of(m);
      const int64_t i = st[k], j = st[k + 1] - 1;  // the run A[i..j] containing m
      if (m - i < j - m) {
        sort(l, i - 1);
        sort(i, r);
        merge(l, i, r);
      } else {
        sort(l, j);
        sort(j + 1, r);
        merge(l, j + 1, r);
      }
    }
  }
  void run(int64_t r) {
    depth.assign(r, 0);
    const int64_t n = st[r];
    if (r >= 2) sort(0, n - 1);
  }
};

template <class K>
uint64_t peeksort_impl(typename K::T* a, uint32_t* v, int64_t n, int64_t* n_merges) {
  PeekTree t;
  int64_t s = 0;
  while (s < n) {
    bool d = false;
    const int64_t e = extend_run_right<K>(a, s, n, &d);
    if (d) reverse_range<K>(a, v, s, e);
    t.st.push_back(s);
    s = e;
  }
  t.st.push_back(n);
  const int64_t r = (int64_t)t.st.size() - 1;
  t.run(r);
  std::vector<typename K::T> ka;
  std::vector<uint32_t> va;
  for (size_t q = 0; q < t.merges.size(); q += 3)
    merge_runs<K>(a, v, t.merges[q], t.merges[q + 1], t.merges[q + 2], ka, va);
  if (n_merges) *n_merges = (int64_t)t.merges.size() / 3;
  return t.cost;
}

template <class K>
void stable_sort_impl(typename K::T* a, uint32_t* v, int64_t n) {
  std::vector<int64_t> idx(n);
  for (int64_t i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return K::less(a[x], a[y]); });
  std::vector<typename K::T> ka(n);
  std::vector<uint32_t> vb;
  for (int64_t i = 0; i < n; ++i) ka[i] = a[idx[i]];
  if (v) {
    vb.resize(n);
    for (int64_t i = 0; i < n; ++i) vb[i] = v[idx[i]];
  }
  std::copy(ka.begin(), ka.end(), a);
  if (v) std::copy(vb.begin(), vb.end(), v);
}

template <class K>
int64_t detect_impl(const typename K::T* a, int64_t n, int64_t* starts, uint8_t* desc) {
  int64_t r = 0, s = 0;
  while (s < n) {
    bool d = false;
    const int64_t e = extend_run_right<K>(a, s, n, &d);
    starts[r] = s;
    desc[r] = d ? 1 : 0;
    ++r;
    s = e;
  }
  starts[r] = n;
  return r;
}

}  // namespace

// =======================================================================================
// C ABI (loaded with ctypes by the tests and the benchmark's CPU baseline)
// =======================================================================================
extern "C" {

// Greedy run partition (Sec. 2; ExtendRunRight of Alg. 2) without modifying the keys.
// starts needs n+1 entries, desc n entries.  Returns r.
int64_t ps_oracle_detect_runs(int kt, const void* keys, int64_t n, int64_t* starts, uint8_t* desc) {
  if (n <= 0) {
    starts[0] = 0;
    return 0;
  }
  switch (kt) {
    case KT_I32: return detect_impl<KeyI32>((const int32_t*)keys, n, starts, desc);
    case KT_U32: return detect_impl<KeyU32>((const uint32_t*)keys, n, starts, desc);
    case KT_U64: return detect_impl<KeyU64>((const uint64_t*)keys, n, starts, desc);
    case KT_F32: return detect_impl<KeyF32>((const uint32_t*)keys, n, starts, desc);
  }
  return -1;
}

// Definition "Node Power": runs [s1, e1) and [e1, e2) of an array of length n.
int ps_oracle_node_power(int64_t s1, int64_t e1, int64_t e2, int64_t n) {
  return node_power_exact(s1, e1, e2, n);
}
int ps_oracle_node_power_bits(int64_t s1, int64_t e1, int64_t e2, int64_t n) {
  return node_power_bits(s1, e1, e2, n);
}

// Alg. 2 on (keys, vals) in place; vals may be NULL.  All trace arrays need n+1 entries
// (merges 3n).  Returns r; *cost receives M.
int64_t ps_oracle_powersort(int kt, void* keys, uint32_t* vals, int64_t n, int64_t min_run,
                            int64_t* starts, uint8_t* desc, int32_t* power, int64_t* node_parent,
                            int64_t* leaf_parent, int32_t* leaf_depth, int64_t* merges,
                            uint64_t* cost) {
  Trace tr;
  tr.starts = starts;
  tr.desc = desc;
  tr.power = power;
  tr.node_parent = node_parent;
  tr.leaf_parent = leaf_parent;
  tr.leaf_depth = leaf_depth;
  tr.merges = merges;
  int64_t r = -1;
  if (n <= 0) {
    starts[0] = 0;
    *cost = 0;
    return 0;
  }
  switch (kt) {
    case KT_I32: r = powersort_impl<KeyI32>((int32_t*)keys, vals, n, min_run, &tr); break;
    case KT_U32: r = powersort_impl<KeyU32>((uint32_t*)keys, vals, n, min_run, &tr); break;
    case KT_U64: r = powersort_impl<KeyU64>((uint64_t*)keys, vals, n, min_run, &tr); break;
    case KT_F32: r = powersort_impl<KeyF32>((uint32_t*)keys, vals, n, min_run, &tr); break;
  }
  *cost = tr.cost;
  return r;
}

// Segmented powersort: every segment [offsets[k], offsets[k+1]) is sorted on its own by Alg. 2
// (positions and n of the Definition are segment-relative).  Per-run outputs are concatenated
// over the segments: starts are global positions (starts[R] = offsets[count]); power holds the
// segment-relative powers with 0 on the boundary between two segments; leaf_depth per run.
// Arrays: starts/power need N+1 entries, desc/leaf_depth N entries (N = offsets[count]).
// Returns the total number of runs R; *cost receives the summed merge cost.
int64_t ps_oracle_sort_segmented(int kt, void* keys, uint32_t* vals, const int64_t* offsets,
                                 int64_t count, int64_t* starts, uint8_t* desc, int32_t* power,
                                 int32_t* leaf_depth, uint64_t* cost) {
  const int64_t N = offsets[count] - offsets[0];
  std::vector<int64_t> st(N + 2), np(N + 2), lp(N + 2), mg(3 * (N + 2));
  std::vector<uint8_t> ds(N + 2);
  std::vector<int32_t> pw(N + 2), ld(N + 2);
  const size_t ksz = (kt == KT_U64) ? 8 : 4;
  int64_t R = 0;
  uint64_t total = 0;
  power[0] = 0;
  for (int64_t k = 0; k < count; ++k) {
    const int64_t lo = offsets[k], len = offsets[k + 1] - offsets[k];
    if (len <= 0) continue;
    uint64_t c = 0;
    char* kb = (char*)keys + (size_t)lo * ksz;
    uint32_t* vb = vals ? vals + lo : nullptr;
    const int64_t r = ps_oracle_powersort(kt, kb, vb, len, 1, st.data(), ds.data(), pw.data(),
                                          np.data(), lp.data(), ld.data(), mg.data(), &c);
    for (int64_t i = 0; i < r; ++i) {
      starts[R + i] = lo + st[i];
      desc[R + i] = ds[i];
      leaf_depth[R + i] = ld[i];
      power[R + i] = (i == 0) ? 0 : pw[i];
    }
    R += r;
    total += c;
  }
  starts[R] = offsets[count];
  power[R] = 0;
  *cost = total;
  return R;
}

// Cartesian tree of the powers (Corollary "Cartesian tree"): the parent of boundary j is the
// nearer of its nearest smaller neighbours on the left and on the right, i.e. the one with the
// larger power; power[0] = power[r] = 0 act as sentinels.  Sequential stack algorithm.
// parent[j] for 1 <= j <= r-1 (-1 for the root).  Returns 0, or -1 if two candidate parents
// tie (which the path-power lemma rules out).
int ps_oracle_cartesian_parent(const int32_t* power, int64_t r, int64_t* parent) {
  std::vector<int64_t> left(r + 1, 0), right(r + 1, r), st;
  for (int64_t j = 0; j <= r; ++j) {
    while (!st.empty() && power[st.back()] >= power[j]) st.pop_back();
    left[j] = st.empty() ? 0 : st.back();
    st.push_back(j);
  }
  st.clear();
  for (int64_t j = r; j >= 0; --j) {
    while (!st.empty() && power[st.back()] >= power[j]) st.pop_back();
    right[j] = st.empty() ? r : st.back();
    st.push_back(j);
  }
  int rc = 0;
  for (int64_t j = 1; j < r; ++j) {
    const int64_t L = left[j], R = right[j];
    const bool l_real = L >= 1 && power[L] >= 1, r_real = R <= r - 1 && power[R] >= 1;
    if (!l_real && !r_real) {
      parent[j] = -1;
    } else if (l_real && r_real) {
      if (power[L] == power[R]) rc = -1;
      parent[j] = power[L] > power[R] ? L : R;
    } else {
      parent[j] = l_real ? L : R;
    }
  }
  return rc;
}

// Alg. 2 simulated on run lengths: merge cost, leaf depths (r entries) and powers (r+1).
uint64_t ps_oracle_powersort_cost(const int64_t* lengths, int64_t r, int32_t* depth_out,
                                  int32_t* power_out) {
  return powersort_cost_from_lengths(lengths, r, depth_out, power_out);
}

// Alg. 1 on data in place; returns its merge cost, *n_merges the number of merges.
uint64_t ps_oracle_peeksort(int kt, void* keys, uint32_t* vals, int64_t n, int64_t* n_merges) {
  uint64_t c = 0;
  int64_t m = 0;
  if (n >= 2) {
    switch (kt) {
      case KT_I32: c = peeksort_impl<KeyI32>((int32_t*)keys, vals, n, &m); break;
      case KT_U32: c = peeksort_impl<KeyU32>((uint32_t*)keys, vals, n, &m); break;
      case KT_U64: c = peeksort_impl<KeyU64>((uint64_t*)keys, vals, n, &m); break;
      case KT_F32: c = peeksort_impl<KeyF32>((uint32_t*)keys, vals, n, &m); break;
    }
  }
  if (n_merges) *n_merges = m;
  return c;
}

// Alg. 1 on run lengths alone: merge cost and leaf depths (r entries).
uint64_t ps_oracle_peeksort_cost(const int64_t* lengths, int64_t r, int32_t* depth_out) {
  PeekTree t;
  t.st.assign(r + 1, 0);
  for (int64_t i = 0; i < r; ++i) t.st[i + 1] = t.st[i] + lengths[i];
  t.run(r);
  if (depth_out)
    for (int64_t i = 0; i < r; ++i) depth_out[i] = t.depth[i];
  return t.cost;
}

// Optimal merge cost over all binary merge trees of the runs in their order (Sec. 2.3: the
// optimal alphabetic tree for leaf weights L_i), by the interval recurrence
// OPT[i][j] = sum(L[i..j]) + min_k OPT[i][k] + OPT[k+1][j].  O(r^3); small r only.
uint64_t ps_oracle_opt_cost(const int64_t* lengths, int64_t r) {
  if (r <= 1) return 0;
  std::vector<uint64_t> pre(r + 1, 0);
  for (int64_t i = 0; i < r; ++i) pre[i + 1] = pre[i] + (uint64_t)lengths[i];
  std::vector<uint64_t> opt((size_t)r * r, 0);
  for (int64_t span = 1; span < r; ++span) {
    for (int64_t i = 0; i + span < r; ++i) {
      const int64_t j = i + span;
      uint64_t best = ~(uint64_t)0;
      for (int64_t k = i; k < j; ++k) {
        const uint64_t c = opt[(size_t)i * r + k] + opt[(size_t)(k + 1) * r + j];
        if (c < best) best = c;
      }
      opt[(size_t)i * r + j] = best + (pre[j + 1] - pre[i]);
    }
  }
  return opt[(size_t)0 * r + (r - 1)];
}

// The plain definition of the result: the stable sort of (key, payload) pairs by key
// (std::stable_sort with the key order above).  vals may be NULL.
void ps_oracle_stable_sort(int kt, void* keys, uint32_t* vals, int64_t n) {
  if (n <= 1) return;
  switch (kt) {
    case KT_I32: stable_sort_impl<KeyI32>((int32_t*)keys, vals, n); break;
    case KT_U32: stable_sort_impl<KeyU32>((uint32_t*)keys, vals, n); break;
    case KT_U64: stable_sort_impl<KeyU64>((uint64_t*)keys, vals, n); break;
    case KT_F32: stable_sort_impl<KeyF32>((uint32_t*)keys, vals, n); break;
  }
}

}  // extern "C"
