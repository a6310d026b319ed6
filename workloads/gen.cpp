// Seeded synthetic inputs for the powersort library and its oracle.
//
// This module only draws random data: run lengths, run contents and their orientation.  It
// holds none of the sorting method's arithmetic (no run detection, node powers, merge trees or
// merging), so that the GPU path and the CPU oracle can both consume its output without
// sharing any code with each other.
//
// Random numbers: xoshiro256** seeded through SplitMix64 (Blackman & Vigna, "Scrambled
// linear pseudorandom number generators", 2018), written from the published definitions.
// All arithmetic is integer or IEEE double and gives identical streams on x86-64 and aarch64.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct Rng {
  uint64_t s[4];
  static uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  }
  explicit Rng(uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) s[i] = splitmix64(x);
  }
  static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
  uint64_t next() {
    const uint64_t result = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
  }
  // uniform integer in [0, range) by the multiply-high method
  uint64_t below(uint64_t range) { return (uint64_t)(((unsigned __int128)next() * range) >> 64); }
  // uniform in (0, 1]
  double unit_open0() { return (double)((next() >> 11) + 1) * (1.0 / 9007199254740992.0); }
  // uniform in [0, 1)
  double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  bool bernoulli(double p) { return unit() < p; }
};

// Binary32 bit patterns in IEEE totalOrder (used only to make runs sorted).
inline bool f32_bits_less(uint32_t a, uint32_t b) {
  const bool na = a >> 31, nb = b >> 31;
  if (na != nb) return na;
  return na ? a > b : a < b;
}

template <class T, class Less>
void fill_run(T* k, int64_t len, bool desc, Less less) {
  std::sort(k, k + len, less);
  if (desc) std::reverse(k, k + len);
}

// Runs with lengths uniform in [1, max_len], contents uniform 32-bit values sorted (signed or
// unsigned order), each run reversed with probability desc_frac; payload = global index.
void runs32(Rng& g, int64_t n, int64_t max_len, double desc_frac, int is_signed, uint32_t* keys) {
  int64_t pos = 0;
  while (pos < n) {
    int64_t len = 1 + (int64_t)g.below((uint64_t)max_len);
    if (len > n - pos) len = n - pos;
    uint32_t* k = keys + pos;
    for (int64_t i = 0; i < len; ++i) k[i] = (uint32_t)(g.next() >> 32);
    const bool desc = g.bernoulli(desc_frac);
    if (is_signed)
      fill_run((int32_t*)k, len, desc, [](int32_t a, int32_t b) { return a < b; });
    else
      fill_run(k, len, desc, [](uint32_t a, uint32_t b) { return a < b; });
    pos += len;
  }
}

}  // namespace

extern "C" {

// Config family "uniform run lengths": n keys made of runs whose lengths are uniform in
// [1, max_len], each filled with sorted uniform-random 32-bit values (signed order when
// is_signed), a fraction desc_frac of runs reversed.  vals[i] = i (may be NULL).
void psgen_runs32(uint64_t seed, int64_t n, int64_t max_len, double desc_frac, int is_signed,
                  uint32_t* keys, uint32_t* vals) {
  Rng g(seed);
  runs32(g, n, max_len < 1 ? 1 : max_len, desc_frac, is_signed, keys);
  if (vals)
    for (int64_t i = 0; i < n; ++i) vals[i] = (uint32_t)i;
}

// A uniformly random permutation of 0..n-1 (Fisher-Yates), as int32 keys.  vals[i] = i.
void psgen_perm32(uint64_t seed, int64_t n, uint32_t* keys, uint32_t* vals) {
  Rng g(seed);
  for (int64_t i = 0; i < n; ++i) keys[i] = (uint32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    const int64_t j = (int64_t)g.below((uint64_t)(i + 1));
    std::swap(keys[i], keys[j]);
  }
  if (vals)
    for (int64_t i = 0; i < n; ++i) vals[i] = (uint32_t)i;
}

// "Random-runs" inputs of the paper's running-time study: a random permutation of 0..n-1 cut
// into segments of geometric length with mean mean_len (support 1, 2, ...), each segment
// sorted ascending.  vals[i] = i.
void psgen_random_runs32(uint64_t seed, int64_t n, double mean_len, uint32_t* keys, uint32_t* vals) {
  psgen_perm32(seed, n, keys, nullptr);
  Rng g(seed ^ 0x5bd1e9955bd1e995ull);
  const double p = 1.0 / mean_len;
  const double lq = std::log1p(-p);
  int64_t pos = 0;
  while (pos < n) {
    // inverse transform: L = 1 + floor(ln U / ln(1-p)), U in (0, 1]
    double u = g.unit_open0();
    int64_t len = 1 + (int64_t)std::floor(std::log(u) / lq);
    if (len < 1) len = 1;
    if (len > n - pos) len = n - pos;
    std::sort(keys + pos, keys + pos + len);
    pos += len;
  }
  if (vals)
    for (int64_t i = 0; i < n; ++i) vals[i] = (uint32_t)i;
}

// Stability stress: uint64 keys drawn from n_distinct random 64-bit values, run lengths
// min(floor(U^(-1/alpha)), max_len) with U uniform in (0, 1] (Pareto), each run sorted and
// reversed with probability desc_frac.  vals[i] = i.
void psgen_pareto64(uint64_t seed, int64_t n, double alpha, int64_t n_distinct, int64_t max_len,
                    double desc_frac, uint64_t* keys, uint32_t* vals) {
  Rng g(seed);
  std::vector<uint64_t> table((size_t)n_distinct);
  for (auto& t : table) t = g.next();
  int64_t pos = 0;
  while (pos < n) {
    double len_d = std::floor(std::pow(g.unit_open0(), -1.0 / alpha));
    int64_t len = len_d > (double)max_len ? max_len : (int64_t)len_d;
    if (len < 1) len = 1;
    if (len > n - pos) len = n - pos;
    uint64_t* k = keys + pos;
    for (int64_t i = 0; i < len; ++i) k[i] = table[g.below((uint64_t)n_distinct)];
    fill_run(k, len, g.bernoulli(desc_frac), [](uint64_t a, uint64_t b) { return a < b; });
    pos += len;
  }
  if (vals)
    for (int64_t i = 0; i < n; ++i) vals[i] = (uint32_t)i;
}

// Served-request keys: binary32 values (bit patterns) with a fraction special_frac of special
// values (NaNs of either sign with random payloads, +0 and -0), the rest normal values of
// random sign and magnitude in [2^-20, 2^20); run lengths Pareto(alpha) clipped to n; each run
// sorted in IEEE totalOrder and reversed with probability desc_frac.  vals[i] = i.
void psgen_pareto_f32(uint64_t seed, int64_t n, double alpha, double special_frac, double desc_frac,
                      uint32_t* keys, uint32_t* vals) {
  Rng g(seed);
  int64_t pos = 0;
  while (pos < n) {
    double len_d = std::floor(std::pow(g.unit_open0(), -1.0 / alpha));
    int64_t len = len_d > (double)n ? n : (int64_t)len_d;
    if (len < 1) len = 1;
    if (len > n - pos) len = n - pos;
    uint32_t* k = keys + pos;
    for (int64_t i = 0; i < len; ++i) {
      uint32_t bits;
      if (g.bernoulli(special_frac)) {
        const uint64_t c = g.below(4);
        const uint32_t sign = (uint32_t)g.below(2) << 31;
        if (c < 2) {  // NaN: exponent all ones, nonzero mantissa
          bits = sign | 0x7f800000u | (1u + (uint32_t)g.below(0x7fffff));
        } else {      // +0 / -0
          bits = sign;
        }
      } else {
        const double mag = std::ldexp(1.0 + g.unit(), (int)g.below(40) - 20);
        float f = (float)(g.below(2) ? -mag : mag);
        std::memcpy(&bits, &f, 4);
      }
      k[i] = bits;
    }
    fill_run(k, len, g.bernoulli(desc_frac), f32_bits_less);
    pos += len;
  }
  if (vals)
    for (int64_t i = 0; i < n; ++i) vals[i] = (uint32_t)i;
}

// Segment sizes floor(2^U) with U uniform in [lo_exp, hi_exp].
void psgen_segment_sizes(uint64_t seed, int64_t count, double lo_exp, double hi_exp, int64_t* sizes) {
  Rng g(seed);
  for (int64_t k = 0; k < count; ++k) {
    const double u = lo_exp + (hi_exp - lo_exp) * g.unit();
    sizes[k] = (int64_t)std::floor(std::exp2(u));
  }
}

// Segmented inputs: segment k of the given sizes (offsets[k]..offsets[k+1]) is filled like
// psgen_runs32 with max_len = floor(2 * sqrt(size)), each from its own stream (so the result
// does not depend on how the segments are spread over threads).  vals[i] = i.
void psgen_segmented_runs32(uint64_t seed, int64_t count, const int64_t* offsets, double desc_frac,
                            int is_signed, uint32_t* keys, uint32_t* vals) {
  std::atomic<int64_t> next(0);
  auto worker = [&]() {
    for (;;) {
      const int64_t k = next.fetch_add(1);
      if (k >= count) break;
      const int64_t lo = offsets[k], len = offsets[k + 1] - offsets[k];
      if (len <= 0) continue;
      Rng g(seed * 0x9e3779b97f4a7c15ull + (uint64_t)k + 1);
      int64_t max_len = (int64_t)std::floor(2.0 * std::sqrt((double)len));
      runs32(g, len, max_len < 1 ? 1 : max_len, desc_frac, is_signed, keys + lo);
      if (vals)
        for (int64_t i = lo; i < lo + len; ++i) vals[i] = (uint32_t)i;
    }
  };
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  if (nt > 32) nt = 32;
  std::vector<std::thread> th;
  for (unsigned t = 0; t + 1 < nt; ++t) th.emplace_back(worker);
  worker();
  for (auto& t : th) t.join();
}

}  // extern "C"
