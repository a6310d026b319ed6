// Key-dependent kernels for 8-byte keys (uint64).
#include "ps_keys.cuh"

namespace ps {
const KeyLaunch kLaunchU64 = Launch<KeyU64>::table();
unsigned long long bounds_hits_keys64() { return bounds_hits_here(); }
}  // namespace ps
