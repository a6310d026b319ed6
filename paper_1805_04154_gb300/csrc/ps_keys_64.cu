// Key-dependent kernels for 8-byte keys (uint64).
#include "ps_keys.cuh"

namespace ps {
const KeyLaunch kLaunchU64 = Launch<KeyU64>::table();
}  // namespace ps
