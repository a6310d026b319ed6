// Key-dependent kernels for the 4-byte key types (int32, uint32, float32 in totalOrder).
#include "ps_keys.cuh"

namespace ps {
const KeyLaunch kLaunchI32 = Launch<KeyI32>::table();
const KeyLaunch kLaunchU32 = Launch<KeyU32>::table();
const KeyLaunch kLaunchF32 = Launch<KeyF32>::table();
unsigned long long bounds_hits_keys32() { return bounds_hits_here(); }
}  // namespace ps
