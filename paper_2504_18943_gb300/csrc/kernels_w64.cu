// Kernel instantiations for 64-bit characteristic-sequence words.
#include "lsyn_device.cuh"

namespace lsyn {
template struct Kernels<uint64_t>;
}  // namespace lsyn
