// Kernel instantiations for 32-bit characteristic-sequence words.
#include "lsyn_device.cuh"

namespace lsyn {
template struct Kernels<uint32_t>;
}  // namespace lsyn
