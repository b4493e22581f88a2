// Kernel instantiations for HalftimeHash16 with 256-bit blocks.
#include "ht_kernels_v3.cuh"

namespace ht {
const KernelSet &kernels_w16_v3() {
  static const KernelSet ks = make_kernel_set_v3<16>();
  return ks;
}
}  // namespace ht
