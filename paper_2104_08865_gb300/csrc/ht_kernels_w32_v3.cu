// Kernel instantiations for HalftimeHash32 with 256-bit blocks.
#include "ht_kernels_v3.cuh"

namespace ht {
const KernelSet &kernels_w32_v3() {
  static const KernelSet ks = make_kernel_set_v3<32>();
  return ks;
}
}  // namespace ht
