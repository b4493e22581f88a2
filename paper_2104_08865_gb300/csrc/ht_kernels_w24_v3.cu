// Kernel instantiations for HalftimeHash24 with 256-bit blocks.
#include "ht_kernels_v3.cuh"

namespace ht {
const KernelSet &kernels_w24_v3() {
  static const KernelSet ks = make_kernel_set_v3<24>();
  return ks;
}
}  // namespace ht
