// Kernel instantiations for HalftimeHash32 under the binary-tree ablation.
#include "ht_badger.cuh"

namespace ht {
const KernelSet &kernels_w32_bin() {
  static const KernelSet ks = make_kernel_set_bin<32>();
  return ks;
}
}  // namespace ht
