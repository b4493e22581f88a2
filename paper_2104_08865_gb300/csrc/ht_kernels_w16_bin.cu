// Kernel instantiations for HalftimeHash16 under the binary-tree ablation.
#include "ht_badger.cuh"

namespace ht {
const KernelSet &kernels_w16_bin() {
  static const KernelSet ks = make_kernel_set_bin<16>();
  return ks;
}
}  // namespace ht
