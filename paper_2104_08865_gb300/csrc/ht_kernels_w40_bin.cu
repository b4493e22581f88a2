// Kernel instantiations for HalftimeHash40 under the binary-tree ablation.
#include "ht_badger.cuh"

namespace ht {
const KernelSet &kernels_w40_bin() {
  static const KernelSet ks = make_kernel_set_bin<40>();
  return ks;
}
}  // namespace ht
