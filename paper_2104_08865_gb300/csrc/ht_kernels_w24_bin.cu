// Kernel instantiations for HalftimeHash24 under the binary-tree ablation.
#include "ht_badger.cuh"

namespace ht {
const KernelSet &kernels_w24_bin() {
  static const KernelSet ks = make_kernel_set_bin<24>();
  return ks;
}
}  // namespace ht
