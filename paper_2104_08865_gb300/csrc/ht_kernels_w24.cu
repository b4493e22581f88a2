// Kernel instantiations for HalftimeHash24 (one translation unit per width
// so the four widths compile in parallel).
#include "ht_range.cuh"

namespace ht {
const KernelSet &kernels_w24() {
  static const KernelSet ks = make_kernel_set<24>();
  return ks;
}
}  // namespace ht
