// Kernel instantiations for HalftimeHash40 (one translation unit per width
// so the four widths compile in parallel).
#include "ht_range.cuh"

namespace ht {
const KernelSet &kernels_w40() {
  static const KernelSet ks = make_kernel_set<40>();
  return ks;
}
}  // namespace ht
