// Kernel instantiations for HalftimeHash16 (one translation unit per width
// so the four widths compile in parallel).
#include "ht_range.cuh"

namespace ht {
const KernelSet &kernels_w16() {
  static const KernelSet ks = make_kernel_set<16>();
  return ks;
}
}  // namespace ht
