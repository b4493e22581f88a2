// Kernel instantiations for HalftimeHash32 (one translation unit per width
// so the four widths compile in parallel).
#include "ht_range.cuh"

namespace ht {
const KernelSet &kernels_w32() {
  static const KernelSet ks = make_kernel_set<32>();
  return ks;
}
}  // namespace ht
