// ht_kernels_v3.cuh -- kernel table of the 256-bit-block variant (B = 4 words
// per block, the block size the paper labels "v3", Section 6.3): the
// warp-chunk kernels with 64-execution sub-chunks, one per half-warp, and the
// multi-block batch planner.  One translation unit per width includes it.
#pragma once

#include "ht_stream.cuh"

namespace ht {

template <int W>
inline KernelSet make_kernel_set_v3() {
  constexpr int B = 4, L = 2;
  KernelSet ks = {};
  ks.single_aligned[L - 1] = (const void *)hash_kernel<W, L, true, true, false, B>;
  ks.single_unaligned[L - 1] = (const void *)hash_kernel<W, L, true, false, false, B>;
  ks.batch[L - 1] = (const void *)hash_kernel<W, L, false, true, false, B>;
  ks.batch_unaligned[L - 1] = (const void *)hash_kernel<W, L, false, false, false, B>;
  ks.batch_map[L - 1] = (const void *)hash_kernel<W, L, false, true, false, B, true>;
  ks.batch_unaligned_map[L - 1] = (const void *)hash_kernel<W, L, false, false, false, B, true>;
  ks.plan_tiles[L] = (const void *)plan_tiles_kernel<W, L, B>;
  ks.plan_totals = (const void *)plan_totals_kernel<W>;
  ks.plan_items = (const void *)plan_items_kernel<W>;
  ks.plan_write[L] = (const void *)plan_write_kernel<W, L, B>;
  ks.wait_probe = (const void *)wait_probe_kernel<W>;
  ks.exec_bytes = Dims<W, B>::exec_bytes;
  ks.k = Spec<W>::k;
  ks.n_seed = Dims<W, B>::n_seed;
  ks.off_T = Dims<W, B>::off_T;
  ks.off_F = Dims<W, B>::off_F;
  ks.off_R = Dims<W, B>::off_R;
  ks.ew = Dims<W, B>::ew;
  ks.lanes = B;
  return ks;
}

}  // namespace ht
