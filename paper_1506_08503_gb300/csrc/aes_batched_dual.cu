// aes_batched_dual.cu -- instantiates the two-direction batched kernels with one or two blocks
// per lane per window; the four-block shapes have their own translation unit, so that the two
// compile in parallel.  One CTA per SM: the tables take 128-192 KiB of shared memory.
#include "aes_batched.cuh"

namespace aesgb {

TTDualFn ttable_batched_dual(int threads, int blocks_per_lane) {
  if (threads == 512 && blocks_per_lane == 1) return tt::tt_batched_dual<512, 1>;
  if (threads == 512 && blocks_per_lane == 2) return tt::tt_batched_dual<512, 2>;
  return ttable_batched_dual_wide(threads, blocks_per_lane);
}

}  // namespace aesgb
