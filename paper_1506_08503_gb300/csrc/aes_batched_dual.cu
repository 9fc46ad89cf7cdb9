// aes_batched_dual.cu -- instantiates the two-direction batched kernels with one or two blocks
// per lane per window; the four-block shapes have their own translation unit, so that the two
// compile in parallel.  One CTA per SM: the tables take 128-192 KiB of shared memory.
#include "aes_batched.cuh"

namespace aesgb {

TTDualFn ttable_batched_dual(int threads, int blocks_per_lane, int nre, int nrd) {
  if (nre == 10 || nrd == 10)
    if (TTDualFn f = ttable_batched_dual_r10(threads, blocks_per_lane, nre, nrd)) return f;
  if (threads == 512 && blocks_per_lane == 1) return tt::tt_batched_dual<512, 1>;
  if (threads == 512 && blocks_per_lane == 2) return tt::tt_batched_dual<512, 2>;
  if (threads == 768) return nullptr;  // 24 warps fit the registers only with AES-128 keys
  return ttable_batched_dual_wide(threads, blocks_per_lane);
}

}  // namespace aesgb
