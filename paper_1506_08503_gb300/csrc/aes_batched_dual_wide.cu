// aes_batched_dual_wide.cu -- instantiates the two-direction batched kernels with four blocks
// per lane per window.
#include "aes_batched.cuh"

namespace aesgb {

TTDualFn ttable_batched_dual_wide(int threads, int blocks_per_lane) {
  if (threads == 512 && blocks_per_lane == 4) return tt::tt_batched_dual<512, 4>;
  if (threads == 384 && blocks_per_lane == 4) return tt::tt_batched_dual<384, 4>;
  if (threads == 256 && blocks_per_lane == 4) return tt::tt_batched_dual<256, 4>;
  return nullptr;
}

}  // namespace aesgb
