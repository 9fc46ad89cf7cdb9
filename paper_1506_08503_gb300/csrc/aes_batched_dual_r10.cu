// aes_batched_dual_r10.cu -- the two-direction batched kernels specialised to AES-128 (every
// message of a direction has 10 rounds): the round loop is fixed and the keys take 11 rows of
// registers instead of 15 plus the last key, which lets 768-thread CTAs (24 warps per SM, at
// most 85 registers a thread) run without spilling.  A direction with no messages counts as
// AES-128.  Own translation unit, so it compiles beside the generic shapes.
#include "aes_batched.cuh"

namespace aesgb {

TTDualFn ttable_batched_dual_r10(int threads, int blocks_per_lane, int nre, int nrd) {
  const bool e = nre == 10, d = nrd == 10;
  if (threads == 512 && blocks_per_lane == 1)
    return e && d ? tt::tt_batched_dual<512, 1, 10, 10> : e ? tt::tt_batched_dual<512, 1, 10, 0>
                                                          : d ? tt::tt_batched_dual<512, 1, 0, 10> : nullptr;
  if (threads == 512 && blocks_per_lane == 2)
    return e && d ? tt::tt_batched_dual<512, 2, 10, 10> : e ? tt::tt_batched_dual<512, 2, 10, 0>
                                                          : d ? tt::tt_batched_dual<512, 2, 0, 10> : nullptr;
  if (threads == 768 && blocks_per_lane == 1) return e && d ? tt::tt_batched_dual<768, 1, 10, 10> : nullptr;
  return nullptr;
}

}  // namespace aesgb
