// aes_batched_enc.cu -- instantiates the batched T-table kernels for one direction (its own
// translation unit so that the two directions compile in parallel).
#include "aes_batched.cuh"

namespace aesgb {

TTBatchedFn ttable_batched_enc(int threads, int blocks_per_lane) {
  return tt::select_batched<AES_ENCRYPT>(threads, blocks_per_lane);
}

}  // namespace aesgb
