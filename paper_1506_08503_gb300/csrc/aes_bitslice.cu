// aes_bitslice.cu -- placeholder until the bitsliced kernel lands.
#include "aes_internal.cuh"
namespace aesgb {
aes_status launch_bitslice(int, int, const KeyWords&, const void*, void*, size_t, cudaStream_t, const BSConfig&) {
  return set_error(AES_EINVAL, "bitsliced kernel not built yet");
}
}  // namespace aesgb
