// aes_ttable_r10.cu -- instantiates the T-table kernels for Nr = 10 (kept in its own translation
// unit so that the fully unrolled kernels compile in parallel).
#include "aes_ttable.cuh"

namespace aesgb {

TTKernelFn ttable_kernel_r10(int dir, int threads, int unroll) {
  return dir == AES_ENCRYPT ? tt::select_config<10, AES_ENCRYPT>(threads, unroll)
                            : tt::select_config<10, AES_DECRYPT>(threads, unroll);
}

}  // namespace aesgb
