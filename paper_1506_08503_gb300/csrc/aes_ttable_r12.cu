// aes_ttable_r12.cu -- instantiates the T-table kernels for Nr = 12 (kept in its own translation
// unit so that the fully unrolled kernels compile in parallel).
#include "aes_ttable.cuh"

namespace aesgb {

TTKernelFn ttable_kernel_r12(int dir, int threads, int unroll) {
  return dir == AES_ENCRYPT ? tt::select_config<12, AES_ENCRYPT>(threads, unroll)
                            : tt::select_config<12, AES_DECRYPT>(threads, unroll);
}

}  // namespace aesgb
