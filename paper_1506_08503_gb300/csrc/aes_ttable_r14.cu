// aes_ttable_r14.cu -- instantiates the T-table kernels for Nr = 14 (kept in its own translation
// unit so that the fully unrolled kernels compile in parallel).
#include "aes_ttable.cuh"

namespace aesgb {

TTKernelFn ttable_kernel_r14(int dir, int threads, int unroll) {
  return dir == AES_ENCRYPT ? tt::select_config<14, AES_ENCRYPT>(threads, unroll)
                            : tt::select_config<14, AES_DECRYPT>(threads, unroll);
}

}  // namespace aesgb
