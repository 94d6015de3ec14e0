// wv_acc_m64z.cu -- the 64-bit-path ablation formulations 19..21 (register
// caps of 96 and 168; groups of 9 / 11 under the cap of 128).  The code is
// in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m64z(int arith, int ilp) {
  constexpr int I = 1;
  (void)ilp;
  switch (arith) {
    case 19: return k_accumulate_m64cap<19, 96>;
    case 20: return k_accumulate_m64cap<20, 168>;
    case 21: return k_accumulate_m64cap<21, kM64MaxReg>;
    default: return acc_kernel_m64w(arith, ilp);
  }
}

}  // namespace wv
