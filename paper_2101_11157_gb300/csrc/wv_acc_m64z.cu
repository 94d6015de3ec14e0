// wv_acc_m64z.cu -- the 64-bit-path ablation formulation 21 (groups of
// 9 / 11 under the register cap of 128).  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m64z(int arith, int ilp) {
  constexpr int I = 1;
  (void)ilp;
  switch (arith) {
    case 21: return k_accumulate_m64cap<21, kM64MaxReg>;
    default: return acc_kernel_m64w(arith, ilp);
  }
}

}  // namespace wv
