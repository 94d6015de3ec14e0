// wv_acc_m64y.cu -- the 64-bit-path ablation formulations 16..18 (larger
// groups; form 9 without the register cap).  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m64y(int arith, int ilp) {
  constexpr int I = 1;
  (void)ilp;
  switch (arith) {
    case 16: return k_accumulate<true, I, 16>;
    case 17: return k_accumulate<true, I, 17>;
    case 18: return k_accumulate<true, I, 18>;
    default: return acc_kernel_m64z(arith, ilp);
  }
}

}  // namespace wv
