// wv_acc_m64w.cu -- the 64-bit instantiations of the paper's arithmetic (23)
// and of the general index (24).  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m64w(int arith, int ilp) {
  constexpr int I = 1;
  (void)ilp;
  switch (arith) {
    case 23: return k_accumulate<true, I, 23>;  // the paper's arithmetic (ablation)
    case 24: return k_accumulate<true, I, 24>;  // general index (wv_residues_general)
    default: return acc_kernel_m64v(arith, ilp);
  }
}

}  // namespace wv
