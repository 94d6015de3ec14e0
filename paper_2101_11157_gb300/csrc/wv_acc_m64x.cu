// wv_acc_m64x.cu -- the 64-bit-path formulations kept for ablation
// (wv_options.arith 10..22: other group sizes, shrink intervals, the two
// flags and the register budgets of M64Form), one chain per thread.  The
// code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m64x(int arith, int) {
  constexpr int I = 1;
  switch (arith) {
    case 10: return k_accumulate<true, I, 10>;
    case 11: return k_accumulate<true, I, 11>;
    case 12: return k_accumulate<true, I, 12>;
    case 13: return k_accumulate<true, I, 13>;
    case 14: return k_accumulate<true, I, 14>;
    case 15: return k_accumulate<true, I, 15>;
    case 16: return k_accumulate<true, I, 16>;
    case 17: return k_accumulate<true, I, 17>;
    case 18: return k_accumulate<true, I, 18>;
    case 19: return k_accumulate_m64cap<19, 96>;
    case 20: return k_accumulate_m64cap<20, 168>;
    case 21: return k_accumulate_m64cap<21, kM64MaxReg>;
    case 23: return k_accumulate<true, 1, 23>;  // the paper's arithmetic (ablation)
    case 24: return k_accumulate<true, 1, 24>;  // general index (wv_residues_general)
    default: return k_accumulate_m64cap<22, kM64MaxReg>;
  }
}

}  // namespace wv
