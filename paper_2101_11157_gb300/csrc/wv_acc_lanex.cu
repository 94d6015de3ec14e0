// wv_acc_lanex.cu -- lane-chain ablation formulations: 32-bit groups of 5
// cubes / 6 squares (40) and 4 cubes / 7 squares (44); 64-bit Euler groups of
// 10 (42) and 11 (43) squares.  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_lane31x(int arith, int ilp) {
  if (arith == 40) return ilp == 1 ? k_accumulate<false, 1, 40, true> : k_accumulate<false, 2, 40, true>;
  if (arith == 44) return ilp == 1 ? k_accumulate<false, 1, 44, true> : k_accumulate<false, 2, 44, true>;
  return acc_kernel_lane31u(arith, ilp);
}

AccKernel acc_kernel_lane64x(int arith) {
  if (arith == 42) return k_accumulate_m64cap<42, kM64MaxReg, true>;
  return k_accumulate_m64cap<43, kM64MaxReg, true>;
}

}  // namespace wv
