// wv_acc_m31y.cu -- the 32-bit-path formulation 39: the grouped form with
// groups of 4 cubes / 5 squares, larger than the default 31 (M31Form in
// wv_accum.cuh), for ablation.  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m31y(int arith, int ilp) {
  (void)arith;
  return ilp == 1 ? k_accumulate<false, 1, 39> : k_accumulate<false, 2, 39>;
}

}  // namespace wv
