// wv_acc_m64.cu -- instantiations of the accumulation kernels for
// 2^30 <= p < 2^37 (formulations 1 and 9).  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m64(int arith, int ilp) {
  if (arith == 9) return k_accumulate_m64cap<9, kM64MaxReg>;
  return ilp == 1 ? k_accumulate<true, 1, 1> : ilp == 2 ? k_accumulate<true, 2, 1>
                                                        : k_accumulate<true, 4, 1>;
}

}  // namespace wv
