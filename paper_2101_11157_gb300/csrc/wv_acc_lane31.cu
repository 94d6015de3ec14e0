// wv_acc_lane31.cu -- the 32-bit accumulation kernel (formulations 41, the
// default, 39 and 31) with lane chains as its work unit.  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_lane31(int arith, int ilp) {
  if (arith == 40 || arith >= 44) return acc_kernel_lane31x(arith, ilp);  // 48 (default) too
  if (arith == 39) return ilp == 1 ? k_accumulate<false, 1, 39, true> : k_accumulate<false, 2, 39, true>;
  if (arith >= 41) return ilp == 1 ? k_accumulate<false, 1, 41, true> : k_accumulate<false, 2, 41, true>;
  return ilp == 1 ? k_accumulate<false, 1, 31, true> : k_accumulate<false, 2, 31, true>;
}

}  // namespace wv
