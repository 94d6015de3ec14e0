// wv_acc_lane64.cu -- the 64-bit accumulation kernel (grouped default, one
// chain per thread) with lane chains as its work unit.  The code is in
// wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_lane64(int arith) {
  if (arith == 42 || arith == 43) return acc_kernel_lane64x(arith);
  if (arith == 49 || arith == 50) return acc_kernel_lane64u(arith);
  return k_accumulate_m64cap<9, kM64MaxReg, true>;
}

}  // namespace wv
