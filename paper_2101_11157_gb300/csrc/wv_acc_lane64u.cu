// wv_acc_lane64u.cu -- the 64-bit accumulation kernel in the u form (G0 =
// u^e from a table of u = prod (s+i)), lane chains: groups of 12 cubes / 16
// squares (49), and per warp 49 or the default by piece length (50).  The
// code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_lane64u(int arith) {
  if (arith == 49) return k_accumulate_m64cap<49, kM64MaxReg, true>;
  return k_accumulate_m64cap<50, kM64MaxReg, true>;
}

}  // namespace wv
