// wv_acc_lane31.cu -- the 32-bit accumulation kernel (formulation 31) with
// lane chains as its work unit.  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_lane31(int ilp) {
  return ilp == 1 ? k_accumulate<false, 1, 31, true> : k_accumulate<false, 2, 31, true>;
}

}  // namespace wv
