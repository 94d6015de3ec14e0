// wv_acc_m31x.cu -- the 32-bit-path formulations 25..28: the grouped form 9
// with none, 4, 6 or all of a group's difference-table additions written as
// three-input adds that only the integer ALU executes (form 9 writes 4 of a
// Bernoulli group's and 2 of an Euler group's that way), for ablation of the
// balance between the ALU and the multiply pipe.  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m31x(int arith, int ilp) {
#define WV_PICK(I)                                                              \
  (arith == 25 ? k_accumulate<false, I, 25> : arith == 26 ? k_accumulate<false, I, 26> \
   : arith == 27 ? k_accumulate<false, I, 27> : k_accumulate<false, I, 28>)
  return ilp == 1 ? WV_PICK(1) : WV_PICK(2);
#undef WV_PICK
}

}  // namespace wv
