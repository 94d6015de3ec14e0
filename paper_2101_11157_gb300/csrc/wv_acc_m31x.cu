// wv_acc_m31x.cu -- the 32-bit-path formulations 25..31: the grouped form 9
// with none, 4, 6 or all of a group's difference-table additions written as
// three-input adds that only the integer ALU executes (form 9 writes 4 of a
// Bernoulli group's and 2 of an Euler group's that way), for ablation of the
// balance between the ALU and the multiply pipe (25..28); and form 9 with
// groups of 3 cubes, of 4 squares, or both (29..31).  Groups of 4 / 5 (39)
// are in wv_acc_m31y.cu.  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m31x(int arith, int ilp) {
#define WV_PICK(I)                                                              \
  (arith == 25 ? k_accumulate<false, I, 25> : arith == 26 ? k_accumulate<false, I, 26> \
   : arith == 27 ? k_accumulate<false, I, 27> : arith == 28 ? k_accumulate<false, I, 28> \
   : arith == 29 ? k_accumulate<false, I, 29> : arith == 30 ? k_accumulate<false, I, 30> \
   : k_accumulate<false, I, 31>)
  if (arith == 39) return acc_kernel_m31y(arith, ilp);
  return ilp == 1 ? WV_PICK(1) : WV_PICK(2);
#undef WV_PICK
}

}  // namespace wv
