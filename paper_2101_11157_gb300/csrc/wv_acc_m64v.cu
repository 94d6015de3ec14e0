// wv_acc_m64v.cu -- the 64-bit-path formulations 32..36: form 9 with part or
// all of its 64-bit table additions written as PTX carry chains (see
// M64Split in wv_accum.cuh), one chain per thread, for ablation of the
// balance between the integer ALU and the multiply pipe; 37, form 9 with the
// earlier (longer) shrink of its tables; 38, form 9 with its per-chain set-up
// unrolled as it was.  The code is in
// wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m64v(int arith, int ilp) {
  (void)ilp;
  switch (arith) {
    case 32: return k_accumulate_m64cap<32, kM64MaxReg>;
    case 33: return k_accumulate_m64cap<33, kM64MaxReg>;
    case 34: return k_accumulate_m64cap<34, kM64MaxReg>;
    case 35: return k_accumulate_m64cap<35, kM64MaxReg>;
    case 36: return k_accumulate_m64cap<36, kM64MaxReg>;
    case 37: return k_accumulate_m64cap<37, kM64MaxReg>;
    case 38: return k_accumulate_m64cap<38, kM64MaxReg>;
    default: return k_accumulate_m64cap<9, kM64MaxReg>;
  }
}

}  // namespace wv
