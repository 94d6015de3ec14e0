// wv_acc_m64x.cu -- the 64-bit-path formulations kept for ablation
// (wv_options.arith 12..18 and 21: other group sizes, shrink intervals and
// register budgets of M64Form), one chain per thread.  The code is in
// wv_accum.cuh; forms 16..24 are instantiated in wv_acc_m64y.cu,
// wv_acc_m64z.cu and wv_acc_m64w.cu so that they compile in parallel.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_m64x(int arith, int ilp) {
  constexpr int I = 1;
  switch (arith) {
    case 12: return k_accumulate<true, I, 12>;
    case 13: return k_accumulate<true, I, 13>;
    case 14: return k_accumulate<true, I, 14>;
    case 15: return k_accumulate<true, I, 15>;
    default: return acc_kernel_m64y(arith, ilp);
  }
}

}  // namespace wv
