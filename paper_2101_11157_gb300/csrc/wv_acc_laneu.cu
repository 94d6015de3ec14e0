// wv_acc_laneu.cu -- the 32-bit accumulation kernel in the u form (G0 = u^e
// from a table of u = prod (s+i)), lane chains: groups of 8 cubes / 10
// squares (45), 6 / 8 (46), 10 / 12 (47), 45 with other ALU-only splits (51,
// 52), and per warp 45 or 41 by piece length (48..50).  The code is in
// wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

AccKernel acc_kernel_lane31u(int arith, int ilp) {
  if (arith == 46) return ilp == 1 ? k_accumulate<false, 1, 46, true> : k_accumulate<false, 2, 46, true>;
  if (arith == 47) return ilp == 1 ? k_accumulate<false, 1, 47, true> : k_accumulate<false, 2, 47, true>;
  if (arith == 51) return ilp == 1 ? k_accumulate<false, 1, 51, true> : k_accumulate<false, 2, 51, true>;
  if (arith == 52) return ilp == 1 ? k_accumulate<false, 1, 52, true> : k_accumulate<false, 2, 52, true>;
  if (arith >= 48) return ilp == 1 ? k_accumulate<false, 1, 48, true> : k_accumulate<false, 2, 48, true>;
  return ilp == 1 ? k_accumulate<false, 1, 45, true> : k_accumulate<false, 2, 45, true>;
}

}  // namespace wv
