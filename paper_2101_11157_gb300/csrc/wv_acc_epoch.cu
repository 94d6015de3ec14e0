// wv_acc_epoch.cu -- instantiations of the serving loop's epoch kernels
// (tiles of many plans per launch).  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

// the 64-bit tiles of an epoch run one chain per thread (the fastest grouped form)
EpochKernel epoch_kernel(bool wide, int ilp) {
  if (wide) return k_epoch<true, 1, 9>;
  return ilp == 1 ? k_epoch<false, 1, 9> : k_epoch<false, 2, 9>;
}

EpochKernel epoch_mixed_kernel(int ilp31, int) {
  return ilp31 == 1 ? k_epoch_mixed<1, 1> : k_epoch_mixed<2, 1>;
}

EpochTilesKernel epoch_tiles_kernel(int ilp31) {
  return ilp31 == 1 ? k_epoch_tiles<1, 1> : k_epoch_tiles<2, 1>;
}

}  // namespace wv
