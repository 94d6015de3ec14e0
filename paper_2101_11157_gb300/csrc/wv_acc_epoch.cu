// wv_acc_epoch.cu -- instantiations of the serving loop's per-path epoch
// kernels (tiles of many plans per launch).  The code is in wv_accum.cuh;
// the ablation forms are in wv_acc_epoch_mixed.cu and wv_acc_epoch_tiles.cu.
#include "wv_accum.cuh"

namespace wv {

// the 64-bit tiles of an epoch run one chain per thread (the fastest grouped form)
EpochKernel epoch_kernel(bool wide, int ilp, bool lane) {
  if (lane) {
    if (wide) return k_epoch<true, 1, 50, true>;
    return ilp == 1 ? k_epoch<false, 1, 48, true> : k_epoch<false, 2, 48, true>;
  }
  if (wide) return k_epoch<true, 1, 9>;
  return ilp == 1 ? k_epoch<false, 1, 48> : k_epoch<false, 2, 48>;
}

}  // namespace wv
