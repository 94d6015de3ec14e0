// wv_acc_epoch_mixed.cu -- instantiations of the serving loop's ablation
// epoch form with one launch over both arithmetic paths.  The code is in
// wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

EpochKernel epoch_mixed_kernel(int ilp31, int, bool lane) {
  if (lane) return ilp31 == 1 ? k_epoch_mixed<1, 1, true> : k_epoch_mixed<2, 1, true>;
  return ilp31 == 1 ? k_epoch_mixed<1, 1> : k_epoch_mixed<2, 1>;
}

}  // namespace wv
