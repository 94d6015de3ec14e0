// wv_acc_epoch_tiles.cu -- instantiations of the serving loop's ablation
// epoch form with one warp per tile.  The code is in wv_accum.cuh.
#include "wv_accum.cuh"

namespace wv {

EpochTilesKernel epoch_tiles_kernel(int ilp31, bool lane) {
  if (lane) return ilp31 == 1 ? k_epoch_tiles<1, 1, true> : k_epoch_tiles<2, 1, true>;
  return ilp31 == 1 ? k_epoch_tiles<1, 1> : k_epoch_tiles<2, 1>;
}

}  // namespace wv
