// Double-float instantiations of the iteration kernels.
#include "kern_inst.cuh"

namespace pot3d {

const MvVariant *mv_variants_df(int *count) {
  static const MvVariant v[] = {make_variant<PDF, 8, 2, 3, 3, false>(), make_variant<PDF, 8, 4, 2, 2, false>(),
                                make_variant<PDF, 16, 2, 3, 1, false>(), make_variant<PDF, 8, 2, 3, 2, false>()};
  *count = 4;
  return v;
}

KLaunch update_launcher_df() { return &ur_launch<PDF, kUpdRsThreads, kUpdRsVecs>; }
int update_occupancy_df() { return ur_occupancy<PDF, kUpdRsThreads, kUpdRsVecs>(); }

} // namespace pot3d
