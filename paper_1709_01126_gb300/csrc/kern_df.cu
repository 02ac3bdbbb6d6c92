// Double-float instantiations of the iteration kernels.
#include "kern_inst.cuh"

namespace pot3d {

const MvVariant *mv_variants_df(int *count) {
  static const MvVariant v[] = {make_variant<PDF, 8, 2, 3>(3), make_variant<PDF, 8, 4, 2>(2)};
  *count = 2;
  return v;
}

KLaunch update_launcher_df() { return &up_launch<PDF>; }

} // namespace pot3d
