// Native FP64 instantiations of the iteration kernels.
#include "kern_inst.cuh"

namespace pot3d {

const MvVariant *mv_variants_f64(int *count) {
  static const MvVariant v[] = {make_variant<PF64, 8, 2, 3, 3, true>(), make_variant<PF64, 8, 4, 2, 2, true>(),
                                make_variant<PF64, 8, 2, 3, 2, true>()};
  *count = 3;
  return v;
}

// FP64 keeps the bulk-copy update: it is bound by the FP64 unit, and the
// register-staged kernel measured slower there (0.149 against 0.133 ms at
// 151 x 301 x 601)
KLaunch update_launcher_f64() { return &up_launch<PF64, kUpdThreadsF64, kUpdSegBytes, kUpdStagesF64>; }
KLineLaunch update_line_launcher_f64() {
  return &up_line_launch<PF64, kUpdThreadsF64, kUpdSegBytes, kUpdStagesF64>;
}
KRLaunch rline_launcher_f64(bool add) {
  return add ? &rl_launch<PF64, true> : &rl_launch<PF64, false>;
}
KILaunch ilu_launcher_f64() { return &il_launch<PF64>; }
int update_occupancy_f64() { return up_occupancy<PF64, kUpdThreadsF64, kUpdSegBytes, kUpdStagesF64>(); }

} // namespace pot3d
