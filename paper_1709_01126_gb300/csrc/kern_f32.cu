// FP32 instantiations of the iteration kernels (inner solve of refinement).
#include "kern_inst.cuh"

namespace pot3d {

const MvVariant *mv_variants_f32(int *count) {
  static const MvVariant v[] = {make_variant<PF32, 4, 4, 3, 3, true>(), make_variant<PF32, 8, 2, 3, 3, true>(),
                                make_variant<PF32, 8, 4, 3, 3, true>(), make_variant<PF32, 16, 4, 3, 1, true>(),
                                make_variant<PF32, 16, 4, 2, 2, true, 2>()};
  *count = 5;
  return v;
}

KLaunch update_launcher_f32() { return &ur_launch<PF32, kUpdRsThreads, kUpdRsVecs>; }
KLineLaunch update_line_launcher_f32() {
  return &up_line_launch<PF32, kUpdThreadsF32, kUpdSegBytes, kUpdStagesF32>;
}
KRLaunch rline_launcher_f32(bool add) {
  return add ? &rl_launch<PF32, true> : &rl_launch<PF32, false>;
}
KILaunch ilu_launcher_f32() { return &il_launch<PF32>; }
int update_occupancy_f32() { return ur_occupancy<PF32, kUpdRsThreads, kUpdRsVecs>(); }

// Tables of all arithmetics (indices AR_F64 = 0, AR_DF = 1, AR_F32 = 2).
const MvVariant *mv_variants_f64(int *count);
const MvVariant *mv_variants_df(int *count);
KLaunch update_launcher_f64();
KLaunch update_launcher_df();
int update_occupancy_f64();
int update_occupancy_df();

const MvVariant *mv_variants(int ai, int *count) {
  if (ai == 0) return mv_variants_f64(count);
  if (ai == 1) return mv_variants_df(count);
  return mv_variants_f32(count);
}

KLaunch update_launcher(int ai) {
  if (ai == 0) return update_launcher_f64();
  if (ai == 1) return update_launcher_df();
  return update_launcher_f32();
}

KLineLaunch update_line_launcher_f64();
KLineLaunch update_line_launcher(int ai) {
  if (ai == 0) return update_line_launcher_f64();
  if (ai == 2) return update_line_launcher_f32();
  return nullptr;
}

KRLaunch rline_launcher_f64(bool add);
KRLaunch rline_launcher(int ai, bool add) {
  if (ai == 0) return rline_launcher_f64(add);
  if (ai == 2) return rline_launcher_f32(add);
  return nullptr;
}

KILaunch ilu_launcher_f64();
KILaunch ilu_launcher(int ai) {
  if (ai == 0) return ilu_launcher_f64();
  if (ai == 2) return ilu_launcher_f32();
  return nullptr;
}

int update_occupancy(int ai) {
  if (ai == 0) return update_occupancy_f64();
  if (ai == 1) return update_occupancy_df();
  return update_occupancy_f32();
}

} // namespace pot3d
