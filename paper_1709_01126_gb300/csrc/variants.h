// Kernel variants of the iteration, one translation unit per arithmetic.
//
// A matvec variant is one tile shape (TJ theta rows x 32*VK phi columns,
// S TMA stages) instantiated for one arithmetic.  The plan keeps the index
// of the variant in use per arithmetic; the autotuner (pot3d_autotune)
// times the variants and r-chunk counts on the plan's own problem.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace pot3d {

using KLaunch = void (*)(const ProbDev *, const int2 *, const int *, int grid, cudaStream_t);

struct MvVariant {
  int tj, vk, stages, es; // shape and element size (bytes)
  int al, tk, rh, bw;     // TMA geometry (see MvLayout)
  int smem_bytes;         // dynamic shared memory per block
  int blocks_per_sm;      // occupancy the launch bounds target
  int (*setup)();         // sets the dynamic shared memory attribute once
  KLaunch launch;
};

// Variants of arithmetic ai (AR_F64, AR_DF, AR_F32); *count receives their number.
const MvVariant *mv_variants(int ai, int *count);
// The update kernel of arithmetic ai.
KLaunch update_launcher(int ai);
// resident blocks per SM of arithmetic ai's update kernel (0: unknown)
int update_occupancy(int ai);

// Update kernel configurations per arithmetic: threads per block, bytes of
// r (and of q) per warp stage, stages per warp.  The FP64 kernel is bound by
// the FP64 unit; the HBM-bound ones keep more segments in flight.
constexpr int kUpdSegBytes = 2560;
constexpr int kUpdThreadsF64 = 256, kUpdStagesF64 = 2;
constexpr int kUpdThreadsDF = 128, kUpdStagesDF = 4;
constexpr int kUpdThreadsF32 = 128, kUpdStagesF32 = 5;

} // namespace pot3d
