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
// The update kernel of arithmetic ai (diagonal scaling).
KLaunch update_launcher(int ai);
// The update kernel with the phi-line preconditioner (FP64 and FP32 only;
// null for double-float): ring buffers of `pitch` values per warp, and the
// setup mode when setup_out is non-null.  Returns 0, or -1 (nothing
// launched) when the ring buffers do not fit in a block's shared memory.
using KLineLaunch = int (*)(const ProbDev *, const int2 *, const int *, int grid, int pitch,
                            double *setup_out, cudaStream_t);
KLineLaunch update_line_launcher(int ai);
// The radial-line kernel (FP64 and FP32 only; null for double-float).
// add = false: the whole update of the iteration with radial lines;
// add = true: the radial share after the phi-line update (both directions).
// setup_out non-null: the setup mode at the start of a PCG run.
using KRLaunch = void (*)(const ProbDev *, int grid, double *setup_out, cudaStream_t);
KRLaunch rline_launcher(int ai, bool add);
constexpr int kRLineThreads = 256;
// The PC2 kernel (subdomain ILU(0); FP64 and FP32 only, null for
// double-float): one warp per box of nr x 1 x 32 cells, kIluThreads / 32
// boxes per block, dynamic shared memory per warp from IluLayout.  setup_out
// as for the radial lines.  Returns 0, or -1 (nothing launched) when the
// warps' shared memory would exceed what a block may use (nr too large).
using KILaunch = int (*)(const ProbDev *, int grid, int nr, double *setup_out, cudaStream_t);
KILaunch ilu_launcher(int ai);
constexpr int kIluThreads = 128;
// resident blocks per SM of arithmetic ai's update kernel (0: unknown)
int update_occupancy(int ai);

// Update kernel configurations per arithmetic: threads per block, bytes of
// r (and of q) per warp stage, stages per warp.  Two blocks of 8 warps per
// SM with one segment in flight per warp beat one block with four in
// flight (FP32 at 151 x 301 x 601 under ncu: 59.7 against 68.3 us): the
// per-row work of the update is latency-bound and needs the warps.
constexpr int kUpdSegBytes = 2560;
// With diagonal scaling (PC1) the double-float and FP32 iterations run the
// register-staged update instead (FP64, bound by its FP64 unit, keeps the
// bulk-copy kernel): threads per block and 16-byte vectors per lane in one
// row segment.  FP32 at 151 x 301 x 601, event-timed in isolation: 63.6 us
// against 69.2 us for the bulk-copy kernel with a clean L2, 65.3 against
// 75.8 us with the matvec's dirty lines still in L2.
constexpr int kUpdRsThreads = 128, kUpdRsVecs = 5;
constexpr int kUpdThreadsF64 = 256, kUpdStagesF64 = 2;
constexpr int kUpdThreadsDF = 256, kUpdStagesDF = 2;
constexpr int kUpdThreadsF32 = 256, kUpdStagesF32 = 2;

} // namespace pot3d
