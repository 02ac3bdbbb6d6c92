// Instantiation helpers for the per-arithmetic kernel translation units.
#pragma once
#include "variants.h"

namespace pot3d {

template <class A, int TJ, int VK, int S, int MB, bool FP, int RPW>
int mv_setup() {
  static int done = 0;
  if (!done) {
    using LY = MvLayout<(int)sizeof(typename A::st), TJ, VK, S>;
    cudaError_t e = cudaFuncSetAttribute(k_matvec<A, TJ, VK, S, MB, FP, RPW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, LY::BYTES);
    if (e != cudaSuccess) return -3; // POT3D_ERR_CUDA
    done = 1;
  }
  return 0;
}

template <class A, int TJ, int VK, int S, int MB, bool FP, int RPW>
void mv_launch(const ProbDev *probs, const int2 *work, const int *nwork, int grid,
               cudaStream_t s) {
  using LY = MvLayout<(int)sizeof(typename A::st), TJ, VK, S>;
  k_matvec<A, TJ, VK, S, MB, FP, RPW><<<grid, dim3(32, TJ / RPW), LY::BYTES, s>>>(probs, work, nwork);
}

// MB: blocks per SM the launch bounds (and so the register budget) target;
// FP: separate unchecked code path for tiles inside the grid in phi;
// RPW: theta rows per warp (TJ / RPW warps per block)
template <class A, int TJ, int VK, int S, int MB, bool FP, int RPW = 1>
MvVariant make_variant() {
  using LY = MvLayout<(int)sizeof(typename A::st), TJ, VK, S>;
  MvVariant v;
  v.tj = TJ;
  v.vk = VK;
  v.stages = S;
  v.es = (int)sizeof(typename A::st);
  v.al = LY::AL;
  v.tk = LY::TK;
  v.rh = LY::RH;
  v.bw = LY::BW;
  v.smem_bytes = LY::BYTES;
  v.blocks_per_sm = MB;
  v.setup = &mv_setup<A, TJ, VK, S, MB, FP, RPW>;
  v.launch = &mv_launch<A, TJ, VK, S, MB, FP, RPW>;
  return v;
}

// Update kernel configurations: NT threads, SEGB-byte segments, STG stages
// per warp (stages - 1 segments of r and q in flight per warp).
template <class A, int NT, int SEGB, int STG>
void up_setup() {
  using LY = UpLayout<NT, SEGB, STG>;
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_update<A, NT, SEGB, STG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         LY::BYTES);
    done = true;
  }
}

template <class A, int NT, int SEGB, int STG>
void up_launch(const ProbDev *probs, const int2 *work, const int *nwork, int grid,
               cudaStream_t s) {
  using LY = UpLayout<NT, SEGB, STG>;
  up_setup<A, NT, SEGB, STG>();
  k_update<A, NT, SEGB, STG><<<grid, NT, LY::BYTES, s>>>(probs, work, nwork, nullptr);
}

// Update of diagonal scaling with register-staged rows (k_update_rs).
template <class A, int NT, int F>
void ur_launch(const ProbDev *probs, const int2 *work, const int *nwork, int grid,
               cudaStream_t s) {
  k_update_rs<A, NT, F><<<grid, NT, 0, s>>>(probs, work, nwork);
}

// Phi-line update: the stage layout plus one ring buffer of `pitch` values
// per warp.  Returns 0, or -1 when the shared memory would exceed what a
// block may use (the ring is too long for this configuration).
template <class A, int NT, int SEGB, int STG>
int up_line_launch(const ProbDev *probs, const int2 *work, const int *nwork, int grid, int pitch,
                   double *setup_out, cudaStream_t s) {
  using LY = UpLayout<NT, SEGB, STG>;
  const size_t bytes = LY::BYTES + (size_t)(NT / 32) * pitch * sizeof(typename A::val);
  static size_t set_to = 0;
  if (bytes > set_to) {
    if (bytes > 227 * 1024 ||
        cudaFuncSetAttribute(k_update<A, NT, SEGB, STG, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    set_to = bytes;
  }
  k_update<A, NT, SEGB, STG, true><<<grid, NT, bytes, s>>>(probs, work, nwork, setup_out);
  return 0;
}

// Radial-line kernel: one block per tiles_c work item, no dynamic shared memory.
template <class A, bool ADD>
void rl_launch(const ProbDev *probs, int grid, double *setup_out, cudaStream_t s) {
  k_rline<A, kRLineThreads, ADD><<<grid, kRLineThreads, 0, s>>>(probs, setup_out);
}

// PC2 kernel: kIluThreads threads, IluLayout bytes per warp.
template <class A>
int il_launch(const ProbDev *probs, int grid, int nr, double *setup_out, cudaStream_t s) {
  const size_t bytes = (size_t)(kIluThreads / 32) * IluLayout<A>::warp_bytes(nr);
  static size_t set_to = 0;
  if (bytes > set_to) {
    if (bytes > 227 * 1024 ||
        cudaFuncSetAttribute(k_ilu<A, kIluThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    set_to = bytes;
  }
  k_ilu<A, kIluThreads><<<grid, kIluThreads, bytes, s>>>(probs, setup_out);
  return 0;
}

// resident blocks of the diagonal-scaling update per SM (0 if the query fails)
template <class A, int NT, int F>
int ur_occupancy() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_update_rs<A, NT, F>, NT, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// resident blocks of the bulk-copy update kernel per SM (0 if the query fails)
template <class A, int NT, int SEGB, int STG>
int up_occupancy() {
  using LY = UpLayout<NT, SEGB, STG>;
  up_setup<A, NT, SEGB, STG>();
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_update<A, NT, SEGB, STG>, NT,
                                                    LY::BYTES) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

} // namespace pot3d
