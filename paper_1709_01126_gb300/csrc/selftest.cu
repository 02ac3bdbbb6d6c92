// pot3d_selftest_wait: runs the iteration kernels' bounded mbarrier wait on
// a barrier that nothing ever completes (no copy is issued, no other thread
// arrives), so the wait gives up after its limit and the kernel reports the
// TIMEOUT status the iteration kernels report; the host reads it back.
// Nothing is in flight when the block exits, so the context stays usable.
#include <algorithm>

#include "kernels.cuh"
#include "plan.h"

namespace {

__global__ void k_wait_selftest(unsigned long long limit_ns, int *status,
                                unsigned long long *elapsed_ns) {
  using namespace pot3d;
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  const uint64_t t0 = global_ns();
  const bool done = mbar_wait_for(&bar, 0u, limit_ns);
  const uint64_t t1 = global_ns();
  if (threadIdx.x == 0) {
    *status = done ? ST_RUNNING : ST_TIMEOUT;
    *elapsed_ns = t1 - t0;
  }
}

} // namespace

extern "C" int pot3d_selftest_wait(double limit_s, int *device_status, double *elapsed_s) {
  using namespace pot3d;
  if (!device_status || !(limit_s > 0.0) || !(limit_s <= 10.0)) return fail(POT3D_ERR_INVALID_ARG);
  struct Out {
    int status;
    unsigned long long ns;
  };
  Out *d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(Out));
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemset(d, 0, sizeof(Out));
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32>>>((unsigned long long)(limit_s * 1e9), &d->status, &d->ns);
    e = cudaGetLastError();
  }
  Out h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(Out), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_status(e);
  *device_status = h.status == ST_TIMEOUT ? POT3D_ERR_TIMEOUT : POT3D_OK;
  if (elapsed_s) *elapsed_s = h.ns * 1e-9;
  return POT3D_OK;
}

// ------------------------------------------------------------------------
// pot3d_probe_fp64_fma: the FP64 FMA rate of the device.  Every thread runs
// kChains independent DFMA chains (enough independent work per warp to
// cover the FP64 unit's latency), `rounds` times; the result is stored only
// under a condition the values never meet, so the chains cannot be removed.
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads)
    k_probe_dfma(int rounds, double a, double b, double *sink) {
  double v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) v[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int r = 0; r < rounds; r++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) v[c] = fma(v[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += v[c];
  if (s == -1.0) sink[blockIdx.x] = s;
}

} // namespace

extern "C" int pot3d_probe_fp64_fma(double min_seconds, double *fma_per_s, double *elapsed_s) {
  using namespace pot3d;
  if (!fma_per_s || !(min_seconds > 0.0) || !(min_seconds <= 5.0)) return fail(POT3D_ERR_INVALID_ARG);
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_status(e);
  const int blocks = 8 * nsm; // 2048 threads per SM resident
  double *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&sink, sizeof(double) * blocks);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // a = 1 - 2^-30 and b = 2^-30 keep every chain bounded near 1
  const double a = 1.0 - 0x1p-30, b = 0x1p-30;
  int rounds = 1 << 12;
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_probe_dfma<<<blocks, kProbeThreads>>>(64, a, b, sink); // warm-up
    e = cudaDeviceSynchronize();
  }
  while (e == cudaSuccess) {
    cudaEventRecord(e0);
    k_probe_dfma<<<blocks, kProbeThreads>>>(rounds, a, b, sink);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess || ms * 1e-3 >= min_seconds || rounds >= (1 << 28)) break;
    // grow towards the requested duration (at most 4x per step)
    const double grow = std::min(4.0, 1.2 * min_seconds / std::max(1e-6, ms * 1e-3));
    rounds = (int)std::min<double>((double)(1 << 28), rounds * std::max(1.5, grow));
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cuda_status(e);
  const double fmas = (double)blocks * kProbeThreads * kChains * (double)rounds;
  *fma_per_s = fmas / (ms * 1e-3);
  if (elapsed_s) *elapsed_s = ms * 1e-3;
  return POT3D_OK;
}
