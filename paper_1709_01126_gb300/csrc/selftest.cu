// pot3d_selftest_wait: runs the iteration kernels' bounded mbarrier wait on
// a barrier that nothing ever completes (no copy is issued, no other thread
// arrives), so the wait gives up after its limit and the kernel reports the
// TIMEOUT status the iteration kernels report; the host reads it back.
// Nothing is in flight when the block exits, so the context stays usable.
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
