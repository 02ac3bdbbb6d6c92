// pot3d_residual_noalloc: the FP64 relative residual of pot3d_residual,
// computed without allocating anything during the call.
//
// Who needs it: code that must not allocate device memory at the point where
// it checks a solution, e.g. a caller whose device memory is owned by
// another allocator (a framework's caching allocator that must see every
// byte), a loop with a fixed memory budget that cannot risk an
// out-of-memory failure halfway, or code that runs where cudaMalloc would
// synchronise the device and stall other work.  Such a caller creates the
// plan once during set-up; this call then only launches kernels, using the
// plan's read-only tables and a fixed scratch array that lives in the
// library itself.
//
// The scratch is a file-scope __device__ array (kNoAllocScratchDoubles
// doubles = 32 KiB).  Every GPU that loads the library holds it until the
// process exits.  All calls share it, so calls whose kernels overlap on the
// GPU (different streams or threads without ordering between them) race and
// may return wrong values; order them on one stream.
#include <cmath>
#include <mutex>

#include <cudaTypedefs.h>

#include "plan.h"

// Capacity of the scratch: per-block partial pairs plus the two final sums.
constexpr int kNoAllocScratchDoubles = 4096;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = (kNoAllocScratchDoubles - 4) / 2;
constexpr int kMaxDevices = 64;

// Device addresses of the array, one per device, looked up with
// cudaGetSymbolAddress the first time the call runs with that device's
// context current (so that first call should come before any stream
// capture).  In host code the array's name is only a host-side stand-in,
// never a device address.  The address belongs to the context that loaded
// the module: each entry remembers that context's unique id, and a call made
// under another context (after cudaDeviceReset, say) looks the address up
// again instead of reusing a stale one.
std::mutex g_mu;
struct ScratchAddr {
  unsigned long long ctx_id;
  double *ptr;
};
ScratchAddr g_addr[kMaxDevices] = {};

// Unique id of the calling thread's current context; 0 when none is current
// yet or the driver entry points are unavailable.
unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    cudaGetLastError();
  });
  if (!get_cur || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int scratch_ptr(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pot3d::cuda_status(e);
  if (dev < 0 || dev >= kMaxDevices) return pot3d::fail(POT3D_ERR_TOO_LARGE);
  std::lock_guard<std::mutex> lk(g_mu);
  const unsigned long long id = current_context_id();
  ScratchAddr &a = g_addr[dev];
  if (!a.ptr || id == 0 || a.ctx_id != id) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      a = ScratchAddr{};
      return pot3d::cuda_status(e);
    }
    // the lookup made the device's primary context current if none was
    a.ctx_id = current_context_id();
    a.ptr = static_cast<double *>(p);
  }
  *out = a.ptr;
  return POT3D_OK;
}

// Per block: sum of b^2 (b from Br on the first radial layer, Eq. 2) and of
// (b - L phi)^2 with the FP64 operator of Eq. 4; written to fixed slots.
__global__ void __launch_bounds__(kNoAllocThreads)
    k_noalloc_partials(const double *__restrict__ br, const double *__restrict__ phi,
                       const double *__restrict__ S, const double *__restrict__ c64, int nr, int nt,
                       int np, double *scratch) {
  using namespace pot3d;
  __shared__ double red[kNoAllocThreads / 32];
  const size_t R = (size_t)nr * nt, n = R * np, plane = (size_t)nt * np;
  double sb = 0.0, sr = 0.0;
  for (size_t e = blockIdx.x * (size_t)kNoAllocThreads + threadIdx.x; e < n;
       e += (size_t)gridDim.x * kNoAllocThreads) {
    const size_t row = e / np;
    const int k = (int)(e - row * np);
    const int i = (int)(row / nt), j = (int)(row - (size_t)i * nt);
    const size_t c = row * np;
    double lx = c64[C64_D * R + row] * phi[c + k];
    if (i + 1 < nr) lx = fma(-c64[C64_RP * R + row], phi[c + plane + k], lx);
    if (i > 0) lx = fma(-c64[C64_RM * R + row], phi[c - plane + k], lx);
    if (j + 1 < nt) lx = fma(-c64[C64_TP * R + row], phi[c + np + k], lx);
    if (j > 0) lx = fma(-c64[C64_TM * R + row], phi[c - np + k], lx);
    const int kp = (k + 1 == np) ? 0 : k + 1, km = (k == 0) ? np - 1 : k - 1;
    lx = fma(-c64[C64_PH * R + row], phi[c + kp] + phi[c + km], lx);
    const double b = (i == 0) ? -S[j] * br[(size_t)j * np + k] : 0.0;
    const double res = b - lx;
    sb = fma(b, b, sb);
    sr = fma(res, res, sr);
  }
  const double tb = block_sum<kNoAllocThreads>(sb, red);
  const double tr = block_sum<kNoAllocThreads>(sr, red);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = tb;
    scratch[2 * blockIdx.x + 1] = tr;
  }
}

// Fixed-order sum of the block partials into the last two slots.
__global__ void __launch_bounds__(kNoAllocThreads) k_noalloc_final(double *scratch, int nblk) {
  using namespace pot3d;
  __shared__ double red[kNoAllocThreads / 32];
  const double b = block_sum_array<kNoAllocThreads>(scratch, nblk, 2, red);
  const double r = block_sum_array<kNoAllocThreads>(scratch + 1, nblk, 2, red);
  if (threadIdx.x == 0) {
    scratch[kNoAllocScratchDoubles - 2] = b;
    scratch[kNoAllocScratchDoubles - 1] = r;
  }
}

} // namespace

extern "C" int pot3d_residual_noalloc(pot3d_plan_t *plan, const double *br, const double *phi,
                                      double *relres) {
  using namespace pot3d;
  if (!plan || !br || !phi || !relres) return fail(POT3D_ERR_INVALID_ARG);
  // host arrays would need a staging copy in device memory
  if (!is_device_ptr(br) || !is_device_ptr(phi)) return fail(POT3D_ERR_INVALID_ARG);
  Plan *P = reinterpret_cast<Plan *>(plan);
  const size_t want = (P->n + kNoAllocThreads - 1) / kNoAllocThreads;
  const int nblk = (int)std::max<size_t>(1, std::min<size_t>(want, (size_t)4 * P->nsm));
  if (nblk > kNoAllocMaxBlocks) return fail(POT3D_ERR_TOO_LARGE);
  double *scratch = nullptr;
  int rc = scratch_ptr(&scratch);
  if (rc) return rc;
  cudaStream_t s = P->stream;
  // every slot read below is written first by this call: nothing to clear
  const double *brs = br;
  if (P->closed) {
    // closed wall: the balanced Br (zero net flux), in the plan's own
    // buffer; the flux partials and their sum use the scratch
    prepare_br(P, br, P->d_br_tmp, scratch, scratch + kNoAllocScratchDoubles - 4, s);
    brs = P->d_br_tmp;
  }
  k_noalloc_partials<<<nblk, kNoAllocThreads, 0, s>>>(brs, phi, P->d_S, P->d_c64, P->nr, P->nt,
                                                      P->np, scratch);
  k_noalloc_final<<<1, kNoAllocThreads, 0, s>>>(scratch, nblk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  double sums[2] = {0.0, 0.0};
  e = cudaMemcpyAsync(sums, scratch + kNoAllocScratchDoubles - 2, sizeof(sums),
                      cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  *relres = sums[0] > 0.0 ? std::sqrt(sums[1]) / std::sqrt(sums[0]) : 0.0;
  return POT3D_OK;
}
