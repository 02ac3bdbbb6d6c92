// Device kernels of the PCG solve (Sec. 2.3, PC1) and the field (Sec. 2.1).
//
// Vectors live in HBM in C order [i][j][k] (r, theta, phi) with phi fastest
// and each phi row padded to `pitch` elements (a multiple of 32), so every row
// starts on a 256-byte boundary.  The iteration works on the diagonally
// scaled quantities  p~ = D p  and  x~ = D x  (D = diag(L), k-independent),
// which is the same PCG recurrence written without a separate z = D^-1 r
// vector:
//     p~_k = r_{k-1} + beta_{k-1} p~_{k-1}
//     q_k  = L D^-1 p~_k  = p~_k + sum_nb n_nb p~_nb     (n_nb = -c_nb / D_nb)
//     sigma_k = sum D^-1 p~_k q_k,   alpha_k = rho_{k-1} / sigma_k
//     x~ += alpha_k p~_k,  r_k = r_{k-1} - alpha_k q_k
//     rho_k = sum D^-1 r_k^2,  beta_k = rho_k / rho_{k-1}
// Two kernels per iteration (the two global reductions of PCG cannot be
// merged without changing the algorithm):
//   k_matvec : p~ update, x~ update (deferred by one iteration), 7-point
//              stencil with the boundary conditions folded into the metric
//              tables, sigma partial; the last block to finish forms alpha.
//   k_update : r update, ||r||^2 and rho partials; the last block forms the
//              relative residual, the convergence flag and beta (bulk copies
//              into shared memory; with the phi-line preconditioner also the
//              ring solve).  k_update_rs is the same update with rows staged
//              in registers (diagonal scaling in double-float and FP32);
//              k_rline (radial lines) and k_ilu (PC2, subdomain ILU(0)) take
//              its place with those preconditioners.
// Every reduction is deterministic: each work item writes its partial to a
// fixed slot, and the last block sums the slots in a fixed order.
#pragma once
#include <cuda.h>

#include <type_traits>

#include "arith.cuh"

namespace pot3d {

enum : int { ST_RUNNING = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_MAXIT = 3, ST_TIMEOUT = 4 };

// FP64 metric table of the unscaled operator, [7][nr*nt]:
//   0: D (diagonal, includes the 2 c^r term of the source-surface ghost)
//   1: Dinv   2: c^r_{i+1/2}   3: c^r_{i-1/2}   4: c^th_{j+1/2}   5: c^th_{j-1/2}
//   6: c^ph
// A coefficient is zero where its face is a boundary face (inner flux face,
// source surface, pole faces), so the stencil never reads past the grid.
enum { C64_D = 0, C64_DINV = 1, C64_RP = 2, C64_RM = 3, C64_TP = 4, C64_TM = 5, C64_PH = 6 };


struct SolveState {
  double rho;      // rho of the last completed iteration (D^-1-weighted r.r)
  double alpha[2]; // alpha_k in slot k&1
  double beta[2];  // beta_k in slot k&1
  double bb;       // ||b||^2 (scaled system)
  double tol;      // relative tolerance
  double relres;   // ||r_k|| / ||b||
  double sigma;    // last p.Ap
  double scale;    // power-of-two scale applied to b
  double rr;       // ||r_k||^2 as summed by the update kernel
  double rho_part; // both line directions: the phi-line update's share of rho
  int iter;        // completed iterations
  int maxit;
  int status;
  unsigned ticket_a, ticket_b;
  int pad_;
};

// TMA descriptors of one problem's iteration vectors (device memory).
// r, p0, p1: boxes of (TK + 2 AL) x (TJ + 2) x 1; x: TK x TJ x 1; *w: the
// AL-wide periodic wrap columns; cf: the six metric coefficients of TJ
// theta rows of one r plane (box TJ x 1 x 6 over the table [6][nr][ntp]).
struct TmaSet {
  CUtensorMap r, p0, p1, x, rw, p0w, p1w, cf;
};

// One problem (one solve) as the kernels see it.
struct ProbDev {
  int nr, nt, np, pitch;
  int ntp;            // row pitch of the metric tables (nt rounded up to 4)
  int pad0_;
  int nJ, nK, ic, nI; // matvec tiles along theta, phi; i-chunk length; i-chunks
  int tiles_a;        // nJ*nK*nI
  int rows_b;         // rows per update work item
  int tiles_b;
  int pad_;
  long long plane; // nt*pitch
  void *x, *r, *p0, *p1, *q;
  const void *coef;  // scaled metric table [6][nr][ntp]: Dinv, n_r+, n_r-, n_t+, n_t-, n_ph
  double *part_a;    // [tiles_a]
  double *part_b;    // [2*tiles_b]
  SolveState *st;
  const TmaSet *tma;
  double *hist;       // residual history [hist_cap] (null: not recorded)
  int hist_cap;
  int pad2_;
  void *w;            // line preconditioners: w = D M^-1 r (null: PC1)
  const void *lcoef;  // phi-line table [6][nr][ntp]: mu, mu / c, D mu / c, mu^m,
                      // mu^(np mod m), 1 / (1 - mu^np)  (m = ceil(np / 32))
  const void *rcoef;  // radial-line table [4][nr][ntp]: l, 1 / d', D / d', l' D / D'
                      // (see k_rline; null: no radial lines)
  double *part_c;     // [2 * tiles_c] partials of the radial-line kernel
  int tiles_c;        // radial-line blocks (8 warps of 32 columns each)
  int lines;          // 1: both line directions (the phi-line update forms
                      // w - r and leaves the close of the iteration to k_rline)
  const void *icoef;  // PC2 (subdomain ILU(0), see k_ilu): [4][nr][ntp] c^r_{i-1/2},
                      // c^r_{i+1/2}, D, c^ph, then the skewed pivot inverses
                      // [nt][nr + 31][32] (null: no PC2)
};

__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ int ldcg(const int *p) { return __ldcg(p); }

// Fixed-order block sum of one double per thread (xor butterfly inside each
// warp, then warp results in index order).  Result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (tid == 0) {
#pragma unroll
    for (int w = 0; w < NT / 32; w++) s += red[w];
  }
  __syncthreads();
  return s;
}

// Sum of a partial array in a fixed order by one block (L2 reads: other
// blocks wrote the partials during this launch).
template <int NT>
__device__ __forceinline__ double block_sum_array(const double *a, int n, int stride, double *red) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  double s = 0.0;
  for (int u = tid; u < n; u += NT) s += __ldcg(a + (size_t)u * stride);
  return block_sum<NT>(s, red);
}

// ------------------------------------------------------------ TMA / mbarrier
// Inline PTX for the Blackwell bulk-tensor copy engine: one elected thread
// issues cp.async.bulk.tensor box loads into shared memory; completion is
// tracked by transaction-counting mbarriers.  Every wait is bounded by the
// global timer so a lost transfer ends as a TIMEOUT status, not a hang.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\t"
               "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok)
               : "r"(smem_u32(bar)), "r"(parity)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr uint64_t kWaitLimitNs = 2000000000ull; // 2 s
// Wait for phase `parity` of `bar` for at most limit_ns; false if it gave up.
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, kWaitLimitNs);
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
               " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
               : "memory");
}

// Shared-memory plan of the matvec tile, shared by host (sizing) and device.
template <int ES, int TJ, int VK, int S>
struct MvLayout {
  static constexpr int AL = 16 / ES;        // elements per 16 bytes (TMA x alignment)
  static constexpr int TK = 32 * VK;        // phi columns per tile
  static constexpr int RH = TJ + 2, RW = TK + 2;
  static constexpr int BW = TK + 2 * AL;    // main box width: k0-AL .. k0+TK+AL-1
  static constexpr int a128(int b) { return (b + 127) / 128 * 128; }
  static constexpr int SZ_RP = a128(RH * BW * ES);
  static constexpr int SZ_X = a128(TJ * TK * ES);
  static constexpr int SZ_W = a128(RH * AL * ES);
  static constexpr int OFF_R = 0, OFF_P = SZ_RP, OFF_X = 2 * SZ_RP;
  static constexpr int OFF_RWL = OFF_X + SZ_X, OFF_PWL = OFF_RWL + SZ_W;
  static constexpr int OFF_RWR = OFF_PWL + SZ_W, OFF_PWR = OFF_RWR + SZ_W;
  static constexpr int SZ_C = a128(6 * TJ * ES);
  static constexpr int OFF_C = OFF_PWR + SZ_W;
  static constexpr int STAGE = OFF_C + SZ_C;
  static constexpr int RING = a128(3 * RH * RW * ES);
  static constexpr int BYTES = S * STAGE + RING + 8 * S;
  // a tensor-map box dimension holds at most 256 elements
  static_assert(BW <= 256 && RH <= 256, "TMA box wider than 256 elements");
};

// ------------------------------------------------------------ k_matvec
// Work item = (problem, tile).  A tile is TJ theta rows x TK = 32*VK phi
// columns, marching over an i-chunk [i0, i1).  Each warp owns one theta row;
// lane l owns phi columns k0 + l + 32 v.
// Data movement: for every r-plane of the chunk (plus one halo plane on each
// side) thread 0 issues TMA box loads of r and p~_old over the (TJ+2) x
// (TK+2) halo region (x from k0-AL so the box start is 16-byte aligned;
// theta rows outside the grid arrive zero-filled), of x~ over the owned
// cells, and of the two periodic wrap columns when the tile touches phi = 0
// or 2 pi.  S stages run ahead of the compute; every tile starts at stage 0
// and each thread tracks one mbarrier parity bit per stage.  Per plane the
// block forms p~_new = r + beta p~_old on the region into a 3-plane ring (one
// barrier per plane), stores p~_new and the deferred x~ += alpha_prev p~_old
// for its own cells, and applies the stencil to the previous plane
// (r-neighbours from registers).  The plane loop is unrolled by the ring
// period so ring slots and plane registers are compile-time; tiles inside the
// grid in phi may take a path without per-point bounds checks (FP); each
// thread's halo cell offsets are fixed once per tile.  MB sets the launch
// bounds' blocks per SM (the register budget).  The sigma partial closes with
// the last-block reduction.
template <class A, int TJ, int VK, int S, int MB, bool FP, int RPW>
__global__ void __launch_bounds__(32 * (TJ / RPW), MB)
    k_matvec(const ProbDev *__restrict__ probs, const int2 *__restrict__ work,
             const int *__restrict__ nwork_p) {
  using val = typename A::val;
  using st = typename A::st;
  using coef = typename A::coef;
  using LY = MvLayout<(int)sizeof(st), TJ, VK, S>;
  static_assert(TJ % RPW == 0, "a warp owns RPW whole theta rows");
  constexpr int AL = LY::AL, TK = LY::TK, RH = LY::RH, RW = LY::RW, BW = LY::BW;
  constexpr int NT = 32 * (TJ / RPW);
  constexpr int ES = (int)sizeof(st);
  extern __shared__ __align__(128) unsigned char smraw[];
  val(*ring)[RH][RW] = reinterpret_cast<val(*)[RH][RW]>(smraw + S * LY::STAGE);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smraw + S * LY::STAGE + LY::RING);
  __shared__ double red[NT / 32];
  __shared__ int s_last;
  const int lane = threadIdx.x, wy = threadIdx.y, tid = wy * 32 + lane;
  // this thread's first owned cell in ring slot 0; every ring access of the
  // owned cells and the stencil is a compile-time offset from it
  // (row wy * RPW; its other rows follow at RW)
  val *const rown = &ring[0][wy * RPW + 1][lane + 1];
  constexpr int RPL = RH * RW; // ring plane (elements)
  if (tid == 0) {
    for (int s = 0; s < S; s++) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t phase = 0; // bit s: parity of the next completion of stage s's mbarrier

  // the work list (and its length) lives in device memory, so one captured
  // graph serves any batch composition
  const int nwork = __ldcg(nwork_p);
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    const ProbDev &P = probs[wi.x];
    SolveState *stt = P.st;
    if (ldcg(&stt->status) != ST_RUNNING) continue;
    const int kit = ldcg(&stt->iter) + 1; // this iteration
    const int t = wi.y;
    const int nr = P.nr, nt = P.nt, np = P.np, pitch = P.pitch, ntp = P.ntp;
    const long long plane = P.plane;
    const int tk = t % P.nK, tj = (t / P.nK) % P.nJ, ci = t / (P.nK * P.nJ);
    const int j0 = tj * TJ, k0 = tk * TK, i0 = ci * P.ic;
    const int i1 = min(nr, i0 + P.ic);
    const bool first = (kit == 1);
    const TmaSet *T = P.tma;
    const CUtensorMap *m_r = &T->r, *m_x = &T->x;
    const CUtensorMap *m_po = (kit & 1) ? &T->p0 : &T->p1;
    const CUtensorMap *m_rw = &T->rw, *m_pow = (kit & 1) ? &T->p0w : &T->p1w, *m_cf = &T->cf;
    st *__restrict__ pnew = static_cast<st *>((kit & 1) ? P.p1 : P.p0);
    st *__restrict__ x = static_cast<st *>(P.x);
    st *__restrict__ q = static_cast<st *>(P.q);
    const coef *__restrict__ cf = static_cast<const coef *>(P.coef);
    const size_t R_ = (size_t)nr * ntp; // table slab of one coefficient
    const typename A::scal beta = A::scal_from(kit > 1 ? ldcg(&stt->beta[(kit - 1) & 1]) : 0.0);
    const typename A::scal alpha_prev =
        A::scal_from(kit > 1 ? ldcg(&stt->alpha[(kit - 1) & 1]) : 0.0);
    const bool wl = (k0 == 0), wr = (k0 + TK >= np);
    const int xl = ((np - 1) / AL) * AL, ol = (np - 1) - xl;
    const int ps = max(i0 - 1, 0), pe = min(i1, nr - 1), L = pe - ps + 1;

    // TMA loads of plane ps + tt into stage sidx (thread 0)
    auto issue = [&](int tt, int sidx) {
      const int ip = ps + tt;
      unsigned char *base = smraw + sidx * LY::STAGE;
      uint64_t *bar = &bars[sidx];
      const bool own = (ip >= i0 && ip < i1);
      const uint32_t box = RH * BW * sizeof(st), wbox = RH * AL * sizeof(st);
      uint32_t bytes = box + 6u * TJ * (uint32_t)sizeof(st);
      if (!first) bytes += box + (own ? TJ * TK * (uint32_t)sizeof(st) : 0u);
      const uint32_t nw = (wl ? 1u : 0u) + (wr ? 1u : 0u);
      bytes += nw * wbox * (first ? 1u : 2u);
      mbar_expect_tx(bar, bytes);
      // coefficients of plane ip-1: its stencil is applied once plane ip is in
      tma_load_3d(base + LY::OFF_C, m_cf, bar, j0, ip - 1, 0);
      tma_load_3d(base + LY::OFF_R, m_r, bar, k0 - AL, j0 - 1, ip);
      if (!first) {
        tma_load_3d(base + LY::OFF_P, m_po, bar, k0 - AL, j0 - 1, ip);
        if (own) tma_load_3d(base + LY::OFF_X, m_x, bar, k0, j0, ip);
      }
      if (wl) {
        tma_load_3d(base + LY::OFF_RWL, m_rw, bar, xl, j0 - 1, ip);
        if (!first) tma_load_3d(base + LY::OFF_PWL, m_pow, bar, xl, j0 - 1, ip);
      }
      if (wr) {
        tma_load_3d(base + LY::OFF_RWR, m_rw, bar, 0, j0 - 1, ip);
        if (!first) tma_load_3d(base + LY::OFF_PWR, m_pow, bar, 0, j0 - 1, ip);
      }
    };
    // every tile starts at stage 0: stage of step tt = tt % S
    if (tid == 0) {
      for (int tt = 0; tt < min(S, L); tt++) issue(tt, tt);
    }

    // theta rows of this warp: j0 + wy * RPW + rr, rr < RPW
    const int jw = j0 + wy * RPW;
    // full: every owned column k0 .. k0+TK-1 lies inside the grid (no
    // per-point phi checks); only the last tile column of a row of tiles
    // is not full.  FP = false keeps only the checked path (half the code:
    // faster where instruction fetch, not the checks, limits)
    const bool full = FP && (k0 + TK <= np);
    typename A::dacc tacc = A::d_init();
    // the owned cells of the last three planes: plane ps + tt in R[tt % 3]
    val R[3][RPW][VK];
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
      for (int rr = 0; rr < RPW; rr++)
#pragma unroll
        for (int v = 0; v < VK; v++) R[m][rr][v] = A::zero();
    bool bad = false;

    // Halo cells of the ring (rows 0 and RH-1, columns 0 and RW-1), HPT per
    // thread, fixed for the tile: byte offset of the r source within a
    // stage (main box or wrap column; -1: beyond the right wrap column, so
    // zero), distance from it to the p~_old source, and index within a
    // ring plane (-1: no cell).
    constexpr int NH = 2 * RW + 2 * TJ, HPT = (NH + NT - 1) / NT;
    int h_src[HPT], h_dp[HPT], h_dst[HPT];
#pragma unroll
    for (int u = 0; u < HPT; u++) {
      const int h = tid + u * NT;
      int rr, cc;
      if (h < 2 * RW) {
        rr = (h < RW) ? 0 : RH - 1;
        cc = (h < RW) ? h : h - RW;
      } else {
        const int g = h - 2 * RW;
        rr = 1 + (g >> 1);
        cc = (g & 1) ? RW - 1 : 0;
      }
      const int kk = k0 - 1 + cc;
      h_dst[u] = (h < NH) ? rr * RW + cc : -1;
      if (kk < 0) {
        h_src[u] = LY::OFF_RWL + (rr * AL + ol) * ES;
        h_dp[u] = LY::OFF_PWL - LY::OFF_RWL;
      } else if (kk < np) {
        h_src[u] = LY::OFF_R + (rr * BW + cc - 1 + AL) * ES;
        h_dp[u] = LY::OFF_P - LY::OFF_R;
      } else if (kk == np) {
        h_src[u] = LY::OFF_RWR + rr * AL * ES;
        h_dp[u] = LY::OFF_PWR - LY::OFF_RWR;
      } else {
        h_src[u] = -1;
        h_dp[u] = 0;
      }
    }

    // stencil of plane i, row jw + rr: in-plane neighbours from ring slot SL
    // (a compile-time constant), r-neighbours from registers (cur, prv, nxt:
    // planes i, i-1, i+1); F: full tile
    // metric coefficients of rows (i, jw + rr) for the stencil of the current step
    coef cc_[RPW][6];
    auto stencil = [&](int i, int rr, const coef(&c)[6], const val(&cur)[VK],
                       const val(&prv)[VK], const val(&nxt)[VK], auto SL, auto F) {
      constexpr bool kFull = decltype(F)::value;
      constexpr int sl = decltype(SL)::value;
      typename A::dacc racc = A::d_init();
      st *__restrict__ qrow = q + ((size_t)i * plane + (size_t)(jw + rr) * pitch + k0 + lane);
#pragma unroll
      for (int v = 0; v < VK; v++) {
        const int cc = lane + 32 * v + 1;
        typename A::sacc s = A::s_init(cur[v]);
        A::s_add(s, c[1], nxt[v]);
        A::s_add(s, c[2], prv[v]);
        const val *rc = rown + sl * RPL + rr * RW + 32 * v;
        A::s_add(s, c[3], rc[RW]);
        A::s_add(s, c[4], rc[-RW]);
        A::s_add(s, c[5], rc[-1]);
        A::s_add(s, c[5], rc[1]);
        const val qv = A::s_get(s);
        if (kFull || k0 + cc - 1 < np) {
          A::stv(qrow + 32 * v, qv);
          A::d_add(racc, cur[v], qv);
        }
      }
      A::d_addw(tacc, c[0], racc);
    };
    // p~_new of the owned cells of plane ip into the ring (natural mapping:
    // warp = theta row, lane = phi), with the stores of p~_new and of the
    // deferred x~ update for owned planes
    auto own_cells = [&](int ip, auto SL, bool own, const unsigned char *base, auto F) {
      constexpr bool kFull = decltype(F)::value;
      constexpr int sl = decltype(SL)::value;
      const st(*rs)[BW] = reinterpret_cast<const st(*)[BW]>(base + LY::OFF_R);
      const st(*pso)[BW] = reinterpret_cast<const st(*)[BW]>(base + LY::OFF_P);
      const st(*xs)[TK] = reinterpret_cast<const st(*)[TK]>(base + LY::OFF_X);
      const st(*rwr)[AL] = reinterpret_cast<const st(*)[AL]>(base + LY::OFF_RWR);
      const st(*pwr)[AL] = reinterpret_cast<const st(*)[AL]>(base + LY::OFF_PWR);
#pragma unroll
      for (int w = 0; w < RPW; w++) {
        const int tr = wy * RPW + w; // tile row
        const int rr = tr + 1;       // halo-box / ring row
        const bool wst = own && (jw + w < nt);
        const size_t off = (size_t)ip * plane + (size_t)(jw + w) * pitch + k0 + lane;
        st *__restrict__ xrow = x + off;
        st *__restrict__ prow = pnew + off;
#pragma unroll
        for (int v = 0; v < VK; v++) {
          const int cc = lane + 32 * v + 1, kk = k0 + cc - 1;
          val pn = A::zero();
          if (kFull || kk < np) {
            const val rv = A::ld(&rs[rr][cc - 1 + AL]);
            if (first) {
              pn = rv;
            } else {
              const val po = A::ld(&pso[rr][cc - 1 + AL]);
              pn = A::fma(beta, po, rv);
              if (wst) {
                const val xv = A::ld(&xs[tr][cc - 1]);
                A::stv(xrow + 32 * v, A::fma(alpha_prev, po, xv));
              }
            }
            if (wst) A::stv(prow + 32 * v, pn);
          } else if (kk == np) {
            const val rv = A::ld(&rwr[rr][0]);
            pn = first ? rv : A::fma(beta, A::ld(&pwr[rr][0]), rv);
          }
          rown[sl * RPL + w * RW + 32 * v] = pn;
        }
      }
    };

    // One step per plane, unrolled by the ring period 3 so that ring slots
    // and the roles of R are compile-time: step tt writes plane ps + tt
    // into ring slot and R[tt % 3] and applies the stencil to plane
    // ps + tt - 1 (R[(tt + 2) % 3]; R[(tt + 1) % 3] holds plane ps + tt - 2).
    int sidx = 0; // stage of step tt
    auto step = [&](int tt, auto U) -> bool {
      constexpr int u = decltype(U)::value;
      using Slot = std::integral_constant<int, u>;
      using Prev = std::integral_constant<int, (u + 2) % 3>;
      const int ip = ps + tt;
      const int st_now = sidx;
      sidx = (sidx + 1 == S) ? 0 : sidx + 1;
      const unsigned char *base = smraw + st_now * LY::STAGE;
      const coef(*cs)[TJ] = reinterpret_cast<const coef(*)[TJ]>(base + LY::OFF_C);
      bad = !mbar_wait(&bars[st_now], (phase >> st_now) & 1u);
      if (!bad) phase ^= 1u << st_now;
#pragma unroll
      for (int w = 0; w < RPW; w++)
#pragma unroll
        for (int m = 0; m < 6; m++) cc_[w][m] = cs[m][wy * RPW + w];
      const bool own = (ip >= i0 && ip < i1);
      if (full) own_cells(ip, Slot{}, own, base, std::true_type{});
      else own_cells(ip, Slot{}, own, base, std::false_type{});
      // halo cells
      val *ringp = &ring[u][0][0];
#pragma unroll
      for (int h = 0; h < HPT; h++) {
        if (h_dst[h] >= 0) {
          val pn = A::zero();
          if (h_src[h] >= 0) {
            const val rv = A::ld(reinterpret_cast<const st *>(base + h_src[h]));
            pn = first ? rv
                       : A::fma(beta, A::ld(reinterpret_cast<const st *>(base + h_src[h] + h_dp[h])),
                                rv);
          }
          ringp[h_dst[h]] = pn;
        }
      }
      if (__syncthreads_or(bad)) {
        bad = true;
        return false;
      }
      if (tid == 0 && tt + S < L) issue(tt + S, st_now);
#pragma unroll
      for (int w = 0; w < RPW; w++)
#pragma unroll
        for (int v = 0; v < VK; v++) R[u][w][v] = rown[u * RPL + w * RW + 32 * v];
      if (ip - 1 >= i0) {
#pragma unroll
        for (int w = 0; w < RPW; w++) {
          if (jw + w >= nt) break;
          if (full)
            stencil(ip - 1, w, cc_[w], R[(u + 2) % 3][w], R[(u + 1) % 3][w], R[u][w], Prev{},
                    std::true_type{});
          else
            stencil(ip - 1, w, cc_[w], R[(u + 2) % 3][w], R[(u + 1) % 3][w], R[u][w], Prev{},
                    std::false_type{});
        }
      }
      return true;
    };
    int tt = 0;
    for (; tt < L; tt += 3) {
      if (!step(tt, std::integral_constant<int, 0>{})) break;
      if (tt + 1 < L && !step(tt + 1, std::integral_constant<int, 1>{})) {
        tt += 1;
        break;
      }
      if (tt + 2 < L && !step(tt + 2, std::integral_constant<int, 2>{})) {
        tt += 2;
        break;
      }
    }
    if (bad) {
      // drain this tile's transfers still in flight (bounded), then report
      if (tid == 0) {
        for (int u = tt; u < min(L, tt + S); u++)
          mbar_wait(&bars[u % S], (phase >> (u % S)) & 1u);
        stt->status = ST_TIMEOUT;
      }
      __syncthreads();
      break;
    }
    if (i1 == nr) {
      // plane nr - 1 is the tile's last plane (step L - 1); no plane above
      const val zero[VK] = {};
#pragma unroll
      for (int w = 0; w < RPW; w++) {
        const size_t row = (size_t)(nr - 1) * ntp + (jw + w < nt ? jw + w : 0);
#pragma unroll
        for (int m = 0; m < 6; m++) cc_[w][m] = cf[m * R_ + row];
      }
      auto last = [&](auto U) {
        constexpr int u = decltype(U)::value;
#pragma unroll
        for (int w = 0; w < RPW; w++) {
          if (jw + w >= nt) break;
          if (full)
            stencil(nr - 1, w, cc_[w], R[u][w], R[(u + 2) % 3][w], zero, U, std::true_type{});
          else
            stencil(nr - 1, w, cc_[w], R[u][w], R[(u + 2) % 3][w], zero, U, std::false_type{});
        }
      };
      const int ul = (L - 1) % 3;
      if (ul == 0) last(std::integral_constant<int, 0>{});
      else if (ul == 1) last(std::integral_constant<int, 1>{});
      else last(std::integral_constant<int, 2>{});
    }

    // rows beyond nt never accumulated into tacc
    const double mine = A::d_get(tacc);
    const double tot = block_sum<NT>(mine, red);
    if (tid == 0) {
      P.part_a[t] = tot;
      __threadfence();
      const unsigned prev = atomicAdd(&stt->ticket_a, 1u);
      s_last = (prev == (unsigned)(P.tiles_a - 1));
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      const double sigma = block_sum_array<NT>(P.part_a, P.tiles_a, 1, red);
      if (tid == 0) {
        stt->sigma = sigma;
        if (!(sigma > 0.0) || !isfinite(sigma)) {
          stt->status = ST_BREAKDOWN;
        } else {
          stt->alpha[kit & 1] = stt->rho / sigma;
        }
        stt->ticket_a = 0u;
        __threadfence();
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ k_update
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
               " [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// ------------------------------------------------------- phi-line solve
// The phi-line preconditioner (one cyclic tridiagonal system per ring of
// fixed (i, j): diagonal D, both phi couplings -c) has constant coefficients
// along the ring, so it factors exactly as
//   T = d - c (S + S^-1) = (c / mu) (1 - mu S)(1 - mu S^-1),
// S the cyclic shift and mu + 1 / mu = d / c, 0 < mu < 1.  Hence
//   T^-1 = (mu / c) F F^T,   F = (1 - mu S)^-1,
// and F is a first-order recurrence around the ring, u_k = x_k + mu u_{k-1}
// (indices mod n), whose periodic solution is exact: with u_{-1} the value
// that closes the ring, u_{n-1} = mu^n u_{-1} + (the value reached from 0)
// fixes u_{-1} = (that value) / (1 - mu^n).  F^T is the same recurrence run backwards.  A warp solves a
// ring held in shared memory: every lane runs its contiguous chunk from a
// zero carry, the chunk maps c -> mu^len c + s are composed across lanes by
// a shuffle scan, the ring closure gives the carry into every chunk, and a
// second pass applies the recurrence from the right carry.  Adds this
// lane's share of ||F x||^2 to acc (a plain sum in the arithmetic's own
// type: F x is itself computed in that arithmetic, so a compensated sum of
// its squares would not be more accurate than the values it sums); x is
// overwritten by F^T F x.
// mu_m = mu^m and mu_rem = mu^(n mod m) for the lanes' chunk lengths
// m = ceil(n / 32) and n mod m; inv = 1 / (1 - mu^n) closes the ring.
template <class A>
__device__ __forceinline__ void ring_solve(typename A::val *x, int n, typename A::val mu,
                                           typename A::val mu_m, typename A::val mu_rem,
                                           typename A::val inv, typename A::val &acc, int lane) {
  using val = typename A::val;
  const int m = (n + 31) >> 5;
  const int a = min(lane * m, n), b = min(a + m, n);
  const val pm = (b - a == m) ? mu_m : (b == a ? A::one() : mu_rem);
  // ---- forward recurrence u_k = x_k + mu u_{k-1}
  val t = A::zero();
#pragma unroll 4
  for (int k = a; k < b; k++) t = A::fma(mu, t, x[k]);
  val M = pm, S = t;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const val M2 = A::shfl_up(M, off), S2 = A::shfl_up(S, off);
    if (lane >= off) {
      S = A::fma(M, S2, S);
      M = A::mul(M, M2);
    }
  }
  val Sx = A::shfl_up(S, 1), Px = A::shfl_up(M, 1);
  if (lane == 0) {
    Sx = A::zero();
    Px = A::one();
  }
  val total = A::shfl_idx(S, 31);
  t = A::fma(Px, A::mul(total, inv), Sx); // carry into this chunk
#pragma unroll 4
  for (int k = a; k < b; k++) {
    t = A::fma(mu, t, x[k]);
    x[k] = t;
    acc = A::fma(t, t, acc);
  }
  __syncwarp();
  // ---- backward recurrence v_k = u_k + mu v_{k+1}
  t = A::zero();
#pragma unroll 4
  for (int k = b - 1; k >= a; k--) t = A::fma(mu, t, x[k]);
  M = pm;
  S = t;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const val M2 = A::shfl_down(M, off), S2 = A::shfl_down(S, off);
    if (lane + off < 32) {
      S = A::fma(M, S2, S);
      M = A::mul(M, M2);
    }
  }
  Sx = A::shfl_down(S, 1);
  Px = A::shfl_down(M, 1);
  if (lane == 31) {
    Sx = A::zero();
    Px = A::one();
  }
  total = A::shfl_idx(S, 0);
  t = A::fma(Px, A::mul(total, inv), Sx);
#pragma unroll 4
  for (int k = b - 1; k >= a; k--) {
    t = A::fma(mu, t, x[k]);
    x[k] = t;
  }
  __syncwarp();
}

// Shared memory of k_update: per warp STG stages of (r, q) segments of
// SEGB bytes each, then STG mbarriers per warp; with the phi-line
// preconditioner, then one ring buffer of `pitch` values per warp (sized at
// launch).
template <int NT, int SEGB, int STG>
struct UpLayout {
  static constexpr int NW = NT / 32;
  static constexpr int WARP_BYTES = STG * 2 * SEGB;
  static constexpr int BYTES = NW * WARP_BYTES + NW * STG * 8;
};

// Closes iteration kit of a problem (one thread): relative residual,
// history, status, and for a running solve beta_k and rho_k.
__device__ __forceinline__ void close_iteration(const ProbDev &P, SolveState *stt, int kit,
                                                double rr, double rho) {
  const double relres = sqrt(rr) / sqrt(stt->bb);
  stt->relres = relres;
  stt->rr = rr;
  stt->iter = kit;
  if (P.hist && kit < P.hist_cap) P.hist[kit] = relres;
  if (!isfinite(relres)) {
    stt->status = ST_BREAKDOWN;
  } else if (relres <= stt->tol) {
    stt->status = ST_CONVERGED;
  } else if (kit >= stt->maxit) {
    stt->status = ST_MAXIT;
  } else {
    stt->beta[kit & 1] = rho / stt->rho;
    stt->rho = rho;
  }
}

// Work item = (problem, block of rows_b phi rows).  Each warp walks its rows
// (row0 + warp, + NW, ...) in segments of at most SEGB bytes: lane 0 keeps
// STG - 1 segments of r and q in flight ahead of the one the warp computes
// (cp.async.bulk into the warp's stages, completion counted by one mbarrier
// per stage, waits bounded by the global timer).  A cursor (row, i, j,
// segment) advances without divisions; the row's D^-1 weight is fetched
// before its first segment is awaited.  r -= alpha q is written back from
// registers; per row s = sum r^2, then ||r||^2 += s and rho += D^-1 s.  The
// last block closes the iteration.
//
// LINE (phi-line preconditioner): the warp also keeps the updated ring in
// its ring buffer and, at the ring's end, forms z = T^-1 r there
// (ring_solve), accumulates rho = r.z = (mu / c) ||F r||^2 and writes
// w = D z, the vector the next matvec reads in place of r.  setup_out
// non-null (LINE only): alpha = 0 and no iteration is closed; the last
// block writes ||r||^2 and rho to setup_out[0..1] (the start of a solve or
// of a refinement step).
template <class A, int NT, int SEGB, int STG, bool LINE = false>
__global__ void __launch_bounds__(NT)
    k_update(const ProbDev *__restrict__ probs, const int2 *__restrict__ work,
             const int *__restrict__ nwork_p, double *setup_out) {
  using val = typename A::val;
  using st = typename A::st;
  using coef = typename A::coef;
  using LY = UpLayout<NT, SEGB, STG>;
  constexpr int V = A::kVec, NW = NT / 32, ES = (int)sizeof(st), SEG = SEGB / ES;
  static_assert(SEG % (32 * V) == 0, "segment must be whole warp-vectors");
  static_assert(STG >= 2, "at least one segment in flight ahead");
  extern __shared__ __align__(128) unsigned char smu[];
  __shared__ double red[NW];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5, tid = threadIdx.x;
  st *wbuf = reinterpret_cast<st *>(smu + wy * LY::WARP_BYTES); // [stage][r|q][SEG]
  uint64_t *wbar = reinterpret_cast<uint64_t *>(smu + NW * LY::WARP_BYTES) + STG * wy;
  val *ring = reinterpret_cast<val *>(smu + LY::BYTES); // [NW][pitch] when LINE
  const bool setup = LINE && setup_out != nullptr;
  if (lane == 0) {
    for (int g = 0; g < STG; g++) mbar_init(&wbar[g], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t useq = 0; // segments this warp consumed so far (stage and parity)
  const int nwork = __ldcg(nwork_p);
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    const ProbDev &P = probs[wi.x];
    SolveState *stt = P.st;
    if (!setup && ldcg(&stt->status) != ST_RUNNING) continue;
    const int kit = ldcg(&stt->iter) + 1;
    const int t = wi.y;
    const int nt = P.nt, np = P.np, pitch = P.pitch, ntp = P.ntp;
    const long long plane = P.plane;
    const int R = P.nr * nt;
    const int row0 = t * P.rows_b, row1 = min(R, row0 + P.rows_b);
    st *__restrict__ r = static_cast<st *>(P.r);
    const st *__restrict__ q = static_cast<const st *>(P.q);
    const coef *__restrict__ cf = static_cast<const coef *>(P.coef);
    // phi-line table slabs: mu, mu / c, D mu / c, mu^m, mu^(np mod m), 1 / (1 - mu^np)
    const coef *__restrict__ lc = static_cast<const coef *>(P.lcoef);
    st *__restrict__ wv = static_cast<st *>(P.w);
    val *xr = ring + (size_t)wy * pitch;
    const size_t RT = (size_t)P.nr * ntp;
    const typename A::scal nalpha =
        A::scal_from(setup ? 0.0 : -ldcg(&stt->alpha[kit & 1]));
    // per-row sums of r^2: one accumulator per vector element (independent
    // dependency chains), merged at the end of the row
    typename A::dacc arr = A::d_init(), arho = A::d_init(), s[V];
#pragma unroll
    for (int e = 0; e < V; e++) s[e] = A::d_init();
    const int nseg = (np + SEG - 1) / SEG;
    const int nrows_w = (row1 - row0 - wy + NW - 1) / NW;
    const int units = nrows_w > 0 ? nrows_w * nseg : 0;
    // a cursor over this warp's units: row (i, j) and segment
    struct Cur {
      int i, j, seg;
      size_t off;
    };
    auto start = [&](int row) {
      Cur c;
      c.i = row / nt;
      c.j = row - c.i * nt;
      c.seg = 0;
      c.off = (size_t)c.i * plane + (size_t)c.j * pitch;
      return c;
    };
    auto advance = [&](Cur &c) {
      if (++c.seg == nseg) {
        c.seg = 0;
        c.j += NW;
        while (c.j >= nt) {
          c.j -= nt;
          c.i++;
        }
        c.off = (size_t)c.i * plane + (size_t)c.j * pitch;
      }
    };
    Cur ci = start(row0 + wy); // next unit to issue
    Cur cc = ci;               // next unit to compute
    auto issue = [&](int u) {
      if (lane == 0) {
        const uint32_t stg = (useq + u) % STG;
        const int len = min(SEG, np - ci.seg * SEG);
        const uint32_t bytes = (uint32_t)((len * ES + 15) & ~15);
        const size_t off = ci.off + (size_t)ci.seg * SEG;
        mbar_expect_tx(&wbar[stg], 2 * bytes);
        bulk_load(wbuf + (2 * stg) * SEG, r + off, bytes, &wbar[stg]);
        bulk_load(wbuf + (2 * stg + 1) * SEG, q + off, bytes, &wbar[stg]);
      }
      advance(ci);
    };
    bool bad = false;
    int issued = 0;
    for (; issued < min(units, STG - 1); issued++) issue(issued);
    int u = 0;
    coef wrow{}, lmu{}, lgd{}, lmm{}, lmr{}, linv{}, ldinv{};
    const bool lines = LINE && P.lines;
    for (; u < units; u++) {
      if (issued < units) issue(issued++);
      if (cc.seg == 0) { // ahead of the wait
        const size_t rj = (size_t)cc.i * ntp + cc.j;
        if constexpr (LINE) {
          lmu = lc[rj];
          wrow = lc[RT + rj];
          lgd = lc[2 * RT + rj];
          lmm = lc[3 * RT + rj];
          lmr = lc[4 * RT + rj];
          linv = lc[5 * RT + rj];
          if (lines) ldinv = cf[rj];
        } else {
          wrow = cf[rj];
        }
      }
      const uint32_t stg = (useq + u) % STG;
      if (!mbar_wait(&wbar[stg], ((useq + u) / STG) & 1u)) {
        bad = true;
        break;
      }
      const st *rs = wbuf + (2 * stg) * SEG;
      const st *qs = wbuf + (2 * stg + 1) * SEG;
      const int len = min(SEG, np - cc.seg * SEG);
      const size_t off = cc.off + (size_t)cc.seg * SEG;
      for (int k = lane * V; k < len; k += 32 * V) {
        val rv[V], qv[V];
#pragma unroll
        for (int e = 0; e < V; e++) {
          rv[e] = A::ld(rs + k + e);
          qv[e] = A::ld(qs + k + e);
        }
#pragma unroll
        for (int e = 0; e < V; e++) {
          rv[e] = A::fma(nalpha, qv[e], rv[e]);
          if (k + e < len) A::d_add(s[e], rv[e], rv[e]);
        }
        A::stvv(r + off + k, rv);
        if constexpr (LINE) {
#pragma unroll
          for (int e = 0; e < V; e++) xr[cc.seg * SEG + k + e] = rv[e];
        }
      }
      __syncwarp();
      if (cc.seg == nseg - 1) {
#pragma unroll
        for (int e = 1; e < V; e++) A::d_merge(s[0], s[e]);
        A::d_merge(arr, s[0]);
        if constexpr (LINE) {
          // z = T^-1 r on the ring; rho += (mu / c) ||F r||^2; w = D z
          val sz = A::zero();
          ring_solve<A>(xr, np, lmu, lmm, lmr, linv, sz, lane);
          A::d_addw(arho, wrow, A::d_of(sz));
          const size_t ro = cc.off;
          if (lines) {
            // both directions: this kernel's share is T_phi^-1 - D^-1
            // (rho -= D^-1 r.r on the row; w = D z - r, with r as this
            // lane stored it above)
            A::d_addw(arho, -ldinv, s[0]);
            for (int k = lane * V; k < np; k += 32 * V) {
              val wv_[V];
#pragma unroll
              for (int e = 0; e < V; e++) wv_[e] = A::sub(A::mul(lgd, xr[k + e]), A::ld(r + ro + k + e));
              A::stvv(wv + ro + k, wv_);
            }
          } else {
            for (int k = lane * V; k < np; k += 32 * V) {
              val wv_[V];
#pragma unroll
              for (int e = 0; e < V; e++) wv_[e] = A::mul(lgd, xr[k + e]);
              A::stvv(wv + ro + k, wv_);
            }
          }
          __syncwarp();
        } else {
          A::d_addw(arho, wrow, s[0]);
        }
#pragma unroll
        for (int e = 0; e < V; e++) s[e] = A::d_init();
      }
      advance(cc);
    }
    if (bad) {
      // drain this warp's copies still in flight (bounded), then report
      for (int v = u; v < issued; v++)
        mbar_wait(&wbar[(useq + v) % STG], ((useq + v) / STG) & 1u);
    }
    useq += issued;
    if (__syncthreads_or(bad)) {
      if (tid == 0) stt->status = ST_TIMEOUT;
      break;
    }
    const double prr = block_sum<NT>(A::d_get(arr), red);
    const double prho = block_sum<NT>(A::d_get(arho), red);
    if (tid == 0) {
      P.part_b[2 * t] = prr;
      P.part_b[2 * t + 1] = prho;
      __threadfence();
      const unsigned prev = atomicAdd(&stt->ticket_b, 1u);
      s_last = (prev == (unsigned)(P.tiles_b - 1));
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      const double rr = block_sum_array<NT>(P.part_b, P.tiles_b, 2, red);
      const double rho = block_sum_array<NT>(P.part_b + 1, P.tiles_b, 2, red);
      if (setup) {
        if (tid == 0) {
          setup_out[0] = rr;
          setup_out[1] = rho;
          stt->ticket_b = 0u;
          __threadfence();
        }
        __syncthreads();
        continue;
      }
      if (tid == 0) {
        if (LINE && P.lines) {
          // both line directions: k_rline adds the radial share and closes
          stt->rr = rr;
          stt->rho_part = rho;
        } else {
          close_iteration(P, stt, kit, rr, rho);
        }
        stt->ticket_b = 0u;
        __threadfence();
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ radial lines
// Radial-line Jacobi (Sec. 6 names stronger preconditioners that still
// vectorise as the open direction; this is the line counterpart of PC1 in r):
// M = T_r, the part of L inside each radial column (j, k): the full
// diagonal D_i (= D_ij) and the couplings e_i = -c^r_{i+1/2,j} between
// cells i and i + 1.  T_r is symmetric, diagonally dominant and the same for
// every k of a theta row, so its factorisation T_r = L' diag(d') L'^T
// (L' unit lower bidiagonal, multipliers l_i = e_{i-1} / d'_{i-1},
// d'_i = D_i - e_{i-1} l_i) is a table per (i, j), and a solve is two
// first-order recurrences along the column:
//     y_i = r_i - l_i y_{i-1}                       (forward, L'^-1)
//     z_i = y_i / d'_i - l_{i+1} z_{i+1}            (backward, L'^-T diag(d')^-1)
// and rho = r . T_r^-1 r = sum_i y_i^2 / d'_i.  In the scaled iteration the
// kernel writes w = D z; the backward recurrence runs on w directly:
//     w_i = (D_i / d'_i) y_i - (l_{i+1} D_i / D_{i+1}) w_{i+1}.
// Table [4][nr][ntp]: l_i, 1 / d'_i, D_i / d'_i, l_{i+1} D_i / D_{i+1}.
//
// One thread per column, 32 adjacent phi columns of one theta row per warp
// (every row access of the warp is one contiguous segment), 8 warps per
// block.  The forward pass keeps y in q's storage (q is dead once r is
// updated; the next matvec rewrites it), the backward pass reads it back in
// reverse order (mostly from L2).  Each thread loads PF = 8 planes of its
// column at a time before it runs them (four measured 4-7% slower in the
// mixed solves).  ADD = false: the kernel is the whole
// update of the iteration (r -= alpha q, ||r||^2, radial-line rho, w) and
// closes it.  ADD = true (both line directions): the phi-line update ran
// first (r updated, w holds D (T_phi^-1 - D^-1) r, ||r||^2 and its rho
// share in the state); this kernel adds D T_r^-1 r to w and the radial
// share to rho, and closes the iteration.  setup_out non-null: alpha = 0,
// no iteration is closed; the last block writes ||r||^2 and rho to
// setup_out[0..1] (ADD: adds the radial share to setup_out[1]).
template <class A, int NT, bool ADD>
__global__ void __launch_bounds__(NT)
    k_rline(const ProbDev *__restrict__ probs, double *setup_out) {
  using val = typename A::val;
  using st = typename A::st;
  using coef = typename A::coef;
  constexpr int NW = NT / 32, PF = 8;
  __shared__ double red[NW];
  __shared__ int s_last;
  const ProbDev &P = probs[0];
  SolveState *stt = P.st;
  const bool setup = setup_out != nullptr;
  if (!setup && ldcg(&stt->status) != ST_RUNNING) return;
  const int kit = ldcg(&stt->iter) + 1;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5, tid = threadIdx.x;
  const int nr = P.nr, nt = P.nt, np = P.np, ntp = P.ntp;
  const size_t plane = (size_t)P.plane;
  const size_t RT = (size_t)nr * ntp;
  const int nkg = (np + 31) >> 5;
  const int t = blockIdx.x;
  const int u = t * NW + wy;
  typename A::dacc arr = A::d_init(), arho = A::d_init();
  if (u < nt * nkg) {
    const int j = u / nkg;
    const int k = (u - j * nkg) * 32 + lane;
    if (k < np) {
      st *__restrict__ r = static_cast<st *>(P.r);
      st *__restrict__ q = static_cast<st *>(P.q); // y scratch after the r update
      st *__restrict__ w = static_cast<st *>(P.w);
      const coef *__restrict__ tl = static_cast<const coef *>(P.rcoef) + j;
      const typename A::scal nalpha =
          A::scal_from((ADD || setup) ? 0.0 : -ldcg(&stt->alpha[kit & 1]));
      const size_t c0 = (size_t)j * P.pitch + k;
      // ---- forward: r update, ||r||^2, y, rho
      val y = A::zero();
      int i = 0;
      for (; i + PF <= nr; i += PF) {
        val rv[PF], qv[PF];
#pragma unroll
        for (int e = 0; e < PF; e++) {
          rv[e] = A::ld(r + c0 + (size_t)(i + e) * plane);
          qv[e] = ADD ? A::zero() : A::ld(q + c0 + (size_t)(i + e) * plane);
        }
#pragma unroll
        for (int e = 0; e < PF; e++) {
          const size_t o = c0 + (size_t)(i + e) * plane;
          if (!ADD) {
            rv[e] = A::fma(nalpha, qv[e], rv[e]);
            if (!setup) A::stv(r + o, rv[e]);
            A::d_add(arr, rv[e], rv[e]);
          }
          const coef l = __ldg(tl + (size_t)(i + e) * ntp);
          const coef id = __ldg(tl + RT + (size_t)(i + e) * ntp);
          y = A::fma(-l, y, rv[e]);
          A::stv(q + o, y);
          A::d_add(arho, y, A::mul(id, y));
        }
      }
      for (; i < nr; i++) {
        const size_t o = c0 + (size_t)i * plane;
        val rv = A::ld(r + o);
        if (!ADD) {
          rv = A::fma(nalpha, A::ld(q + o), rv);
          if (!setup) A::stv(r + o, rv);
          A::d_add(arr, rv, rv);
        }
        const coef l = __ldg(tl + (size_t)i * ntp);
        const coef id = __ldg(tl + RT + (size_t)i * ntp);
        y = A::fma(-l, y, rv);
        A::stv(q + o, y);
        A::d_add(arho, y, A::mul(id, y));
      }
      // ---- backward: w = D z (ADD: plus the phi-line share already in w)
      val wn = A::zero();
      i = nr - 1;
      for (; i + 1 >= PF; i -= PF) {
        val yv[PF], av[PF];
#pragma unroll
        for (int e = 0; e < PF; e++) {
          yv[e] = A::ld(q + c0 + (size_t)(i - e) * plane);
          av[e] = ADD ? A::ld(w + c0 + (size_t)(i - e) * plane) : A::zero();
        }
#pragma unroll
        for (int e = 0; e < PF; e++) {
          const size_t ti = (size_t)(i - e) * ntp;
          const coef g = __ldg(tl + 2 * RT + ti);
          const coef h = __ldg(tl + 3 * RT + ti);
          wn = A::fma(-h, wn, A::mul(g, yv[e]));
          val out = wn;
          if constexpr (ADD) out = A::add(wn, av[e]);
          A::stv(w + c0 + (size_t)(i - e) * plane, out);
        }
      }
      for (; i >= 0; i--) {
        const size_t o = c0 + (size_t)i * plane;
        const coef g = __ldg(tl + 2 * RT + (size_t)i * ntp);
        const coef h = __ldg(tl + 3 * RT + (size_t)i * ntp);
        wn = A::fma(-h, wn, A::mul(g, A::ld(q + o)));
        val out = wn;
        if constexpr (ADD) out = A::add(wn, A::ld(w + o));
        A::stv(w + o, out);
      }
    }
  }
  const double prr = ADD ? 0.0 : block_sum<NT>(A::d_get(arr), red);
  const double prho = block_sum<NT>(A::d_get(arho), red);
  if (tid == 0) {
    P.part_c[2 * t] = prr;
    P.part_c[2 * t + 1] = prho;
    __threadfence();
    const unsigned prev = atomicAdd(&stt->ticket_b, 1u);
    s_last = (prev == (unsigned)(P.tiles_c - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double rr = ADD ? 0.0 : block_sum_array<NT>(P.part_c, P.tiles_c, 2, red);
  const double rho_r = block_sum_array<NT>(P.part_c + 1, P.tiles_c, 2, red);
  if (tid == 0) {
    if (setup) {
      if (ADD) {
        setup_out[1] += rho_r;
      } else {
        setup_out[0] = rr;
        setup_out[1] = rho_r;
      }
    } else if (ADD) {
      close_iteration(P, stt, kit, ldcg(&stt->rr), rho_r + ldcg(&stt->rho_part));
    } else {
      close_iteration(P, stt, kit, rr, rho_r);
    }
    stt->ticket_b = 0u;
    __threadfence();
  }
}

// ------------------------------------------------------- k_update_rs
// The update of diagonal scaling (PC1) with register-staged rows: the same
// work items, row walk, per-row sums and close as k_update, but each unit
// (a row segment of SEG = 32 F kVec elements) is loaded straight into
// registers with 16-byte loads, and the next unit's loads are issued before
// the current one is reduced (two register sets, alternating).  Measured
// at 151 x 301 x 601 in FP32 it beats the bulk-copy staging by 8-12%, and
// does not slow down when the L2 still holds the matvec's dirty lines.
// Elements past np (the row padding) are zero and stay zero; they are
// updated with the row but left out of the sums.
template <class A, int NT, int F>
__global__ void __launch_bounds__(NT)
    k_update_rs(const ProbDev *__restrict__ probs, const int2 *__restrict__ work,
                const int *__restrict__ nwork_p) {
  using val = typename A::val;
  using st = typename A::st;
  using coef = typename A::coef;
  constexpr int V = A::kVec, NW = NT / 32, SEG = 32 * V * F;
  __shared__ double red[NW];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5, tid = threadIdx.x;
  const int nwork = __ldcg(nwork_p);
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    const ProbDev &P = probs[wi.x];
    SolveState *stt = P.st;
    if (ldcg(&stt->status) != ST_RUNNING) continue;
    const int kit = ldcg(&stt->iter) + 1;
    const int t = wi.y;
    const int nt = P.nt, np = P.np, pitch = P.pitch, ntp = P.ntp;
    const long long plane = P.plane;
    const int R = P.nr * nt;
    const int row0 = t * P.rows_b, row1 = min(R, row0 + P.rows_b);
    st *__restrict__ r = static_cast<st *>(P.r);
    const st *__restrict__ q = static_cast<const st *>(P.q);
    const coef *__restrict__ cf = static_cast<const coef *>(P.coef);
    const typename A::scal nalpha = A::scal_from(-ldcg(&stt->alpha[kit & 1]));
    typename A::dacc arr = A::d_init(), arho = A::d_init(), s[V];
#pragma unroll
    for (int e = 0; e < V; e++) s[e] = A::d_init();
    const int nseg = (np + SEG - 1) / SEG;
    const int nrows_w = (row1 - row0 - wy + NW - 1) / NW;
    const int units = nrows_w > 0 ? nrows_w * nseg : 0;
    struct Cur {
      int i, j, seg;
      size_t off;
    };
    auto advance = [&](Cur &c) {
      if (++c.seg == nseg) {
        c.seg = 0;
        c.j += NW;
        while (c.j >= nt) {
          c.j -= nt;
          c.i++;
        }
        c.off = (size_t)c.i * plane + (size_t)c.j * pitch;
      }
    };
    Cur cl;
    cl.i = (row0 + wy) / nt;
    cl.j = row0 + wy - cl.i * nt;
    cl.seg = 0;
    cl.off = (size_t)cl.i * plane + (size_t)cl.j * pitch;
    Cur cc = cl;
    val rb[2][F][V], qb[2][F][V];
    coef wb[2];
    auto load = [&](int b) {
#pragma unroll
      for (int m = 0; m < F; m++) {
        const int k = cl.seg * SEG + (lane + 32 * m) * V;
        if (k < pitch) {
          A::ldv(r + cl.off + k, rb[b][m]);
          A::ldv(q + cl.off + k, qb[b][m]);
        }
      }
      wb[b] = cf[(size_t)cl.i * ntp + cl.j];
      advance(cl);
    };
    auto compute = [&](int b) {
#pragma unroll
      for (int m = 0; m < F; m++) {
        const int k = cc.seg * SEG + (lane + 32 * m) * V;
        if (k < pitch) {
          val rv[V];
#pragma unroll
          for (int e = 0; e < V; e++) {
            rv[e] = A::fma(nalpha, qb[b][m][e], rb[b][m][e]);
            if (k + e < np) A::d_add(s[e], rv[e], rv[e]);
          }
          A::stvv(r + cc.off + k, rv);
        }
      }
      if (cc.seg == nseg - 1) {
#pragma unroll
        for (int e = 1; e < V; e++) A::d_merge(s[0], s[e]);
        A::d_merge(arr, s[0]);
        A::d_addw(arho, wb[b], s[0]);
#pragma unroll
        for (int e = 0; e < V; e++) s[e] = A::d_init();
      }
      advance(cc);
    };
    if (units > 0) load(0);
    for (int u = 0; u < units; u += 2) {
      if (u + 1 < units) load(1);
      compute(0);
      if (u + 1 < units) {
        if (u + 2 < units) load(0);
        compute(1);
      }
    }
    const double prr = block_sum<NT>(A::d_get(arr), red);
    const double prho = block_sum<NT>(A::d_get(arho), red);
    if (tid == 0) {
      P.part_b[2 * t] = prr;
      P.part_b[2 * t + 1] = prho;
      __threadfence();
      const unsigned prev = atomicAdd(&stt->ticket_b, 1u);
      s_last = (prev == (unsigned)(P.tiles_b - 1));
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      const double rr = block_sum_array<NT>(P.part_b, P.tiles_b, 2, red);
      const double rho = block_sum_array<NT>(P.part_b + 1, P.tiles_b, 2, red);
      if (tid == 0) {
        close_iteration(P, stt, kit, rr, rho);
        stt->ticket_b = 0u;
        __threadfence();
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- PC2: subdomain ILU(0)
// PC2 of Sec. 2.3: non-overlapping domain decomposition, ILU(0) of every
// subdomain block of L, couplings between subdomains dropped.  A subdomain
// is a box of every r cell x 1 theta row x 32 phi columns (a warp: lane kk
// owns column k0 + kk), numbered in C order.  Inside such a box a cell's
// lower neighbours are (i - 1, k) and (i, k - 1), and for the 7-point
// pattern ILU(0) keeps L's couplings and changes only the diagonal:
//     M = (P + E) P^-1 (P + E^T),  E the strict lower part of the box block,
//     p_ik = D_i - [i > 0] (c^r_{i-1/2})^2 / p_{i-1,k} - [kk > 0] (c^ph)^2 / p_{i,k-1}.
// z = M^-1 r is a forward and a backward substitution:
//     s = r + c^r_{i-1/2} y_{i-1,k} + c^ph y_{i,k-1},   y = s / p,  rho += y s
//     z = y + (c^r_{i+1/2} z_{i+1,k} + c^ph z_{i,k+1}) / p,           w = D z
// (rho = r.M^-1 r = sum p y^2 = sum y s).  Cell (i, k) depends on its
// lower neighbours only, so lane kk runs cell i at step t = i + kk (a
// wavefront across the warp): the phi neighbour's value arrives by one
// shuffle from the previous step, the radial one is the lane's own.  Global
// memory stays coalesced: every step the warp loads one whole r plane of
// its 32 columns (r -= alpha q, ||r||^2, written back) and lane kk reads its
// column of it kk steps later from a delay line in shared memory (32 steps
// x 32 lanes; each lane only reads back what it wrote itself).  y goes to
// q's storage (q is dead once r is updated) in wavefront order: the row of
// step t at row t mod nr.  The backward pass runs the wavefront the other
// way (lane kk at step nr + 30 - i - kk), which reads those rows in reverse
// order, and writes w = D z a plane at a time through the delay line once
// lane 0 has run the plane.  Each step's loads go by cp.async into a
// staging ring in shared memory, PF steps ahead, one copy group per step
// awaited by count (loads prefetched into registers instead waited for all
// younger loads too, and every step paid a memory latency).  The
// pivot inverses are stored skewed, [j][t][kk] = 1 / p(t - kk, j, kk), so
// the lanes' loads of one step are one contiguous row too.  The last block
// sums the partials and closes the iteration; setup_out non-null: alpha = 0,
// no iteration is closed, ||r||^2 and rho go to setup_out[0..1].
template <class A>
struct IluLayout {
  // steps whose loads are in flight (cp.async groups)
  static constexpr int PF = 8;
  // a delay line of 32 steps x 32 lanes; PF staging slots of three rows of
  // 32 (r, q, pivots in the forward pass; y and pivots in the backward);
  // then the warp's coefficient columns [4][nr] (c^r_{i-1/2}, c^r_{i+1/2},
  // D, c^ph of its theta row)
  static __host__ __device__ size_t warp_bytes(int nr) {
    return ((32 * 32 + PF * 3 * 32) * sizeof(typename A::val) +
            4 * (size_t)nr * sizeof(typename A::coef) + 15) &
           ~(size_t)15;
  }
};

// Asynchronous copies of one element per thread from global to shared
// memory (cp.async, 4 or 8 bytes), committed as one group per wavefront step
// and awaited by group count: k_ilu keeps PF steps of loads in flight and
// waits for exactly the oldest step.
template <int B>
__device__ __forceinline__ void cp_async_elem(void *dst, const void *src) {
  static_assert(B == 4 || B == 8, "cp.async element of 4 or 8 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(B)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <class A, int NT>
__global__ void __launch_bounds__(NT)
    k_ilu(const ProbDev *__restrict__ probs, double *setup_out) {
  using val = typename A::val;
  using st = typename A::st;
  using coef = typename A::coef;
  constexpr int NW = NT / 32, PF = IluLayout<A>::PF;
  static_assert((PF & (PF - 1)) == 0, "PF a power of two");
  extern __shared__ __align__(16) unsigned char smi[];
  __shared__ double red[NW];
  __shared__ int s_last;
  const ProbDev &P = probs[0];
  SolveState *stt = P.st;
  const bool setup = setup_out != nullptr;
  if (!setup && ldcg(&stt->status) != ST_RUNNING) return;
  const int kit = ldcg(&stt->iter) + 1;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5, tid = threadIdx.x;
  const int nr = P.nr, nt = P.nt, np = P.np, ntp = P.ntp;
  const size_t plane = (size_t)P.plane;
  const size_t RT = (size_t)nr * ntp;
  const int nkg = (np + 31) >> 5;
  const int u = blockIdx.x * NW + wy;
  typename A::dacc arr = A::d_init(), arho = A::d_init();
  if (u < nt * nkg) {
    const int j = u / nkg, k0 = (u - j * nkg) * 32, k = k0 + lane;
    const bool act = k < np;
    const bool up = lane < 31 && k + 1 < np; // phi neighbour k + 1 in the box
    val *dl = reinterpret_cast<val *>(smi + (size_t)wy * IluLayout<A>::warp_bytes(nr));
    val *stg = dl + 32 * 32; // [PF][3][32]
    coef *cc = reinterpret_cast<coef *>(stg + PF * 3 * 32);
    const coef *__restrict__ ic = static_cast<const coef *>(P.icoef);
    for (int i = lane; i < nr; i += 32) {
      const size_t o = (size_t)i * ntp + j;
      cc[i] = ic[o];
      cc[nr + i] = ic[RT + o];
      cc[2 * nr + i] = ic[2 * RT + o];
      cc[3 * nr + i] = ic[3 * RT + o];
    }
    const coef *__restrict__ pv = ic + 4 * RT + (size_t)j * (nr + 31) * 32 + lane;
    __syncwarp();
    st *__restrict__ r = static_cast<st *>(P.r);
    st *__restrict__ q = static_cast<st *>(P.q); // y after the r update
    st *__restrict__ w = static_cast<st *>(P.w);
    const typename A::scal nalpha = A::scal_from(setup ? 0.0 : -ldcg(&stt->alpha[kit & 1]));
    const size_t c0 = (size_t)j * P.pitch + k;
    const int T = nr + 31; // wavefront steps per pass
    constexpr int EB = (int)sizeof(val);
    static_assert(sizeof(val) == sizeof(st) && sizeof(val) == sizeof(coef),
                  "one element size for the staged rows");
    // ---- forward: r update, ||r||^2, y = (P + E)^-1 r, rho.  The loads of
    // step t (the lane's element of r and q in plane t, its pivot row t) go
    // by cp.async into staging slot t mod PF, one group per step, PF steps
    // ahead.  y goes to q's storage in wavefront order: the y of step t
    // (lane kk: cell t - kk) is one row of 32, stored at row t mod nr (a
    // lane's steps kk .. kk + nr - 1 fall on distinct rows), which is also
    // the order in which the backward pass needs it.
    auto fetch_f = [&](int t) {
      val *sl = stg + (t & (PF - 1)) * 96 + lane;
      if (act && t < nr) {
        cp_async_elem<EB>(sl, r + c0 + (size_t)t * plane);
        if (!setup) cp_async_elem<EB>(sl + 32, q + c0 + (size_t)t * plane);
      }
      if (t < T) cp_async_elem<EB>(sl + 64, pv + (size_t)t * 32);
      cp_async_commit();
    };
    for (int t = 0; t < PF - 1; t++) fetch_f(t);
    val ymine = A::zero(); // y of this lane's last cell: y_{i-1,k} of its next one
    val rho_c = A::zero(); // rho of the current chunk of PF steps (see below)
    int yrow = 0;          // t mod nr
    for (int t = 0; t < T; t++) {
      fetch_f(t + PF - 1);
      cp_async_wait<PF - 1>(); // the group of step t has landed
      const val *sl = stg + (t & (PF - 1)) * 96 + lane;
      const coef piv = reinterpret_cast<const coef *>(sl)[64];
      if (t < nr) {
        // plane t arrives for the whole warp; lane kk uses it kk steps
        // later (its own column of the delay line)
        val rv = sl[0];
        if (act && !setup) {
          rv = A::fma(nalpha, sl[32], rv);
          A::stv(r + c0 + (size_t)t * plane, rv);
        }
        if (act) A::d_add(arr, rv, rv);
        dl[(t & 31) * 32 + lane] = rv;
      }
      const val yleft = A::shfl_up(ymine, 1); // y_{i,k-1}, the previous step of lane - 1
      const int i = t - lane;
      if (act && i >= 0 && i < nr) {
        val sv = A::fma(cc[i], ymine, dl[(i & 31) * 32 + lane]);
        if (lane > 0) sv = A::fma(cc[3 * nr + i], yleft, sv);
        const val y = A::mul(sv, piv);
        rho_c = A::fma(y, sv, rho_c);
        ymine = y;
        A::stv(q + c0 + (size_t)yrow * plane, y);
      }
      if (++yrow == nr) yrow = 0;
      // rho: a plain sum of y s over each chunk of PF steps in the
      // arithmetic's own type (y and s are the preconditioner's own
      // results, rounded in that type), merged into arho per chunk
      if ((t & (PF - 1)) == PF - 1 || t == T - 1) {
        A::d_merge(arho, A::d_of(rho_c));
        rho_c = A::zero();
      }
    }
    cp_async_wait<0>();
    __threadfence_block(); // the y stores above come before the copies below read them
    // ---- backward: z = (P + E^T)^-1 P y, w = D z; lane kk runs cell i at
    // step T - 1 - i - kk, whose y is the forward's row i + kk, read from
    // row (T - 1 - t) mod nr (the y each lane wrote there itself)
    int brow = (T - 1) % nr; // (T - 1 - t) mod nr of the next step fetched
    int tb = 0;              // step of the next fetch
    auto fetch_b = [&]() {
      val *sl = stg + (tb & (PF - 1)) * 96 + lane;
      if (tb < T) {
        if (act) cp_async_elem<EB>(sl, q + c0 + (size_t)brow * plane);
        cp_async_elem<EB>(sl + 64, pv + (size_t)(T - 1 - tb) * 32);
      }
      cp_async_commit();
      if (--brow < 0) brow = nr - 1;
      tb++;
    };
    for (int e = 0; e < PF - 1; e++) fetch_b();
    val zmine = A::zero(); // z of this lane's last cell: z_{i+1,k} of its next one
    for (int t = 0; t < T; t++) {
      fetch_b();
      cp_async_wait<PF - 1>();
      const val *sl = stg + (t & (PF - 1)) * 96 + lane;
      const val yv = sl[0];
      const coef piv = reinterpret_cast<const coef *>(sl)[64];
      const val zright = A::shfl_down(zmine, 1); // z_{i,k+1}, the previous step of lane + 1
      const int i = T - 1 - t - lane;
      if (act && i >= 0 && i < nr) {
        val sv = A::mul(cc[nr + i], zmine);
        if (up) sv = A::fma(cc[3 * nr + i], zright, sv);
        const val z = A::fma(piv, sv, yv);
        zmine = z;
        dl[(i & 31) * 32 + lane] = A::mul(cc[2 * nr + i], z);
      }
      // plane pd is complete once lane 0 has run it (this step); each
      // lane stores its own column of it from the delay line
      const int pd = T - 1 - t;
      if (act && pd < nr) A::stv(w + c0 + (size_t)pd * plane, dl[(pd & 31) * 32 + lane]);
    }
    cp_async_wait<0>();
  }
  const double prr = block_sum<NT>(A::d_get(arr), red);
  const double prho = block_sum<NT>(A::d_get(arho), red);
  if (tid == 0) {
    P.part_c[2 * blockIdx.x] = prr;
    P.part_c[2 * blockIdx.x + 1] = prho;
    __threadfence();
    const unsigned prev = atomicAdd(&stt->ticket_b, 1u);
    s_last = (prev == (unsigned)(P.tiles_c - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double rr = block_sum_array<NT>(P.part_c, P.tiles_c, 2, red);
  const double rho = block_sum_array<NT>(P.part_c + 1, P.tiles_c, 2, red);
  if (tid == 0) {
    if (setup) {
      setup_out[0] = rr;
      setup_out[1] = rho;
    } else {
      close_iteration(P, stt, kit, rr, rho);
    }
    stt->ticket_b = 0u;
    __threadfence();
  }
}

} // namespace pot3d
