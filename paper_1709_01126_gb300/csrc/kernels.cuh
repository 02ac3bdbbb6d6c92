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
//              relative residual, the convergence flag and beta.
// Every reduction is deterministic: each work item writes its partial to a
// fixed slot, and the last block sums the slots in a fixed order.
#pragma once
#include "arith.cuh"

namespace pot3d {

enum : int { ST_RUNNING = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_MAXIT = 3 };

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
  int iter;        // completed iterations
  int maxit;
  int status;
  unsigned ticket_a, ticket_b;
  int pad_;
};

// One problem (one solve) as the kernels see it.
struct ProbDev {
  int nr, nt, np, pitch;
  int nJ, nK, ic, nI; // matvec tiles along theta, phi; i-chunk length; i-chunks
  int tiles_a;        // nJ*nK*nI
  int rows_b;         // rows per update work item
  int tiles_b;
  int pad_;
  long long plane; // nt*pitch
  void *x, *r, *p0, *p1, *q;
  const void *coef;  // scaled metric table [6][nr*nt]: Dinv, n_r+, n_r-, n_t+, n_t-, n_ph
  double *part_a;    // [tiles_a]
  double *part_b;    // [2*tiles_b]
  SolveState *st;
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

// ------------------------------------------------------------ k_matvec
// Work item = (problem, tile).  A tile is TJ theta rows x TK = 32*VK phi
// columns, marching over an i-chunk [i0, i1).  Each warp owns one theta row;
// lane l owns phi columns k0 + l + 32 v.  Per plane the block stages p~_new
// on the (TJ+2) x (TK+2) halo region in shared memory (three rotating plane
// buffers, one barrier per plane); the r-neighbours come from registers.
template <class A, int TJ, int VK>
__global__ void __launch_bounds__(32 * TJ)
    k_matvec(const ProbDev *__restrict__ probs, const int2 *__restrict__ work, int nwork) {
  using val = typename A::val;
  using st = typename A::st;
  using coef = typename A::coef;
  constexpr int TK = 32 * VK, RW = TK + 2, RH = TJ + 2, RC = RW * RH, NT = 32 * TJ;
  __shared__ val sm[3][RH][RW];
  __shared__ double red[NT / 32];
  __shared__ int s_last;
  const int lane = threadIdx.x, wy = threadIdx.y, tid = wy * 32 + lane;

  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    const ProbDev &P = probs[wi.x];
    SolveState *stt = P.st;
    if (ldcg(&stt->status) != ST_RUNNING) continue;
    const int kit = ldcg(&stt->iter) + 1; // this iteration
    const int t = wi.y;
    const int nr = P.nr, nt = P.nt, np = P.np, pitch = P.pitch;
    const int tk = t % P.nK, tj = (t / P.nK) % P.nJ, ci = t / (P.nK * P.nJ);
    const int j0 = tj * TJ, k0 = tk * TK, i0 = ci * P.ic;
    const int i1 = min(nr, i0 + P.ic);
    const st *__restrict__ r = static_cast<const st *>(P.r);
    const st *__restrict__ pold = static_cast<const st *>((kit & 1) ? P.p0 : P.p1);
    st *__restrict__ pnew = static_cast<st *>((kit & 1) ? P.p1 : P.p0);
    st *__restrict__ x = static_cast<st *>(P.x);
    st *__restrict__ q = static_cast<st *>(P.q);
    const coef *__restrict__ cf = static_cast<const coef *>(P.coef);
    const size_t R = (size_t)nr * nt;
    const typename A::scal beta = A::scal_from(kit > 1 ? ldcg(&stt->beta[(kit - 1) & 1]) : 0.0);
    const typename A::scal alpha_prev =
        A::scal_from(kit > 1 ? ldcg(&stt->alpha[(kit - 1) & 1]) : 0.0);
    const bool first = (kit == 1);

    // Stage plane ip into buffer b: p~_new = r + beta p~_old on the halo
    // region; the owning tile also stores p~_new and updates x~.
    auto load_plane = [&](int ip, int b, bool own) {
      const size_t pbase = (size_t)ip * P.plane;
      for (int c = tid; c < RC; c += NT) {
        const int rr = c / RW, cc = c - rr * RW;
        const int jj = j0 - 1 + rr, kk = k0 - 1 + cc;
        val v = A::zero();
        if (jj >= 0 && jj < nt && kk <= np) {
          const int km = kk < 0 ? kk + np : (kk >= np ? kk - np : kk);
          const size_t off = pbase + (size_t)jj * pitch + km;
          const val rv = A::ld(r + off);
          if (first) {
            v = rv;
          } else {
            const val po = A::ld(pold + off);
            v = A::fma(beta, po, rv);
            if (own && rr >= 1 && rr <= TJ && cc >= 1 && cc <= TK && kk < np) {
              const val xv = A::ld(x + off);
              A::stv(x + off, A::fma(alpha_prev, po, xv));
            }
          }
          if (own && rr >= 1 && rr <= TJ && cc >= 1 && cc <= TK && kk < np) A::stv(pnew + off, v);
        }
        sm[b][rr][cc] = v;
      }
    };

    const int j = j0 + wy;
    const bool jv = j < nt;
    typename A::dacc tacc = A::d_init();
    val prv[VK], cur[VK];
    int bp = 0, bc = 1, bn = 2;
    if (i0 > 0) load_plane(i0 - 1, bp, false);
    load_plane(i0, bc, true);
    __syncthreads();
#pragma unroll
    for (int v = 0; v < VK; v++) {
      prv[v] = (i0 > 0) ? sm[bp][wy + 1][lane + 32 * v + 1] : A::zero();
      cur[v] = sm[bc][wy + 1][lane + 32 * v + 1];
    }
    for (int i = i0; i < i1; i++) {
      // metric coefficients of row (i, j); uniform across the warp
      coef cDi{}, cRp{}, cRm{}, cTp{}, cTm{}, cPh{};
      if (jv) {
        const size_t row = (size_t)i * nt + j;
        cDi = cf[row];
        cRp = cf[R + row];
        cRm = cf[2 * R + row];
        cTp = cf[3 * R + row];
        cTm = cf[4 * R + row];
        cPh = cf[5 * R + row];
      }
      const bool has_next = (i + 1 < nr);
      if (has_next) load_plane(i + 1, bn, i + 1 < i1);
      __syncthreads();
      if (jv) {
        typename A::dacc racc = A::d_init();
        const size_t rowoff = (size_t)i * P.plane + (size_t)j * pitch;
#pragma unroll
        for (int v = 0; v < VK; v++) {
          const int cc = lane + 32 * v + 1;
          const val nxt = has_next ? sm[bn][wy + 1][cc] : A::zero();
          typename A::sacc s = A::s_init(cur[v]);
          A::s_add(s, cRp, nxt);
          A::s_add(s, cRm, prv[v]);
          A::s_add(s, cTp, sm[bc][wy + 2][cc]);
          A::s_add(s, cTm, sm[bc][wy][cc]);
          A::s_add(s, cPh, sm[bc][wy + 1][cc - 1]);
          A::s_add(s, cPh, sm[bc][wy + 1][cc + 1]);
          const val qv = A::s_get(s);
          const int kk = k0 + cc - 1;
          if (kk < np) {
            A::stv(q + rowoff + kk, qv);
            A::d_add(racc, cur[v], qv);
          }
          prv[v] = cur[v];
          cur[v] = nxt;
        }
        A::d_addw(tacc, cDi, racc);
      }
      const int tmp = bp;
      bp = bc;
      bc = bn;
      bn = tmp;
    }

    const double mine = jv ? A::d_get(tacc) : 0.0;
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
// Work item = (problem, block of rows_b phi rows).  Warps take rows, lanes
// take 16-byte vectors along phi.  r -= alpha q; per row s = sum r^2, then
// ||r||^2 += s and rho += D^-1 s.  The last block closes the iteration.
template <class A, int NT>
__global__ void __launch_bounds__(NT)
    k_update(const ProbDev *__restrict__ probs, const int2 *__restrict__ work, int nwork) {
  using val = typename A::val;
  using st = typename A::st;
  using coef = typename A::coef;
  constexpr int V = A::kVec, NW = NT / 32;
  __shared__ double red[NW];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5, tid = threadIdx.x;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    const ProbDev &P = probs[wi.x];
    SolveState *stt = P.st;
    if (ldcg(&stt->status) != ST_RUNNING) continue;
    const int kit = ldcg(&stt->iter) + 1;
    const int t = wi.y;
    const int nt = P.nt, np = P.np, pitch = P.pitch;
    const size_t R = (size_t)P.nr * nt;
    const int row0 = t * P.rows_b, row1 = min((int)R, row0 + P.rows_b);
    st *__restrict__ r = static_cast<st *>(P.r);
    const st *__restrict__ q = static_cast<const st *>(P.q);
    const coef *__restrict__ cf = static_cast<const coef *>(P.coef);
    const typename A::scal nalpha = A::scal_from(-ldcg(&stt->alpha[kit & 1]));
    typename A::dacc arr = A::d_init(), arho = A::d_init();
    for (int row = row0 + wy; row < row1; row += NW) {
      const int i = row / nt, j = row - i * nt;
      const coef dinv = cf[row];
      const size_t base = (size_t)i * P.plane + (size_t)j * pitch;
      typename A::dacc s = A::d_init();
      for (int k = lane * V; k < np; k += 32 * V) {
        val rv[V], qv[V];
        A::ldv(r + base + k, rv);
        A::ldv(q + base + k, qv);
#pragma unroll
        for (int u = 0; u < V; u++) {
          rv[u] = A::fma(nalpha, qv[u], rv[u]);
          if (k + u < np) A::d_add(s, rv[u], rv[u]);
        }
        A::stvv(r + base + k, rv);
      }
      // ||r||^2 += s ; rho += Dinv * s
      A::d_merge(arr, s);
      A::d_addw(arho, dinv, s);
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
        const double relres = sqrt(rr) / sqrt(stt->bb);
        stt->relres = relres;
        stt->iter = kit;
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
        stt->ticket_b = 0u;
        __threadfence();
      }
    }
    __syncthreads();
  }
}

} // namespace pot3d
