// Set-up, finish, FP64 residual, refinement and field kernels.  None of
// these runs inside the PCG iteration; they run once per solve (or once per
// refinement step).
#pragma once
#include "kernels.cuh"

namespace pot3d {

// Right-hand side of the inner boundary (Eq. 2): b_{0,j,k} = -S_j Br_{j,k}
// with S_j = r0^2 sin(th_j) dth_j dphi (the inner face area).  Partials per
// block: sum b^2 and sum Dinv b^2.
template <int NT>
__global__ void __launch_bounds__(NT)
    k_bstats(const double *__restrict__ br, const double *__restrict__ S,
             const double *__restrict__ c64, int nr, int nt, int np, double *part) {
  __shared__ double red[NT / 32];
  const size_t R = (size_t)nr * nt;
  const size_t n0 = (size_t)nt * np;
  double s2 = 0.0, sw = 0.0;
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n0; e += (size_t)gridDim.x * NT) {
    const int j = (int)(e / np);
    const double b = -S[j] * br[e];
    s2 = fma(b, b, s2);
    sw = fma(c64[C64_DINV * R + j] * b, b, sw);
  }
  const double t2 = block_sum<NT>(s2, red);
  const double tw = block_sum<NT>(sw, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t2;
    part[2 * blockIdx.x + 1] = tw;
  }
}

// Sums [n] pairs of partials in a fixed order into out[0..1].
template <int NT>
__global__ void __launch_bounds__(NT) k_sum_pairs(const double *part, int n, double *out) {
  __shared__ double red[NT / 32];
  const double a = block_sum_array<NT>(part, n, 2, red);
  const double b = block_sum_array<NT>(part + 1, n, 2, red);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

// Starts a PCG solve from sums[0] = ||b||^2, sums[1] = sum Dinv b^2 of the
// UNSCALED right-hand side.  Chooses the power-of-two scale that brings the
// RMS of b to O(1) (exact in binary floating point; it keeps the squares of
// tiny residuals inside the float range of the double-float arithmetic).
// With x0, sums[2], sums[3] hold ||r0||^2 and sum Dinv r0^2 of the unscaled
// initial residual.
static __global__ void k_start(SolveState *st, const double *sums, double n0, double tol, int maxit,
                               int use_x0, double forced_scale, double *hist) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double bb = sums[0];
  double scale = 1.0;
  if (!isfinite(bb) || (use_x0 && !isfinite(sums[2]))) {
    st->scale = 1.0;
    st->bb = bb;
    st->iter = 0;
    st->relres = bb;
    st->status = ST_BREAKDOWN;
    st->ticket_a = st->ticket_b = 0u;
    return;
  }
  if (forced_scale > 0.0) {
    scale = forced_scale;
  } else if (bb > 0.0) {
    const double rms = sqrt(bb / n0);
    scale = ldexp(1.0, -ilogb(rms));
  }
  st->scale = scale;
  st->bb = bb * scale * scale;
  st->tol = tol;
  st->maxit = maxit;
  st->iter = 0;
  st->alpha[0] = st->alpha[1] = 0.0;
  st->beta[0] = st->beta[1] = 0.0;
  st->sigma = 0.0;
  st->rr = 0.0;
  st->ticket_a = st->ticket_b = 0u;
  st->pad_ = 0;
  const double rr = use_x0 ? sums[2] : bb;
  st->rho = (use_x0 ? sums[3] : sums[1]) * scale * scale;
  if (bb == 0.0) {
    st->relres = 0.0;
    st->status = ST_CONVERGED;
    if (hist) hist[0] = 0.0;
    return;
  }
  const double relres = sqrt(rr * scale * scale) / sqrt(st->bb);
  st->relres = relres;
  st->status = (relres <= tol) ? ST_CONVERGED : ST_RUNNING;
  if (hist) hist[0] = relres;
}

// rho of the state from sums[1] (phi-line start: r . T^-1 r of r_0).
static __global__ void k_set_rho(SolveState *st, const double *sums) {
  if (threadIdx.x == 0 && blockIdx.x == 0) st->rho = sums[1];
}

// Residual replacement of the refinement loop (reliable update): the inner
// PCG stopped after iteration K; its correction was folded into x64, the
// FP64 residual recomputed and scaled into r32 (sums: ||r32||^2 and
// sum Dinv r32^2).  The iteration continues from K with the search
// direction kept: the x~ term of iteration K is void (alpha_K = 0, x~ = 0)
// and beta_K = rho_new / rho_{K-1} * (s_old / s_new) absorbs the change of
// scale of p~.
static __global__ void k_resume(SolveState *st, const double *sums, double ratio, double tol,
                                int seg_cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int K = st->iter;
  st->maxit = K + seg_cap; // a segment that stalls ends on the cap and restarts
  const double bb = sums[0], rho = sums[1];
  st->alpha[K & 1] = 0.0;
  st->beta[K & 1] = rho / st->rho * ratio;
  st->rho = rho;
  st->bb = bb;
  st->tol = tol;
  st->relres = 1.0;
  st->ticket_a = st->ticket_b = 0u;
  st->status = (bb > 0.0 && isfinite(bb)) ? ST_RUNNING : ST_CONVERGED;
}

// r (plane 0, padded) = scale * b.
template <class A>
__global__ void k_write_rhs(const double *__restrict__ br, const double *__restrict__ S, int nt,
                            int np, int pitch, const SolveState *st, typename A::st *r) {
  const double scale = __ldcg(&st->scale);
  const size_t n0 = (size_t)nt * np;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n0;
       e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / np), k = (int)(e - (size_t)j * np);
    A::stv(r + (size_t)j * pitch + k, A::from_double(-S[j] * br[e] * scale));
  }
}

// FP64 7-point operator (Eq. 4) on x stored with row pitch xpitch:
//   mode 0: out = b - L x   (b from Br on plane 0; br may be null for b = 0)
//   mode 1: out = L x
// out has row pitch opitch.  Per-block partials: sum out^2, sum Dinv out^2.
template <int NT>
__global__ void __launch_bounds__(NT)
    k_op64(const double *__restrict__ x, int xpitch, const double *__restrict__ br,
           const double *__restrict__ S, const double *__restrict__ c64, int nr, int nt, int np,
           int mode, double *__restrict__ out, int opitch, double *part) {
  __shared__ double red[NT / 32];
  const size_t R = (size_t)nr * nt;
  const size_t n = R * np;
  const size_t xplane = (size_t)nt * xpitch;
  double s2 = 0.0, sw = 0.0;
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.x * NT) {
    const size_t row = e / np;
    const int k = (int)(e - row * np);
    const int i = (int)(row / nt), j = (int)(row - (size_t)i * nt);
    const size_t xc = (size_t)i * xplane + (size_t)j * xpitch;
    const double v = x[xc + k];
    double lx = c64[C64_D * R + row] * v;
    if (i + 1 < nr) lx = fma(-c64[C64_RP * R + row], x[xc + xplane + k], lx);
    if (i > 0) lx = fma(-c64[C64_RM * R + row], x[xc - xplane + k], lx);
    if (j + 1 < nt) lx = fma(-c64[C64_TP * R + row], x[xc + xpitch + k], lx);
    if (j > 0) lx = fma(-c64[C64_TM * R + row], x[xc - xpitch + k], lx);
    const int kp = (k + 1 == np) ? 0 : k + 1, km = (k == 0) ? np - 1 : k - 1;
    lx = fma(-c64[C64_PH * R + row], x[xc + kp] + x[xc + km], lx);
    double o;
    if (mode == 0) {
      const double b = (i == 0 && br) ? -S[j] * br[(size_t)j * np + k] : 0.0;
      o = b - lx;
    } else {
      o = lx;
    }
    if (out) out[(size_t)i * nt * opitch + (size_t)j * opitch + k] = o;
    s2 = fma(o, o, s2);
    sw = fma(c64[C64_DINV * R + row] * o, o, sw);
  }
  const double t2 = block_sum<NT>(s2, red);
  const double tw = block_sum<NT>(sw, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t2;
    part[2 * blockIdx.x + 1] = tw;
  }
}

// Initial guess: r = scale * r64 (padded FP64, the unscaled b - L x0) and
// x~ = scale * D x0 (x0 dense).
template <class A>
__global__ void k_x0_setup(const double *__restrict__ r64, const double *__restrict__ x0,
                           const double *__restrict__ c64, int nr, int nt, int np, int pitch,
                           const SolveState *st, typename A::st *r, typename A::st *x) {
  const double scale = __ldcg(&st->scale);
  const size_t R = (size_t)nr * nt, n = R * np;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t row = e / np;
    const int k = (int)(e - row * np);
    const size_t o = row * pitch + k;
    A::stv(r + o, A::from_double(scale * r64[o]));
    A::stv(x + o, A::from_double(scale * c64[C64_D * R + row] * x0[e]));
  }
}

// phi (dense) = Dinv (x~ + alpha_K p~_K) / scale, K = completed iterations.
// The matvec of iteration k applies the x~ term of iteration k-1, so x~
// lacks the last term unless the solve stopped inside a matvec (breakdown:
// that matvec already applied it and iteration K+1 never completed).
template <class A>
__global__ void k_finish(const ProbDev *probs, const double *__restrict__ c64, double *phi,
                         int add_last) {
  const ProbDev &P = probs[0];
  const SolveState *st = P.st;
  const int K = __ldcg(&st->iter);
  const int status = __ldcg(&st->status);
  const bool add = add_last && K > 0 && status != ST_BREAKDOWN;
  const double alpha = add ? __ldcg(&st->alpha[K & 1]) : 0.0;
  const double inv_scale = 1.0 / __ldcg(&st->scale);
  const typename A::st *x = static_cast<const typename A::st *>(P.x);
  const typename A::st *p = static_cast<const typename A::st *>((K & 1) ? P.p1 : P.p0);
  const size_t R = (size_t)P.nr * P.nt, n = R * P.np;
  const typename A::scal a = A::scal_from(alpha);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t row = e / P.np;
    const int k = (int)(e - row * P.np);
    const size_t o = row * P.pitch + k;
    typename A::val xv = A::ld(x + o);
    if (add) xv = A::fma(a, A::ld(p + o), xv);
    phi[e] = A::to_double(xv) * c64[C64_DINV * R + row] * inv_scale;
  }
}

// Refinement: r32 = scale * r64 (padded to padded), with per-block
// partials of ||r32||^2 and sum Dinv32 r32^2 computed from the stored floats.
template <int NT>
__global__ void __launch_bounds__(NT)
    k_inner_rhs(const double *__restrict__ r64, const float *__restrict__ dinv32, int nr, int nt,
                int ntp, int np, int pitch, double scale, float *r32, double *part) {
  __shared__ double red[NT / 32];
  const size_t R = (size_t)nr * nt, n = R * np;
  double s2 = 0.0, sw = 0.0;
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.x * NT) {
    const size_t row = e / np;
    const int k = (int)(e - row * np);
    const size_t o = row * pitch + k;
    const float f = __double2float_rn(scale * r64[o]);
    r32[o] = f;
    const double d = (double)f;
    const size_t i = row / nt, j = row - i * nt;
    s2 = fma(d, d, s2);
    sw = fma((double)dinv32[i * ntp + j] * d, d, sw);
  }
  const double t2 = block_sum<NT>(s2, red);
  const double tw = block_sum<NT>(sw, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t2;
    part[2 * blockIdx.x + 1] = tw;
  }
}

// Refinement update x64 += Dinv (x~32 + alpha p~32) / scale (FP64).
static __global__ void k_refine_update(const ProbDev *probs, const double *__restrict__ c64,
                                double *x64, double inv_scale) {
  const ProbDev &P = probs[0];
  const SolveState *st = P.st;
  const int K = __ldcg(&st->iter);
  const int status = __ldcg(&st->status);
  const bool add = K > 0 && status != ST_BREAKDOWN;
  const double alpha = add ? __ldcg(&st->alpha[K & 1]) : 0.0;
  const float *x = static_cast<const float *>(P.x);
  const float *p = static_cast<const float *>((K & 1) ? P.p1 : P.p0);
  const size_t R = (size_t)P.nr * P.nt, n = R * P.np;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t row = e / P.np;
    const int k = (int)(e - row * P.np);
    const size_t o = row * P.pitch + k;
    double d = (double)x[o];
    if (add) d = fma(alpha, (double)p[o], d);
    x64[o] = fma(d * c64[C64_DINV * R + row], inv_scale, x64[o]);
  }
}

// Copy a padded FP64 vector to the dense layout (and back).
static __global__ void k_unpad(const double *__restrict__ src, int spitch, double *__restrict__ dst,
                        int dpitch, size_t rows, int np) {
  const size_t n = rows * np;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t row = e / np;
    const int k = (int)(e - row * np);
    dst[row * dpitch + k] = src[row * spitch + k];
  }
}

// ------------------------------------------------- closed-wall boundary
// With the closed wall (Br = 0 at the outer face, Sec. 2.1) the operator's
// null space is the constants: the right-hand side must carry zero net flux
// and the solution is fixed up to a constant.

// Block partials of the inner-face flux sum_jk S_j Br_jk, as pairs (flux, 0)
// for k_sum_pairs.
template <int NT>
__global__ void __launch_bounds__(NT)
    k_flux(const double *__restrict__ br, const double *__restrict__ S, int nt, int np,
           double *part) {
  __shared__ double red[NT / 32];
  const size_t n0 = (size_t)nt * np;
  double f = 0.0;
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n0; e += (size_t)gridDim.x * NT) {
    const int j = (int)(e / np);
    f = fma(S[j], br[e], f);
  }
  const double t = block_sum<NT>(f, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

// out = br - sum[0] * inv_area: Br without its area-weighted mean (the
// discrete monopole), so that b has zero net flux.
static __global__ void k_shift(const double *__restrict__ br, double *__restrict__ out, size_t n0,
                               const double *sum, double inv_area) {
  const double m = __ldcg(sum) * inv_area;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n0;
       e += (size_t)gridDim.x * blockDim.x)
    out[e] = br[e] - m;
}

// Block partials of sum x (dense, n values), as pairs (sum, 0).
template <int NT>
__global__ void __launch_bounds__(NT) k_sum_partials(const double *__restrict__ x, size_t n,
                                                     double *part) {
  __shared__ double red[NT / 32];
  double s = 0.0;
  for (size_t e = blockIdx.x * (size_t)NT + threadIdx.x; e < n; e += (size_t)gridDim.x * NT)
    s += x[e];
  const double t = block_sum<NT>(s, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t;
    part[2 * blockIdx.x + 1] = 0.0;
  }
}

// The closed-wall gauge: x -= sum[0] / n (zero mean over the cells).
static __global__ void k_sub_mean(double *__restrict__ x, size_t n, const double *sum, double inv_n) {
  const double m = __ldcg(sum) * inv_n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    x[e] -= m;
}

// ------------------------------------------------------------------ field
// Pole averages (Eq. 3): poles[2 i] = mean_k Phi[i][0][k] (north),
// poles[2 i + 1] = mean_k Phi[i][nt-1][k] (south).  One block per (i, pole).
template <int NT>
__global__ void __launch_bounds__(NT)
    k_pole_avg(const double *__restrict__ phi, int nr, int nt, int np, double *poles) {
  __shared__ double red[NT / 32];
  const int i = blockIdx.x >> 1, pole = blockIdx.x & 1;
  const int j = pole ? nt - 1 : 0;
  const double *row = phi + ((size_t)i * nt + j) * np;
  double s = 0.0;
  for (int k = threadIdx.x; k < np; k += NT) s += row[k];
  const double t = block_sum<NT>(s, red);
  if (threadIdx.x == 0) poles[2 * i + pole] = t / (double)np;
}

// Field tables (FP64):
//   irs [nr+1]: 1 / (r-spacing across radial face f); f = nr uses the
//               mirror ghost of the source surface, f = 0 is unused.
//   its [nt+1]: 1 / (theta-spacing across colatitude face f); f = 0 and nt
//               use the mirror across the pole.
//   irc [nr]  : 1 / r_i          isd [nt]: 1 / (sin th_j dphi)
//   wt [nr*nt]: its[j] / r_i (colatitude faces j >= 1 of row (i, j))
//   wp [nr*nt]: 1 / (r_i sin th_j dphi) (phi faces of row (i, j))
//   wpole [2*nr]: 2 its[0] / r_i, 2 its[nt] / r_i (the two pole faces)
struct FieldTabs {
  const double *irs, *its, *irc, *isd;
  const double *wt, *wp, *wpole;
  int closed; // closed wall: Br = 0 on the outer face
};

// B = grad Phi on the staggered faces; see the header for the layout.
// One thread per cell (i, j, k) in C order writes every face the cell owns:
// the radial face below it (i), the colatitude face north of it (j) and the
// phi face after it; the last radial layer also writes the outer face and
// the last colatitude row the south pole face.  Consecutive threads take
// consecutive k, so every read of Phi (the cell, its lower radial and
// northern neighbours, its phi successor) and every write is coalesced, and
// Phi comes from HBM once (the neighbouring rows were read just before and
// sit in L2).  GB300's FP64 unit, not HBM, bounds this kernel: each face
// costs one FP64 subtraction and one multiplication by a per-row factor
// from the tables (6 FP64 operations per cell).  Index arithmetic in 32
// bits (the host checks n < 2^31).
constexpr int kFieldThreads = 256;
static __global__ void __launch_bounds__(kFieldThreads)
    k_field(const double *__restrict__ phi, const double *__restrict__ br,
            const double *__restrict__ poles, FieldTabs T, int nr, int nt, int np,
            double *__restrict__ B) {
  const unsigned n = (unsigned)nr * nt * np, rplane = (unsigned)nt * np;
  double *const Bt = B + (size_t)(nr + 1) * rplane; // colatitude faces [nr][nt+1][np]
  double *const Bp = Bt + (size_t)nr * (nt + 1) * np;
  for (unsigned e = blockIdx.x * kFieldThreads + threadIdx.x; e < n;
       e += gridDim.x * kFieldThreads) {
    const unsigned q = e / np, k = e - q * np, i = q / nt, j = q - i * nt;
    const double v = phi[e];
    // ghost chosen so that dPhi/dr = Br on the inner face (Eq. 2)
    if (i == 0) B[e] = br[(size_t)j * np + k];
    else B[e] = (v - phi[e - rplane]) * T.irs[i];
    const size_t ot = ((size_t)i * (nt + 1) + j) * np + k;
    // ghost 2 avg - Phi across the north pole: the face value is the ring's
    // phi-average (Eq. 3)
    if (j == 0) Bt[ot] = (v - poles[2 * i]) * T.wpole[2 * i];
    else Bt[ot] = (v - phi[e - np]) * T.wt[q];
    const unsigned ep = (k + 1 == (unsigned)np) ? e + 1 - np : e + 1;
    Bp[e] = (phi[ep] - v) * T.wp[q];
    // source surface: ghost -Phi (Phi = 0 there); closed wall: ghost Phi
    if (i == (unsigned)nr - 1) B[e + rplane] = T.closed ? 0.0 : (-2.0 * v) * T.irs[nr];
    if (j == (unsigned)nt - 1) Bt[ot + np] = (poles[2 * i + 1] - v) * T.wpole[2 * i + 1];
  }
}

} // namespace pot3d
