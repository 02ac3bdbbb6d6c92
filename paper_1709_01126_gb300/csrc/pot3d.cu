// libpot3d: plan, solve, refinement and field entry points (include/pot3d.h).
//
// Host side of the GB300 potential-field solver.  The plan builds the mesh
// and the per-(r, theta) metric tables in FP64 on the host (Sec. 2.2), uploads
// them once, and keeps every vector resident on the device for the whole
// solve (Sec. 3.1: data stay on the accelerator; the host only polls a few
// bytes of solver state between chunks of iterations).
#include "pot3d.h"
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

using namespace pot3d;

static thread_local int g_last_error = POT3D_OK;

namespace pot3d {

int fail(int code) {
  g_last_error = code;
  return code;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return POT3D_OK;
  if (e == cudaErrorMemoryAllocation) return fail(POT3D_ERR_OOM);
  return fail(POT3D_ERR_CUDA);
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// ------------------------------------------------------------- the mesh
// Radial faces: explicit, or r0 + cumulative widths dr_1 g^i (g = r_ratio),
// the last face pinned to r1.  Colatitude faces: explicit or j pi / nt.
static int build_mesh(Plan *P, const pot3d_grid_t *g) {
  const int nr = g->nr, nt = g->nt, np = g->np;
  P->rf.resize(nr + 1);
  P->tf.resize(nt + 1);
  if (g->r_faces) {
    for (int i = 0; i <= nr; i++) P->rf[i] = g->r_faces[i];
  } else {
    const double r0 = g->r0, r1 = g->r1, ratio = g->r_ratio;
    if (!(r1 > r0) || !(r0 > 0.0) || !(ratio > 0.0) || !std::isfinite(ratio))
      return POT3D_ERR_INVALID_ARG;
    double w = (ratio == 1.0) ? (r1 - r0) / nr : (r1 - r0) * (ratio - 1.0) / (std::pow(ratio, nr) - 1.0);
    P->rf[0] = r0;
    for (int i = 0; i < nr; i++) {
      P->rf[i + 1] = P->rf[i] + w;
      w *= ratio;
    }
    P->rf[nr] = r1;
  }
  if (g->t_faces) {
    for (int j = 0; j <= nt; j++) P->tf[j] = g->t_faces[j];
  } else {
    for (int j = 0; j <= nt; j++) P->tf[j] = M_PI * (double)j / (double)nt;
    P->tf[0] = 0.0;
    P->tf[nt] = M_PI;
  }
  for (int i = 0; i < nr; i++)
    if (!(P->rf[i + 1] > P->rf[i]) || !std::isfinite(P->rf[i + 1])) return POT3D_ERR_INVALID_ARG;
  if (!(P->rf[0] > 0.0)) return POT3D_ERR_INVALID_ARG;
  for (int j = 0; j < nt; j++)
    if (!(P->tf[j + 1] > P->tf[j])) return POT3D_ERR_INVALID_ARG;
  if (P->tf[0] < 0.0 || P->tf[nt] > M_PI + 1e-12) return POT3D_ERR_INVALID_ARG;
  P->rc.resize(nr);
  P->drc.resize(nr);
  P->tc.resize(nt);
  P->dtc.resize(nt);
  for (int i = 0; i < nr; i++) {
    P->rc[i] = 0.5 * (P->rf[i] + P->rf[i + 1]);
    P->drc[i] = P->rf[i + 1] - P->rf[i];
  }
  for (int j = 0; j < nt; j++) {
    P->tc[j] = 0.5 * (P->tf[j] + P->tf[j + 1]);
    P->dtc[j] = P->tf[j + 1] - P->tf[j];
  }
  P->dphi = 2.0 * M_PI / np;
  return POT3D_OK;
}

// --------------------------------------------------------- metric tables
// Volume-weighted operator of Eq. 4 (symmetric form of the Sec. 2.2
// stencil with the spherical metric factors):
//   c^r  on face r_{i+1/2}  = r_{i+1/2}^2 sin th_j dth_j dphi / (r_{i+1} - r_i)
//   c^th on face th_{j+1/2} = dr_i sin th_{j+1/2} dphi / (th_{j+1} - th_j)
//   c^ph                    = dr_i dth_j / (sin th_j dphi)
// Boundary faces: the inner face carries the Br flux (right-hand side), the
// source surface couples to the ghost -Phi (adds 2 c^r to D; the closed wall
// carries no flux and adds nothing), the pole faces have zero area
// (sin 0 = sin pi = 0).
static void build_tables(Plan *P) {
  const int nr = P->nr, nt = P->nt;
  const size_t R = P->R;
  const double dphi = P->dphi;
  P->c64h.assign(7 * R, 0.0);
  double *D = &P->c64h[C64_D * R], *Di = &P->c64h[C64_DINV * R];
  double *cRp = &P->c64h[C64_RP * R], *cRm = &P->c64h[C64_RM * R];
  double *cTp = &P->c64h[C64_TP * R], *cTm = &P->c64h[C64_TM * R], *cPh = &P->c64h[C64_PH * R];
  std::vector<double> sc(nt), sf(nt + 1);
  for (int j = 0; j < nt; j++) sc[j] = std::sin(P->tc[j]);
  for (int j = 0; j <= nt; j++) sf[j] = (j == 0 || j == nt) ? 0.0 : std::sin(P->tf[j]);
  for (int i = 0; i < nr; i++) {
    for (int j = 0; j < nt; j++) {
      const size_t row = (size_t)i * nt + j;
      const double ang = sc[j] * P->dtc[j] * dphi;
      const double rp = P->rf[i + 1], rm = P->rf[i];
      double out = 0.0;
      if (i + 1 < nr) cRp[row] = rp * rp * ang / (P->rc[i + 1] - P->rc[i]);
      else if (!P->closed) out = 2.0 * (rp * rp * ang / (2.0 * (P->rf[nr] - P->rc[nr - 1])));
      if (i > 0) cRm[row] = rm * rm * ang / (P->rc[i] - P->rc[i - 1]);
      if (j + 1 < nt) cTp[row] = P->drc[i] * sf[j + 1] * dphi / (P->tc[j + 1] - P->tc[j]);
      if (j > 0) cTm[row] = P->drc[i] * sf[j] * dphi / (P->tc[j] - P->tc[j - 1]);
      cPh[row] = P->drc[i] * P->dtc[j] / (sc[j] * dphi);
      D[row] = cRp[row] + cRm[row] + cTp[row] + cTm[row] + 2.0 * cPh[row] + out;
      Di[row] = 1.0 / D[row];
    }
  }
  P->S.resize(nt);
  const double r0 = P->rf[0];
  double area = 0.0;
  for (int j = 0; j < nt; j++) {
    P->S[j] = r0 * r0 * sc[j] * P->dtc[j] * dphi;
    area += P->S[j];
  }
  P->inv_area = 1.0 / (area * P->np);
  // field tables
  P->irs.assign(nr + 1, 0.0);
  for (int f = 1; f < nr; f++) P->irs[f] = 1.0 / (P->rc[f] - P->rc[f - 1]);
  P->irs[nr] = 1.0 / (2.0 * (P->rf[nr] - P->rc[nr - 1]));
  P->its.assign(nt + 1, 0.0);
  for (int f = 1; f < nt; f++) P->its[f] = 1.0 / (P->tc[f] - P->tc[f - 1]);
  P->its[0] = 1.0 / (2.0 * (P->tc[0] - P->tf[0]));
  P->its[nt] = 1.0 / (2.0 * (P->tf[nt] - P->tc[nt - 1]));
  P->irc.resize(nr);
  for (int i = 0; i < nr; i++) P->irc[i] = 1.0 / P->rc[i];
  P->isd.resize(nt);
  for (int j = 0; j < nt; j++) P->isd[j] = 1.0 / (sc[j] * dphi);
  // per-row factors of the field kernel (one multiplication per face)
  P->fwt.assign(R, 0.0);
  P->fwp.assign(R, 0.0);
  P->fwpole.assign(2 * nr, 0.0);
  for (int i = 0; i < nr; i++) {
    for (int j = 0; j < nt; j++) {
      P->fwt[(size_t)i * nt + j] = P->its[j] * P->irc[i];
      P->fwp[(size_t)i * nt + j] = P->irc[i] * P->isd[j];
    }
    P->fwpole[2 * i] = 2.0 * P->its[0] * P->irc[i];
    P->fwpole[2 * i + 1] = 2.0 * P->its[nt] * P->irc[i];
  }
}

// Scaled, negated table of the iteration: Dinv, -c/D of the neighbour.
void scaled_table(const Plan *P, std::vector<double> &t) {
  const int nr = P->nr, nt = P->nt;
  const size_t R = P->R;
  const double *Di = &P->c64h[C64_DINV * R];
  t.assign(6 * R, 0.0);
  for (int i = 0; i < nr; i++) {
    for (int j = 0; j < nt; j++) {
      const size_t row = (size_t)i * nt + j;
      t[row] = Di[row];
      if (i + 1 < nr) t[R + row] = -P->c64h[C64_RP * R + row] * Di[row + nt];
      if (i > 0) t[2 * R + row] = -P->c64h[C64_RM * R + row] * Di[row - nt];
      if (j + 1 < nt) t[3 * R + row] = -P->c64h[C64_TP * R + row] * Di[row + 1];
      if (j > 0) t[4 * R + row] = -P->c64h[C64_TM * R + row] * Di[row - 1];
      t[5 * R + row] = -P->c64h[C64_PH * R + row] * Di[row];
    }
  }
}

template <class T>
static int upload(T **dst, const std::vector<T> &h) {
  if (cudaMalloc((void **)dst, sizeof(T) * std::max<size_t>(1, h.size())) != cudaSuccess) {
    cudaGetLastError();
    return POT3D_ERR_OOM;
  }
  if (!h.empty() && cudaMemcpy(*dst, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return POT3D_ERR_CUDA;
  return POT3D_OK;
}

// Device copy of the iteration table in the arithmetic's coefficient type,
// laid out [6][nr][ntp] (theta rows padded to a multiple of 4 so that every
// row of the table starts on a 16-byte boundary for the TMA).
int ensure_arith(Plan *P, int ai) {
  ArithData &A = P->ar[ai];
  if (A.ready) return POT3D_OK;
  std::vector<double> t;
  scaled_table(P, t);
  const int ntp = P->ntp;
  const size_t RP = (size_t)P->nr * ntp;
  std::vector<double> tp(6 * RP, 0.0);
  for (int m = 0; m < 6; m++)
    for (int i = 0; i < P->nr; i++)
      for (int j = 0; j < P->nt; j++)
        tp[m * RP + (size_t)i * ntp + j] = t[m * P->R + (size_t)i * P->nt + j];
  int rc = POT3D_OK;
  if (ai == AR_F64) {
    rc = upload((double **)&A.coef, tp);
  } else if (ai == AR_DF) {
    std::vector<float2> h(tp.size());
    for (size_t u = 0; u < tp.size(); u++) {
      const float hi = (float)tp[u];
      h[u] = make_float2(hi, (float)(tp[u] - (double)hi));
    }
    rc = upload((float2 **)&A.coef, h);
  } else {
    std::vector<float> h(tp.size());
    for (size_t u = 0; u < tp.size(); u++) h[u] = (float)tp[u];
    rc = upload((float **)&A.coef, h);
  }
  if (rc) return rc;
  if (cudaMalloc(&A.d_state, sizeof(SolveState)) != cudaSuccess ||
      cudaMalloc(&A.d_prob, sizeof(ProbDev)) != cudaSuccess) {
    cudaGetLastError();
    return POT3D_ERR_OOM;
  }
  cudaMemset(A.d_state, 0, sizeof(SolveState));
  rc = set_decomposition(P, ai, 0, 0, 0);
  if (rc) return rc;
  A.ready = true;
  return POT3D_OK;
}

// Phi-line table: per (i, j) ring, T = d - c (S + S^-1) with d = D_ij and
// c = c^ph_ij factors as (c / mu)(1 - mu S)(1 - mu S^-1) with
// mu + 1 / mu = d / c (the root below 1, in the form without cancellation);
// the update kernel needs mu, mu / c (rho = (mu / c) ||F r||^2),
// D mu / c (w = D z), and for the ring solve the powers mu^m and
// mu^(np mod m) of the lanes' chunk lengths (m = ceil(np / 32)) and
// 1 / (1 - mu^np).  Layout [6][nr][ntp] like the metric table.
int ensure_line(Plan *P, int ai) {
  ArithData &A = P->ar[ai];
  if (A.lcoef) return POT3D_OK;
  const int nr = P->nr, nt = P->nt, ntp = P->ntp, np = P->np;
  const int m = (np + 31) / 32, rem = np % m;
  const size_t R = P->R, RP = (size_t)nr * ntp;
  std::vector<double> t(6 * RP, 0.0);
  for (int i = 0; i < nr; i++)
    for (int j = 0; j < nt; j++) {
      const size_t row = (size_t)i * nt + j, o = (size_t)i * ntp + j;
      const double d = P->c64h[C64_D * R + row], c = P->c64h[C64_PH * R + row];
      const double mu = 2.0 * c / (d + std::sqrt((d - 2.0 * c) * (d + 2.0 * c)));
      t[o] = mu;
      t[RP + o] = mu / c;
      t[2 * RP + o] = d * (mu / c);
      t[3 * RP + o] = std::pow(mu, m);
      t[4 * RP + o] = std::pow(mu, rem);
      t[5 * RP + o] = 1.0 / (1.0 - std::pow(mu, np));
    }
  int rc;
  if (ai == AR_F64) {
    rc = upload((double **)&A.lcoef, t);
  } else {
    std::vector<float> h(t.size());
    for (size_t u = 0; u < t.size(); u++) h[u] = (float)t[u];
    rc = upload((float **)&A.lcoef, h);
  }
  return rc;
}

// Radial-line table: per theta row j, the tridiagonal T_r of every radial
// column (diagonal D_i, couplings e_i = -c^r_{i+1/2} between i and i + 1;
// e_{nr-1} = 0: the outer face is a boundary face) factored as
// L' diag(d') L'^T: l_i = e_{i-1} / d'_{i-1}, d'_i = D_i - e_{i-1} l_i.
// The kernel needs l_i, 1 / d'_i (rho), D_i / d'_i and
// l_{i+1} D_i / D_{i+1} (w = D z directly).  Layout [4][nr][ntp].
int rline_tiles(const Plan *P) {
  const long units = (long)P->nt * ((P->np + 31) / 32);
  return (int)((units + kRLineThreads / 32 - 1) / (kRLineThreads / 32));
}

int ensure_rline(Plan *P, int ai) {
  ArithData &A = P->ar[ai];
  const int tiles = rline_tiles(P);
  if (A.tiles_c < tiles) {
    cudaFree(A.part_c);
    A.part_c = nullptr;
    A.tiles_c = 0;
    if (cudaMalloc(&A.part_c, sizeof(double) * 2 * tiles) != cudaSuccess) {
      cudaGetLastError();
      return POT3D_ERR_OOM;
    }
    A.tiles_c = tiles;
  }
  if (A.rcoef) return POT3D_OK;
  const int nr = P->nr, nt = P->nt, ntp = P->ntp;
  const size_t R = P->R, RP = (size_t)nr * ntp;
  std::vector<double> t(4 * RP, 0.0);
  for (int j = 0; j < nt; j++) {
    double dprev = 0.0;
    for (int i = 0; i < nr; i++) {
      const size_t row = (size_t)i * nt + j, o = (size_t)i * ntp + j;
      const double D = P->c64h[C64_D * R + row];
      const double e = i > 0 ? -P->c64h[C64_RP * R + row - nt] : 0.0;
      const double l = i > 0 ? e / dprev : 0.0;
      const double dp = D - e * l;
      t[o] = l;
      t[RP + o] = 1.0 / dp;
      t[2 * RP + o] = D / dp;
      dprev = dp;
    }
    for (int i = 0; i + 1 < nr; i++) {
      const size_t row = (size_t)i * nt + j, o = (size_t)i * ntp + j;
      t[3 * RP + o] = t[o + ntp] * P->c64h[C64_D * R + row] / P->c64h[C64_D * R + row + nt];
    }
  }
  int rc;
  if (ai == AR_F64) {
    rc = upload((double **)&A.rcoef, t);
  } else {
    std::vector<float> h(t.size());
    for (size_t u = 0; u < t.size(); u++) h[u] = (float)t[u];
    rc = upload((float **)&A.rcoef, h);
  }
  return rc;
}

// PC2 (subdomain ILU(0), k_ilu): boxes of nr x 1 x 32 cells.  Table, in
// the arithmetic's coefficient type: [4][nr][ntp] c^r_{i-1/2}, c^r_{i+1/2},
// D and c^ph per (i, j) (zero where the face is a boundary face), then the
// pivot inverses skewed for the wavefront, [nt][nr + 31][32] with entry
// (j, t, kk) = 1 / p(t - kk, j, kk) (0 outside 0 <= t - kk < nr), where
//     p(i, j, kk) = D_ij - [i > 0] (c^r_{i-1/2,j})^2 / p(i-1, j, kk)
//                        - [kk > 0] (c^ph_ij)^2 / p(i, j, kk-1)
// (ILU(0) of the 7-point pattern changes only the diagonal; a box's cells
// k0 + kk have the pivots of column kk whatever the box's width).
int ilu_tiles(const Plan *P) {
  const long units = (long)P->nt * ((P->np + 31) / 32);
  return (int)((units + kIluThreads / 32 - 1) / (kIluThreads / 32));
}

int ensure_ilu(Plan *P, int ai) {
  ArithData &A = P->ar[ai];
  const int tiles = ilu_tiles(P);
  if (A.tiles_i < tiles) {
    cudaFree(A.part_i);
    A.part_i = nullptr;
    A.tiles_i = 0;
    if (cudaMalloc(&A.part_i, sizeof(double) * 2 * tiles) != cudaSuccess) {
      cudaGetLastError();
      return POT3D_ERR_OOM;
    }
    A.tiles_i = tiles;
  }
  if (A.icoef) return POT3D_OK;
  const int nr = P->nr, nt = P->nt, ntp = P->ntp, T = nr + 31;
  const size_t R = P->R, RP = (size_t)nr * ntp;
  std::vector<double> t(4 * RP + (size_t)nt * T * 32, 0.0);
  std::vector<double> piv((size_t)nr * 32);
  for (int j = 0; j < nt; j++) {
    for (int i = 0; i < nr; i++) {
      const size_t row = (size_t)i * nt + j, o = (size_t)i * ntp + j;
      t[o] = P->c64h[C64_RM * R + row];
      t[RP + o] = P->c64h[C64_RP * R + row];
      t[2 * RP + o] = P->c64h[C64_D * R + row];
      t[3 * RP + o] = P->c64h[C64_PH * R + row];
    }
    for (int i = 0; i < nr; i++) {
      const size_t row = (size_t)i * nt + j;
      const double D = P->c64h[C64_D * R + row], crm = P->c64h[C64_RM * R + row],
                   cph = P->c64h[C64_PH * R + row];
      for (int kk = 0; kk < 32; kk++) {
        double p = D;
        if (i > 0) p -= crm * crm / piv[(size_t)(i - 1) * 32 + kk];
        if (kk > 0) p -= cph * cph / piv[(size_t)i * 32 + kk - 1];
        if (!(p > 0.0)) return POT3D_ERR_BREAKDOWN;
        piv[(size_t)i * 32 + kk] = p;
      }
    }
    double *sk = t.data() + 4 * RP + (size_t)j * T * 32;
    for (int tt = 0; tt < T; tt++)
      for (int kk = 0; kk < 32; kk++) {
        const int i = tt - kk;
        if (i >= 0 && i < nr) sk[(size_t)tt * 32 + kk] = 1.0 / piv[(size_t)i * 32 + kk];
      }
  }
  if (ai == AR_F64) return upload((double **)&A.icoef, t);
  std::vector<float> h(t.size());
  for (size_t u = 0; u < t.size(); u++) h[u] = (float)t[u];
  return upload((float **)&A.icoef, h);
}

// ----------------------------------------------------------- workspace
// Vectors: x~, r, p~0, p~1, q and, with a line preconditioner, w in
// the iteration's arithmetic; x64, r64 in FP64 for refinement.
size_t workspace_bytes(const Plan *P) {
  const size_t v8 = align256(P->npad * 8), v4 = align256(P->npad * 4);
  const int nv = P->opts.precond != POT3D_PC_JACOBI ? 6 : 5;
  const size_t f64 = nv * v8;
  const size_t mixed = nv * v4 + 2 * v8;
  return P->prec == POT3D_PREC_MIXED ? mixed : std::max(f64, mixed);
}

int ensure_workspace(Plan *P) {
  const size_t b = workspace_bytes(P);
  if (P->ws && P->ws_bytes >= b) return POT3D_OK;
  if (P->ws && !P->ws_owned) return POT3D_ERR_INVALID_ARG; // the caller's buffer is too small
  if (P->ws) cudaFree(P->ws);
  P->ws = nullptr;
  if (cudaMalloc(&P->ws, b) != cudaSuccess) {
    cudaGetLastError();
    return POT3D_ERR_OOM;
  }
  P->ws_bytes = b;
  P->ws_owned = true;
  return POT3D_OK;
}

// Vector v (0..4: x~, r, p~0, p~1, q; 5: w) of an arithmetic with element
// size es; FP64 refinement vectors x64, r64 follow the FP32 vectors.
void *ws_vec(const Plan *P, int v, size_t es) { return P->ws + v * align256(P->npad * es); }
static int n_iter_vecs(const Plan *P) { return P->opts.precond != POT3D_PC_JACOBI ? 6 : 5; }
double *ws_x64(const Plan *P) {
  return (double *)(P->ws + n_iter_vecs(P) * align256(P->npad * 4));
}
double *ws_r64(const Plan *P) {
  return (double *)(P->ws + n_iter_vecs(P) * align256(P->npad * 4) + align256(P->npad * 8));
}

int stage(Plan *P, size_t bytes) {
  if (P->stage_bytes >= bytes) return POT3D_OK;
  if (P->d_stage) cudaFree(P->d_stage);
  P->d_stage = nullptr;
  P->stage_bytes = 0;
  if (cudaMalloc((void **)&P->d_stage, bytes) != cudaSuccess) {
    cudaGetLastError();
    return POT3D_ERR_OOM;
  }
  P->stage_bytes = bytes;
  return POT3D_OK;
}

} // namespace pot3d

// ====================================================================== API
extern "C" {

int pot3d_last_error(void) { return g_last_error; }

const char *pot3d_strerror(int code) {
  switch (code) {
  case POT3D_OK: return "ok";
  case POT3D_ERR_INVALID_ARG: return "invalid argument";
  case POT3D_ERR_OOM: return "out of memory";
  case POT3D_ERR_CUDA: return "CUDA runtime error";
  case POT3D_ERR_NOT_CONVERGED: return "iteration cap reached before the tolerance";
  case POT3D_ERR_BREAKDOWN: return "PCG breakdown (p.Ap <= 0 or not finite)";
  case POT3D_ERR_TIMEOUT: return "device-side wait timed out";
  case POT3D_ERR_UNSUPPORTED: return "unsupported option";
  case POT3D_ERR_BUSY: return "no room to admit the request now";
  case POT3D_ERR_TOO_LARGE: return "request needs more than a fixed-size buffer holds";
  default: return "unknown error";
  }
}

pot3d_plan_t *pot3d_plan(const pot3d_grid_t *g, const pot3d_bc_t *bc) {
  g_last_error = POT3D_OK;
  if (!g || g->nr < 2 || g->nt < 2 || g->np < 3) {
    fail(POT3D_ERR_INVALID_ARG);
    return nullptr;
  }
  if (g->precision < POT3D_PREC_FP64 || g->precision > POT3D_PREC_MIXED) {
    fail(POT3D_ERR_INVALID_ARG);
    return nullptr;
  }
  if (bc) {
    if (bc->outer != POT3D_OUTER_SOURCE_SURFACE && bc->outer != POT3D_OUTER_CLOSED_WALL) {
      fail(POT3D_ERR_INVALID_ARG);
      return nullptr;
    }
    if (bc->pole != POT3D_POLE_AVERAGE) {
      fail(POT3D_ERR_UNSUPPORTED);
      return nullptr;
    }
  }
  const long long n = (long long)g->nr * g->nt * g->np;
  if (n > (1LL << 40)) {
    fail(POT3D_ERR_INVALID_ARG);
    return nullptr;
  }
  Plan *P = new Plan();
  P->nr = g->nr;
  P->nt = g->nt;
  P->np = g->np;
  P->prec = g->precision;
  P->R = (size_t)g->nr * g->nt;
  P->n = P->R * g->np;
  P->pitch = (g->np + 31) / 32 * 32;
  P->ntp = (g->nt + 3) / 4 * 4;
  P->npad = P->R * P->pitch;
  P->closed = bc && bc->outer == POT3D_OUTER_CLOSED_WALL;
  int rc = build_mesh(P, g);
  if (rc) {
    delete P;
    fail(rc);
    return nullptr;
  }
  build_tables(P);
  rc = plan_device_init(P);
  if (rc) {
    plan_free(P);
    fail(rc);
    return nullptr;
  }
  return reinterpret_cast<pot3d_plan_t *>(P);
}

void pot3d_destroy(pot3d_plan_t *plan) {
  if (plan) plan_free(reinterpret_cast<Plan *>(plan));
}

int pot3d_set_stream(pot3d_plan_t *plan, void *s) {
  if (!plan) return fail(POT3D_ERR_INVALID_ARG);
  Plan *P = reinterpret_cast<Plan *>(plan);
  P->user_stream = (cudaStream_t)s;
  P->stream = s ? (cudaStream_t)s : P->own_stream;
  // graphs are tied to the stream they were captured from only by launch;
  // they stay valid
  return POT3D_OK;
}

int pot3d_set_opts(pot3d_plan_t *plan, const pot3d_opts_t *o) {
  if (!plan || !o) return fail(POT3D_ERR_INVALID_ARG);
  if (o->max_iters < 0 || o->chunk < 0 || o->inner_tol < 0 || !(o->inner_tol < 1.0) ||
      o->max_outer < 0 || o->verify < 0 || o->verify > 1 || o->precond < 0 || o->precond > 4 ||
      o->history < 0 || o->history > 1)
    return fail(POT3D_ERR_INVALID_ARG);
  Plan *P = reinterpret_cast<Plan *>(plan);
  P->opts = *o;
  return POT3D_OK;
}

int pot3d_get_info(const pot3d_plan_t *plan, pot3d_info_t *info) {
  if (!plan || !info) return fail(POT3D_ERR_INVALID_ARG);
  const Plan *P = reinterpret_cast<const Plan *>(plan);
  info->n = (long long)P->n;
  info->pitch = P->pitch;
  const int ai = P->prec == POT3D_PREC_FP64 ? AR_F64 : (P->prec == POT3D_PREC_FP64_DF ? AR_DF : AR_F32);
  if (P->ar[ai].ready) {
    info->tiles_matvec = P->ar[ai].tiles_a;
    info->tiles_update = P->ar[ai].tiles_b;
  } else {
    int nv = 0;
    const MvVariant &v = mv_variants(ai, &nv)[0];
    const int nI = heuristic_chunks(P, v), ic = (P->nr + nI - 1) / nI;
    info->tiles_matvec = ((P->nt + v.tj - 1) / v.tj) * ((P->np + v.tk - 1) / v.tk) *
                         ((P->nr + ic - 1) / ic);
    info->tiles_update = (int)((P->R + kRowsPerUpdateItem - 1) / kRowsPerUpdateItem);
  }
  info->workspace_bytes = workspace_bytes(P);
  const double es = (P->prec == POT3D_PREC_MIXED) ? 4.0 : 8.0;
  // matvec: read r, p~_old, x~; write p~_new, q, x~.  update: read r, q; write r.
  info->bytes_matvec = 6.0 * es * (double)P->n;
  info->bytes_update = 3.0 * es * (double)P->n;
  return POT3D_OK;
}

int pot3d_last_stats(const pot3d_plan_t *plan, pot3d_stats_t *s) {
  if (!plan || !s) return fail(POT3D_ERR_INVALID_ARG);
  *s = reinterpret_cast<const Plan *>(plan)->stats;
  return POT3D_OK;
}

size_t pot3d_workspace_bytes(const pot3d_plan_t *plan) {
  if (!plan) return 0;
  return workspace_bytes(reinterpret_cast<const Plan *>(plan));
}

int pot3d_test_freeze_poll(pot3d_plan_t *plan, int on) {
  if (!plan || on < 0 || on > 1) return fail(POT3D_ERR_INVALID_ARG);
  reinterpret_cast<Plan *>(plan)->freeze_poll = (on == 1);
  return POT3D_OK;
}

int pot3d_set_workspace(pot3d_plan_t *plan, void *dev_ptr, size_t bytes) {
  if (!plan || !dev_ptr) return fail(POT3D_ERR_INVALID_ARG);
  Plan *P = reinterpret_cast<Plan *>(plan);
  if (bytes < workspace_bytes(P) || ((uintptr_t)dev_ptr & 255u)) return fail(POT3D_ERR_INVALID_ARG);
  if (!is_device_ptr(dev_ptr)) return fail(POT3D_ERR_INVALID_ARG);
  if (P->ws && P->ws_owned) cudaFree(P->ws);
  P->ws = (char *)dev_ptr;
  P->ws_bytes = bytes;
  P->ws_owned = false;
  return POT3D_OK;
}

} // extern "C"
