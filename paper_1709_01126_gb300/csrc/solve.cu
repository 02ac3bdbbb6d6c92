// Device set-up, the PCG driver loop, iterative refinement, field, apply
// and residual entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include <cudaTypedefs.h>

#include "aux_kernels.cuh"
#include "plan.h"

namespace pot3d {

#define TRY(x)                                                                                     \
  do {                                                                                             \
    int rc_ = (x);                                                                                 \
    if (rc_) return fail(rc_);                                                                     \
  } while (0)
#define CTRY(x)                                                                                    \
  do {                                                                                             \
    cudaError_t e_ = (x);                                                                          \
    if (e_ != cudaSuccess) return cuda_status(e_);                                                 \
  } while (0)

static int aux_grid(const Plan *P, size_t n) {
  size_t b = (n + kAuxThreads - 1) / kAuxThreads;
  return (int)std::max<size_t>(1, std::min<size_t>(b, (size_t)P->aux_blocks));
}

int plan_device_init(Plan *P) {
  int dev = 0;
  CTRY(cudaGetDevice(&dev));
  CTRY(cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, dev));
  CTRY(cudaStreamCreateWithFlags(&P->own_stream, cudaStreamDefault));
  P->stream = P->own_stream;
  auto up = [](double **d, const std::vector<double> &h) -> cudaError_t {
    cudaError_t e = cudaMalloc((void **)d, sizeof(double) * h.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice);
  };
  CTRY(up(&P->d_c64, P->c64h));
  CTRY(up(&P->d_S, P->S));
  CTRY(up(&P->d_irs, P->irs));
  CTRY(up(&P->d_its, P->its));
  CTRY(up(&P->d_irc, P->irc));
  CTRY(up(&P->d_isd, P->isd));
  CTRY(up(&P->d_fwt, P->fwt));
  CTRY(up(&P->d_fwp, P->fwp));
  CTRY(up(&P->d_fwpole, P->fwpole));
  CTRY(cudaMalloc(&P->d_poles, sizeof(double) * 2 * P->nr));
  CTRY(cudaMalloc(&P->d_br_last, sizeof(double) * P->nt * P->np));
  if (P->closed) CTRY(cudaMalloc(&P->d_br_tmp, sizeof(double) * P->nt * P->np));
  P->aux_blocks = 4 * P->nsm;
  CTRY(cudaMalloc(&P->d_part, sizeof(double) * 2 * P->aux_blocks));
  CTRY(cudaMalloc(&P->d_sums, sizeof(double) * 8));
  CTRY(cudaMallocHost(&P->h_sums, sizeof(double) * 8));
  CTRY(cudaMallocHost(&P->h_state, 2 * sizeof(SolveState)));
  memset(P->h_state, 0, 2 * sizeof(SolveState));
  for (auto &e : P->poll_ev) CTRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return POT3D_OK;
}

void plan_free(Plan *P) {
  if (P->stream) cudaStreamSynchronize(P->stream);
  for (auto &A : P->ar) {
    if (A.graph) cudaGraphExecDestroy(A.graph);
    cudaFree(A.coef);
    cudaFree(A.d_prob);
    cudaFree(A.d_state);
    cudaFree(A.part_a);
    cudaFree(A.part_b);
    cudaFree(A.part_c);
    cudaFree(A.lcoef);
    cudaFree(A.rcoef);
    cudaFree(A.icoef);
    cudaFree(A.part_i);
    cudaFree(A.d_tma);
    cudaFree(A.d_work_a);
    cudaFree(A.d_work_b);
    cudaFree(A.d_nwork);
  }
  for (auto e : P->ev) cudaEventDestroy(e);
  for (auto e : P->poll_ev)
    if (e) cudaEventDestroy(e);
  cudaFree(P->d_c64);
  cudaFree(P->d_S);
  cudaFree(P->d_irs);
  cudaFree(P->d_its);
  cudaFree(P->d_irc);
  cudaFree(P->d_isd);
  cudaFree(P->d_fwt);
  cudaFree(P->d_fwp);
  cudaFree(P->d_fwpole);
  cudaFree(P->d_poles);
  cudaFree(P->d_br_last);
  cudaFree(P->d_br_tmp);
  cudaFree(P->d_hist);
  cudaFree(P->d_part);
  cudaFree(P->d_sums);
  cudaFree(P->d_stage);
  if (P->ws_owned) cudaFree(P->ws);
  if (P->h_sums) cudaFreeHost(P->h_sums);
  if (P->h_state) cudaFreeHost(P->h_state);
  if (P->own_stream) cudaStreamDestroy(P->own_stream);
  cudaGetLastError();
  delete P;
}

// ------------------------------------------------------------- iteration
// r-chunks of a matvec tile column: enough work items for about four waves
// of blocks across the SMs, chunks no shorter than 8 planes.
int heuristic_chunks(const Plan *P, const MvVariant &v) {
  const int nJ = (P->nt + v.tj - 1) / v.tj, nK = (P->np + v.tk - 1) / v.tk;
  const int cols = nJ * nK;
  int nI = (4 * P->nsm + cols - 1) / cols;
  return std::max(1, std::min(nI, std::max(1, P->nr / 8)));
}

// Reliable updates: each FP64 residual replacement costs a host round trip
// (about 0.5-1 ms) plus one FP64 operator application, and the FP32 inner
// PCG loses less convergence the more often its residual is replaced.  On
// large grids frequent replacement wins (151x301x601 to 1e-10: 6399 inner
// iterations, 1.29 s at 0.5 against 7314, 1.44 s at 0.1); on small ones the
// round trips dominate (81x121x241: 0.088 s at 0.1, 0.102 s at 0.5).
// Plain restarts need a tight inner solve.
double default_inner_tol(const Plan *P, bool restart) {
  if (restart) return 1e-4;
  return P->n >= 8000000 ? 0.5 : 0.1;
}

// Sets the matvec variant, r-chunk count and update rows per item of
// arithmetic ai and uploads the work lists (one problem: items (0, t)).
int set_decomposition(Plan *P, int ai, int var, int nI, int rows_b) {
  ArithData &D = P->ar[ai];
  int nv = 0;
  const MvVariant *vs = mv_variants(ai, &nv);
  if (var < 0 || var >= nv) return POT3D_ERR_INVALID_ARG;
  const MvVariant &v = vs[var];
  if (nI <= 0) nI = heuristic_chunks(P, v);
  nI = std::min(nI, P->nr);
  D.var = var;
  D.nJ = (P->nt + v.tj - 1) / v.tj;
  D.nK = (P->np + v.tk - 1) / v.tk;
  D.ic = (P->nr + nI - 1) / nI;
  D.nI = (P->nr + D.ic - 1) / D.ic;
  D.tiles_a = D.nJ * D.nK * D.nI;
  D.rows_b = rows_b > 0 ? rows_b : kRowsPerUpdateItem;
  D.tiles_b = (int)((P->R + D.rows_b - 1) / D.rows_b);
  if (D.tiles_a > D.cap_a) {
    cudaFree(D.d_work_a);
    cudaFree(D.part_a);
    D.d_work_a = nullptr;
    D.part_a = nullptr;
    CTRY(cudaMalloc(&D.d_work_a, sizeof(int2) * D.tiles_a));
    CTRY(cudaMalloc(&D.part_a, sizeof(double) * D.tiles_a));
    D.cap_a = D.tiles_a;
  }
  if (D.tiles_b > D.cap_b) {
    cudaFree(D.d_work_b);
    cudaFree(D.part_b);
    D.d_work_b = nullptr;
    D.part_b = nullptr;
    CTRY(cudaMalloc(&D.d_work_b, sizeof(int2) * D.tiles_b));
    CTRY(cudaMalloc(&D.part_b, sizeof(double) * 2 * D.tiles_b));
    D.cap_b = D.tiles_b;
  }
  if (!D.d_nwork) CTRY(cudaMalloc(&D.d_nwork, sizeof(int) * 2));
  std::vector<int2> wa(D.tiles_a), wb(D.tiles_b);
  for (int t = 0; t < D.tiles_a; t++) wa[t] = make_int2(0, t);
  for (int t = 0; t < D.tiles_b; t++) wb[t] = make_int2(0, t);
  const int counts[2] = {D.tiles_a, D.tiles_b};
  CTRY(cudaMemcpy(D.d_work_a, wa.data(), sizeof(int2) * wa.size(), cudaMemcpyHostToDevice));
  CTRY(cudaMemcpy(D.d_work_b, wb.data(), sizeof(int2) * wb.size(), cudaMemcpyHostToDevice));
  CTRY(cudaMemcpy(D.d_nwork, counts, sizeof(counts), cudaMemcpyHostToDevice));
  if (v.setup() != 0) return POT3D_ERR_CUDA;
  // graphs hold the old grid sizes
  if (D.graph) cudaGraphExecDestroy(D.graph);
  D.graph = nullptr;
  return POT3D_OK;
}

static void launch_matvec(Plan *P, int ai) {
  ArithData &D = P->ar[ai];
  int nv = 0;
  const MvVariant &v = mv_variants(ai, &nv)[D.var];
  // one block per tile: the hardware block scheduler balances tiles of
  // unequal cost better than a persistent grid (measured)
  v.launch(D.d_prob, D.d_work_a, D.d_nwork, D.tiles_a, P->stream);
}

// The update step of an iteration per preconditioner: PC1 and phi lines run
// the update kernel; radial lines the column kernel alone (it is the whole
// update); both directions the phi-line update (forming D (T_phi^-1 - D^-1) r)
// and then the column kernel, which adds D T_r^-1 r and closes the iteration;
// PC2 the subdomain ILU(0) kernel alone (it is the whole update too).
static int update_launches(const Plan *P) { return (P->line && P->rline) ? 2 : 1; }

static void launch_update(Plan *P, int ai) {
  ArithData &D = P->ar[ai];
  if (P->ilu) {
    // the shared memory fits: checked by line_setup before the solve
    ilu_launcher(ai)(D.d_prob, D.tiles_i, P->nr, nullptr, P->stream);
    return;
  }
  if (P->line) {
    // the shared memory fits: checked by line_setup before the solve
    update_line_launcher(ai)(D.d_prob, D.d_work_b, D.d_nwork + 1, D.tiles_b, P->pitch, nullptr,
                             P->stream);
    if (P->rline) rline_launcher(ai, true)(D.d_prob, D.tiles_c, nullptr, P->stream);
    return;
  }
  if (P->rline) {
    rline_launcher(ai, false)(D.d_prob, D.tiles_c, nullptr, P->stream);
    return;
  }
  update_launcher(ai)(D.d_prob, D.d_work_b, D.d_nwork + 1, D.tiles_b, P->stream);
}

// The preconditioner of the next PCG run (from the options): which update
// kernels run, and their tables.
static int select_precond(Plan *P, int ai) {
  const int pc = P->opts.precond;
  P->line = pc == POT3D_PC_PHI_LINE || pc == POT3D_PC_LINES;
  P->rline = pc == POT3D_PC_R_LINE || pc == POT3D_PC_LINES;
  P->ilu = pc == POT3D_PC_ILU;
  if (P->ilu) {
    // a box must not close the phi ring (np > 32)
    if (!ilu_launcher(ai) || P->np <= 32) return POT3D_ERR_UNSUPPORTED;
    TRY(ensure_ilu(P, ai));
  }
  if (P->line) {
    if (!update_line_launcher(ai)) return POT3D_ERR_UNSUPPORTED;
    TRY(ensure_line(P, ai));
  }
  if (P->rline) {
    if (!rline_launcher(ai, false)) return POT3D_ERR_UNSUPPORTED;
    TRY(ensure_rline(P, ai));
  }
  return POT3D_OK;
}

// Start of a PCG run with a line preconditioner (solve or refinement step):
// the kernels in their setup mode on the current r (alpha = 0) write
// w = D M^-1 r for the first matvec and ||r||^2, r.M^-1 r to sums[0..1].
static int line_setup(Plan *P, int ai, double *sums) {
  ArithData &D = P->ar[ai];
  if (P->ilu) {
    if (ilu_launcher(ai)(D.d_prob, D.tiles_i, P->nr, sums, P->stream) != 0)
      return POT3D_ERR_UNSUPPORTED; // the warps' rings do not fit in shared memory
    P->stats.launches += 1;
  }
  if (P->line) {
    if (update_line_launcher(ai)(D.d_prob, D.d_work_b, D.d_nwork + 1, D.tiles_b, P->pitch, sums,
                                 P->stream) != 0)
      return POT3D_ERR_UNSUPPORTED; // the rings do not fit in shared memory
    P->stats.launches += 1;
  }
  if (P->rline) {
    rline_launcher(ai, P->line)(D.d_prob, D.tiles_c, sums, P->stream);
    P->stats.launches += 1;
  }
  return POT3D_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time dependency on libcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  }
  return fn;
}

// 3-D map over a padded vector [nr][nt][pitch] with a (bx, by, 1) box.
int encode3d(CUtensorMap *m, void *base, int es, const Plan *P, int bx, int by) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return POT3D_ERR_CUDA;
  cuuint64_t dims[3] = {(cuuint64_t)P->pitch, (cuuint64_t)P->nt, (cuuint64_t)P->nr};
  cuuint64_t strides[2] = {(cuuint64_t)P->pitch * es, (cuuint64_t)P->nt * P->pitch * es};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = fn(m, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 3,
                  base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? POT3D_OK : POT3D_ERR_CUDA;
}

// metric table [6][nr][ntp]: box of kTJ theta rows x 1 plane x 6 tables
int encode_coef_map(CUtensorMap *m, const void *coef, int es, const Plan *P, int tj) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return POT3D_ERR_CUDA;
  cuuint64_t dims[3] = {(cuuint64_t)P->ntp, (cuuint64_t)P->nr, 6u};
  cuuint64_t strides[2] = {(cuuint64_t)P->ntp * es, (cuuint64_t)P->nr * P->ntp * es};
  cuuint32_t box[3] = {(cuuint32_t)tj, 1u, 6u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult cr = fn(m, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 3,
                   const_cast<void *>(coef), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return cr == CUDA_SUCCESS ? POT3D_OK : POT3D_ERR_CUDA;
}

// TMA descriptors of one problem's vectors for matvec variant v.
int encode_tma_set(TmaSet *T, const ProbDev &h, const void *coef, const MvVariant &v,
                   const Plan *P) {
  const int es = v.es;
  // the matvec forms p~ from r (PC1: D z = r) or from w = D z (phi lines)
  void *rsrc = h.w ? h.w : h.r;
  int rc = encode3d(&T->r, rsrc, es, P, v.bw, v.rh);
  if (!rc) rc = encode3d(&T->p0, h.p0, es, P, v.bw, v.rh);
  if (!rc) rc = encode3d(&T->p1, h.p1, es, P, v.bw, v.rh);
  if (!rc) rc = encode3d(&T->x, h.x, es, P, v.tk, v.tj);
  if (!rc) rc = encode3d(&T->rw, rsrc, es, P, v.al, v.rh);
  if (!rc) rc = encode3d(&T->p0w, h.p0, es, P, v.al, v.rh);
  if (!rc) rc = encode3d(&T->p1w, h.p1, es, P, v.al, v.rh);
  if (!rc) rc = encode_coef_map(&T->cf, coef, es, P, v.tj);
  return rc;
}

static int build_tma(Plan *P, int ai) {
  ArithData &D = P->ar[ai];
  int nv = 0;
  const MvVariant &v = mv_variants(ai, &nv)[D.var];
  ProbDev &h = D.h_prob;
  int rc = encode_tma_set(&D.h_tma, h, D.coef, v, P);
  if (rc) return rc;
  if (!D.d_tma) {
    if (cudaMalloc(&D.d_tma, sizeof(TmaSet)) != cudaSuccess) {
      cudaGetLastError();
      return POT3D_ERR_OOM;
    }
  }
  h.tma = D.d_tma;
  if (cudaMemcpyAsync(D.d_tma, &D.h_tma, sizeof(TmaSet), cudaMemcpyHostToDevice, P->stream) !=
      cudaSuccess)
    return POT3D_ERR_CUDA;
  return v.setup() == 0 ? POT3D_OK : POT3D_ERR_CUDA;
}

static int auto_chunk(const Plan *P, int ai) {
  double t_it;
  if (ai == AR_F64) t_it = 13.0 * (double)P->n / 0.45e12; // FP64-unit bound
  else t_it = (ai == AR_DF ? 72.0 : 36.0) * (double)P->n / 4.0e12;
  t_it = std::max(t_it, 8e-6);
  int c = (int)(3e-3 / t_it);
  return std::max(2, std::min(c, 256));
}

template <class A>
static int iterate(Plan *P, int ai, int iter0 = 0) {
  ArithData &D = P->ar[ai];
  const bool timing = P->opts.time_kernels != 0;
  const bool graphs = !timing && P->opts.use_graphs >= 0;
  const int chunk = P->opts.chunk > 0 ? P->opts.chunk : auto_chunk(P, ai);
  if (timing && (int)P->ev.size() < 3 * chunk) {
    for (int u = (int)P->ev.size(); u < 3 * chunk; u++) {
      cudaEvent_t e;
      CTRY(cudaEventCreate(&e));
      P->ev.push_back(e);
    }
  }
  int done_before = iter0, last_iter = iter0 - 1;
  if (!timing) {
    // Chunks as one graph (or plain launches), with one chunk always queued
    // ahead of the host's poll: the state snapshot of chunk N is read (event)
    // while chunk N+1 runs, so the GPU does not idle on the round trip.  A
    // chunk queued after the solve stopped does nothing (its kernels see the
    // status and exit).
    const int pc_key = (P->line ? 1 : 0) | (P->rline ? 2 : 0) | (P->ilu ? 4 : 0);
    if (graphs && (!D.graph || D.graph_chunk != chunk || D.graph_pc != pc_key)) {
      if (D.graph) cudaGraphExecDestroy(D.graph);
      D.graph = nullptr;
      cudaGraph_t g;
      CTRY(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
      for (int c = 0; c < chunk; c++) {
        launch_matvec(P, ai);
        launch_update(P, ai);
      }
      CTRY(cudaStreamEndCapture(P->stream, &g));
      cudaError_t e = cudaGraphInstantiate(&D.graph, g, 0);
      cudaGraphDestroy(g);
      CTRY(e);
      D.graph_chunk = chunk;
      D.graph_pc = pc_key;
    }
    SolveState *snap[2] = {P->h_state, P->h_state + 1};
    auto enqueue = [&](int b) -> int {
      if (graphs) {
        CTRY(cudaGraphLaunch(D.graph, P->stream));
      } else {
        for (int c = 0; c < chunk; c++) {
          launch_matvec(P, ai);
          launch_update(P, ai);
        }
      }
      CTRY(cudaGetLastError());
      P->stats.launches += (1LL + update_launches(P)) * chunk;
      CTRY(cudaMemcpyAsync(snap[b], D.d_state, sizeof(SolveState), cudaMemcpyDeviceToHost,
                           P->stream));
      CTRY(cudaEventRecord(P->poll_ev[b], P->stream));
      return POT3D_OK;
    };
    int b = 0;
    bool have_frozen = false;
    SolveState frozen{};
    TRY(enqueue(0));
    for (;;) {
      TRY(enqueue(b ^ 1));
      CTRY(cudaEventSynchronize(P->poll_ev[b]));
      if (P->freeze_poll) {
        // testing hook: the host keeps seeing its first snapshot
        if (have_frozen) *snap[b] = frozen;
        else frozen = *snap[b];
        have_frozen = true;
      }
      if (snap[b]->status != ST_RUNNING) break;
      // a running solve must advance every chunk; if it does not, the
      // device state is inconsistent: stop instead of polling forever
      if (snap[b]->iter <= last_iter) {
        cudaStreamSynchronize(P->stream);
        return fail(POT3D_ERR_TIMEOUT);
      }
      last_iter = snap[b]->iter;
      b ^= 1;
    }
    // the last queued chunk saw the finished state; its snapshot is final
    CTRY(cudaStreamSynchronize(P->stream));
    if (b == 0) *snap[0] = *snap[1];
    return POT3D_OK;
  }
  // time_kernels: plain launches between CUDA events, one chunk at a time
  for (;;) {
    for (int c = 0; c < chunk; c++) {
      CTRY(cudaEventRecord(P->ev[3 * c], P->stream));
      launch_matvec(P, ai);
      CTRY(cudaEventRecord(P->ev[3 * c + 1], P->stream));
      launch_update(P, ai);
      CTRY(cudaEventRecord(P->ev[3 * c + 2], P->stream));
    }
    CTRY(cudaGetLastError());
    P->stats.launches += (1LL + update_launches(P)) * chunk;
    CTRY(cudaMemcpyAsync(P->h_state, D.d_state, sizeof(SolveState), cudaMemcpyDeviceToHost,
                         P->stream));
    CTRY(cudaStreamSynchronize(P->stream));
    if (P->freeze_poll) {
      // testing hook: the host keeps seeing its first snapshot
      if (last_iter >= iter0) P->h_state->iter = last_iter;
    }
    // only iterations that did work count (kernels exit early once done)
    const int real = std::min(chunk, P->h_state->iter - done_before);
    done_before = P->h_state->iter;
    for (int c = 0; c < real; c++) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, P->ev[3 * c], P->ev[3 * c + 1]);
      cudaEventElapsedTime(&b, P->ev[3 * c + 1], P->ev[3 * c + 2]);
      P->stats.kernel_ms[0] += a;
      P->stats.kernel_ms[1] += b;
      P->stats.kernel_ms[2] += 1.0;
      P->stats.kernel_ms[3] += 1.0;
    }
    if (P->h_state->status != ST_RUNNING) break;
    // a running solve must advance every chunk; if it does not, the
    // device state is inconsistent: stop instead of polling forever
    if (P->h_state->iter <= last_iter) return fail(POT3D_ERR_TIMEOUT);
    last_iter = P->h_state->iter;
  }
  return POT3D_OK;
}

template <class A>
static void fill_prob(Plan *P, int ai, void *x, void *r, void *p0, void *p1, void *q,
                      void *w = nullptr) {
  ArithData &D = P->ar[ai];
  ProbDev &h = D.h_prob;
  h = ProbDev{};
  h.nr = P->nr;
  h.nt = P->nt;
  h.np = P->np;
  h.pitch = P->pitch;
  h.ntp = P->ntp;
  h.nJ = D.nJ;
  h.nK = D.nK;
  h.ic = D.ic;
  h.nI = D.nI;
  h.tiles_a = D.tiles_a;
  h.rows_b = D.rows_b;
  h.tiles_b = D.tiles_b;
  h.plane = (long long)P->nt * P->pitch;
  h.x = x;
  h.r = r;
  h.p0 = p0;
  h.p1 = p1;
  h.q = q;
  h.coef = D.coef;
  h.part_a = D.part_a;
  h.part_b = D.part_b;
  h.st = D.d_state;
  h.w = w;
  h.lcoef = P->line ? D.lcoef : nullptr;
  h.rcoef = P->rline ? D.rcoef : nullptr;
  h.part_c = P->ilu ? D.part_i : D.part_c;
  h.tiles_c = P->ilu ? D.tiles_i : D.tiles_c;
  h.lines = (P->line && P->rline) ? 1 : 0;
  h.icoef = P->ilu ? D.icoef : nullptr;
}

static int status_code(int st) {
  switch (st) {
  case ST_CONVERGED: return POT3D_OK;
  case ST_MAXIT: return POT3D_ERR_NOT_CONVERGED;
  case ST_BREAKDOWN: return POT3D_ERR_BREAKDOWN;
  case ST_TIMEOUT: return POT3D_ERR_TIMEOUT;
  default: return POT3D_ERR_CUDA;
  }
}

int default_maxit(const Plan *P) { return 100 * (P->nr + P->nt + P->np); }

void prepare_br(const Plan *P, const double *br, double *out, double *part, double *sum,
                cudaStream_t s) {
  const size_t n0 = (size_t)P->nt * P->np;
  if (!P->closed) {
    if (out != br) cudaMemcpyAsync(out, br, n0 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return;
  }
  const int g = aux_grid(P, n0);
  k_flux<kAuxThreads><<<g, kAuxThreads, 0, s>>>(br, P->d_S, P->nt, P->np, part);
  k_sum_pairs<kAuxThreads><<<1, kAuxThreads, 0, s>>>(part, g, sum);
  k_shift<<<g, kAuxThreads, 0, s>>>(br, out, n0, sum, P->inv_area);
}

void gauge_phi(const Plan *P, double *phi, double *part, double *sum, cudaStream_t s) {
  if (!P->closed) return;
  const int g = aux_grid(P, P->n);
  k_sum_partials<kAuxThreads><<<g, kAuxThreads, 0, s>>>(phi, P->n, part);
  k_sum_pairs<kAuxThreads><<<1, kAuxThreads, 0, s>>>(part, g, sum);
  k_sub_mean<<<g, kAuxThreads, 0, s>>>(phi, P->n, sum, 1.0 / (double)P->n);
}

// Iterations one continued inner segment may take before it is ended and
// the next refinement step restarts the inner PCG from zero.
int segment_cap(const Plan *P) { return 20 * (P->nr + P->nt + P->np); }

// Inputs may be host or device pointers; host arrays are staged through
// one device buffer [br | phi | B].
struct Io {
  const double *br = nullptr;
  double *phi = nullptr;
  double *B = nullptr;
  bool br_host = false, phi_host = false, B_host = false;
};

static int stage_io(Plan *P, const double *br, double *phi, double *B, bool phi_in, Io &io) {
  io.br_host = br && !is_device_ptr(br);
  io.phi_host = phi && !is_device_ptr(phi);
  io.B_host = B && !is_device_ptr(B);
  const size_t nb = (size_t)P->nt * P->np;
  const size_t nB = (size_t)(P->nr + 1) * P->nt * P->np + (size_t)P->nr * (P->nt + 1) * P->np + P->n;
  size_t need = 0;
  if (io.br_host) need += nb;
  if (io.phi_host) need += P->n;
  if (io.B_host) need += nB;
  if (need) TRY(stage(P, need * sizeof(double)));
  size_t off = 0;
  io.br = br;
  io.phi = phi;
  io.B = B;
  if (io.br_host) {
    io.br = P->d_stage + off;
    CTRY(cudaMemcpyAsync((void *)io.br, br, nb * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    off += nb;
  }
  if (io.phi_host) {
    io.phi = P->d_stage + off;
    if (phi_in)
      CTRY(cudaMemcpyAsync(io.phi, phi, P->n * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    off += P->n;
  }
  if (io.B_host) io.B = P->d_stage + off;
  return POT3D_OK;
}

template <class A>
static int solve_pcg(Plan *P, int ai, const double *br, double tol, double *phi, int *iters) {
  TRY(ensure_arith(P, ai));
  TRY(select_precond(P, ai));
  TRY(ensure_workspace(P));
  const bool x0 = P->opts.use_x0 != 0;
  Io io;
  TRY(stage_io(P, br, phi, nullptr, x0, io));
  const size_t es = sizeof(typename A::st);
  void *x = ws_vec(P, 0, es), *r = ws_vec(P, 1, es), *p0 = ws_vec(P, 2, es),
       *p1 = ws_vec(P, 3, es), *q = ws_vec(P, 4, es);
  void *w = (P->line || P->rline || P->ilu) ? ws_vec(P, 5, es) : nullptr;
  ArithData &D = P->ar[ai];
  fill_prob<A>(P, ai, x, r, p0, p1, q, w);
  TRY(build_tma(P, ai));
  cudaStream_t s = P->stream;
  // the Br of the right-hand side (closed wall: balanced), kept for the field
  prepare_br(P, io.br, P->d_br_last, P->d_part, P->d_sums + 6, s);
  const double *brs = P->d_br_last;
  P->have_br = true;
  CTRY(cudaMemsetAsync(P->ws, 0, (w ? 6 : 5) * ((P->npad * es + 255) & ~(size_t)255), s));
  const size_t n0 = (size_t)P->nt * P->np;
  const int gb = aux_grid(P, n0);
  k_bstats<kAuxThreads><<<gb, kAuxThreads, 0, s>>>(brs, P->d_S, P->d_c64, P->nr, P->nt, P->np,
                                                   P->d_part);
  k_sum_pairs<kAuxThreads><<<1, kAuxThreads, 0, s>>>(P->d_part, gb, P->d_sums);
  if (x0) {
    const int g = aux_grid(P, P->n);
    k_op64<kAuxThreads><<<g, kAuxThreads, 0, s>>>(io.phi, P->np, brs, P->d_S, P->d_c64, P->nr,
                                                  P->nt, P->np, 0, (double *)q, P->pitch,
                                                  P->d_part);
    k_sum_pairs<kAuxThreads><<<1, kAuxThreads, 0, s>>>(P->d_part, g, P->d_sums + 2);
  }
  const int maxit = P->opts.max_iters > 0 ? P->opts.max_iters : default_maxit(P);
  P->hist_n = 0;
  if (P->opts.history) {
    if (P->hist_alloc < maxit + 1) {
      cudaFree(P->d_hist);
      P->d_hist = nullptr;
      P->hist_alloc = 0;
      if (cudaMalloc(&P->d_hist, sizeof(double) * (maxit + 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(POT3D_ERR_OOM);
      }
      P->hist_alloc = maxit + 1;
    }
    D.h_prob.hist = P->d_hist;
    D.h_prob.hist_cap = maxit + 1;
  } else {
    D.h_prob.hist = nullptr;
    D.h_prob.hist_cap = 0;
  }
  CTRY(cudaMemcpyAsync(D.d_prob, &D.h_prob, sizeof(ProbDev), cudaMemcpyHostToDevice, s));
  k_start<<<1, 1, 0, s>>>(D.d_state, P->d_sums, (double)n0, tol, maxit, x0 ? 1 : 0, 0.0,
                          P->opts.history ? P->d_hist : nullptr);
  if (x0) {
    k_x0_setup<A><<<aux_grid(P, P->n), kAuxThreads, 0, s>>>(
        (const double *)q, io.phi, P->d_c64, P->nr, P->nt, P->np, P->pitch, D.d_state,
        (typename A::st *)r, (typename A::st *)x);
    CTRY(cudaMemsetAsync(q, 0, P->npad * es, s));
  } else {
    k_write_rhs<A><<<aux_grid(P, n0), kAuxThreads, 0, s>>>(brs, P->d_S, P->nt, P->np, P->pitch,
                                                           D.d_state, (typename A::st *)r);
  }
  CTRY(cudaGetLastError());
  memset(&P->stats, 0, sizeof(P->stats));
  if (w) {
    // w_0 = D M^-1 r_0 and rho_0 = r_0 . M^-1 r_0 (scaled units)
    TRY(line_setup(P, ai, P->d_sums + 4));
    k_set_rho<<<1, 1, 0, s>>>(D.d_state, P->d_sums + 4);
    P->stats.launches += 1;
  }
  P->stats.launches += x0 ? 7 : 4;
  TRY(iterate<A>(P, ai));
  P->stats.launches += 1;
  k_finish<A><<<aux_grid(P, P->n), kAuxThreads, 0, s>>>(D.d_prob, P->d_c64, io.phi, 1);
  gauge_phi(P, io.phi, P->d_part, P->d_sums + 6, s);
  // the FP64 residual of the returned Phi (||b||^2 is in d_sums[0])
  const int g = aux_grid(P, P->n);
  k_op64<kAuxThreads><<<g, kAuxThreads, 0, s>>>(io.phi, P->np, brs, P->d_S, P->d_c64, P->nr,
                                                P->nt, P->np, 0, nullptr, P->np, P->d_part);
  k_sum_pairs<kAuxThreads><<<1, kAuxThreads, 0, s>>>(P->d_part, g, P->d_sums + 2);
  P->stats.launches += 2;
  CTRY(cudaGetLastError());
  CTRY(cudaMemcpyAsync(P->h_sums, P->d_sums, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
  if (io.phi_host)
    CTRY(cudaMemcpyAsync(phi, io.phi, P->n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CTRY(cudaStreamSynchronize(s));
  const SolveState &hs = *P->h_state;
  P->stats.status = status_code(hs.status);
  P->stats.iters = hs.iter;
  P->stats.outer_iters = 0;
  P->stats.relres = hs.relres;
  P->stats.sigma = hs.sigma;
  P->stats.rr = hs.rr;
  const double bb = P->h_sums[0];
  P->stats.relres_fp64 = bb > 0 ? std::sqrt(P->h_sums[2]) / std::sqrt(bb) : 0.0;
  P->stats.flags = (P->stats.status == POT3D_OK && P->stats.relres_fp64 > tol) ? POT3D_FLAG_ABOVE_TOL : 0;
  if (P->opts.history) P->hist_n = std::min(hs.iter + 1, P->hist_alloc);
  if (iters) *iters = hs.iter;
  return P->stats.status ? fail(P->stats.status) : POT3D_OK;
}

// FP64 iterative refinement (defect correction) around FP32 PCG.
static int solve_mixed(Plan *P, const double *br, double tol, double *phi, int *outer,
                       int *inner) {
  TRY(ensure_arith(P, AR_F32));
  TRY(select_precond(P, AR_F32));
  TRY(ensure_workspace(P));
  const bool x0 = P->opts.use_x0 != 0;
  Io io;
  TRY(stage_io(P, br, phi, nullptr, x0, io));
  cudaStream_t s = P->stream;
  ArithData &D = P->ar[AR_F32];
  void *x = ws_vec(P, 0, 4), *r = ws_vec(P, 1, 4), *p0 = ws_vec(P, 2, 4), *p1 = ws_vec(P, 3, 4),
       *q = ws_vec(P, 4, 4);
  void *w = (P->line || P->rline || P->ilu) ? ws_vec(P, 5, 4) : nullptr;
  double *x64 = ws_x64(P), *r64 = ws_r64(P);
  fill_prob<PF32>(P, AR_F32, x, r, p0, p1, q, w);
  TRY(build_tma(P, AR_F32));
  CTRY(cudaMemcpyAsync(D.d_prob, &D.h_prob, sizeof(ProbDev), cudaMemcpyHostToDevice, s));
  // the Br of the right-hand side (closed wall: balanced), kept for the field
  prepare_br(P, io.br, P->d_br_last, P->d_part, P->d_sums + 6, s);
  const double *brs = P->d_br_last;
  P->have_br = true;
  const size_t v4 = (P->npad * 4 + 255) & ~(size_t)255;
  CTRY(cudaMemsetAsync(P->ws, 0, (w ? 6 : 5) * v4, s));
  CTRY(cudaMemsetAsync(x64, 0, P->npad * 8, s));
  CTRY(cudaMemsetAsync(r64, 0, P->npad * 8, s));
  if (x0)
    k_unpad<<<aux_grid(P, P->n), kAuxThreads, 0, s>>>(io.phi, P->np, x64, P->pitch, P->R, P->np);
  const size_t n0 = (size_t)P->nt * P->np;
  const int gb = aux_grid(P, n0);
  k_bstats<kAuxThreads><<<gb, kAuxThreads, 0, s>>>(brs, P->d_S, P->d_c64, P->nr, P->nt, P->np,
                                                   P->d_part);
  k_sum_pairs<kAuxThreads><<<1, kAuxThreads, 0, s>>>(P->d_part, gb, P->d_sums);
  const int gn = aux_grid(P, P->n);
  const float *dinv32 = static_cast<const float *>(D.coef); // slab 0 of the F32 table
  const bool restart = P->opts.mixed_restart != 0;
  const double inner_tol = P->opts.inner_tol > 0 ? P->opts.inner_tol : default_inner_tol(P, restart);
  const int max_outer = P->opts.max_outer > 0 ? P->opts.max_outer : (restart ? 30 : 200);
  const int inner_maxit = P->opts.max_iters > 0 ? P->opts.max_iters : default_maxit(P);
  memset(&P->stats, 0, sizeof(P->stats));
  P->stats.launches = 2 + (x0 ? 1 : 0);
  int n_outer = 0, n_inner = 0, status = POT3D_OK;
  double bb = 0.0, prev = INFINITY, relres = INFINITY, scale = 1.0;
  bool resumable = false; // an inner PCG stopped cleanly and may continue
  for (;;) {
    k_op64<kAuxThreads><<<gn, kAuxThreads, 0, s>>>(x64, P->pitch, brs, P->d_S, P->d_c64, P->nr,
                                                   P->nt, P->np, 0, r64, P->pitch, P->d_part);
    k_sum_pairs<kAuxThreads><<<1, kAuxThreads, 0, s>>>(P->d_part, gn, P->d_sums + 2);
    P->stats.launches += 2;
    CTRY(cudaGetLastError());
    CTRY(cudaMemcpyAsync(P->h_sums, P->d_sums, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    CTRY(cudaStreamSynchronize(s));
    bb = P->h_sums[0];
    const double rr = P->h_sums[2];
    relres = (bb > 0) ? std::sqrt(rr) / std::sqrt(bb) : 0.0;
    if (!std::isfinite(relres)) {
      status = POT3D_ERR_BREAKDOWN;
      break;
    }
    if (relres <= tol) break;
    // restarts must gain a factor 2 per step; replacements only must not
    // grow the residual
    if (n_outer >= max_outer || !(relres < (restart ? 0.5 : 1.0) * prev)) {
      status = POT3D_ERR_NOT_CONVERGED;
      break;
    }
    prev = relres;
    // inner system L d = scale * r64 in FP32
    const double rms = std::sqrt(rr / (double)P->n);
    const double new_scale = std::ldexp(1.0, -std::ilogb(rms));
    k_inner_rhs<kAuxThreads><<<gn, kAuxThreads, 0, s>>>(r64, dinv32, P->nr, P->nt, P->ntp, P->np,
                                                        P->pitch, new_scale, (float *)r, P->d_part);
    k_sum_pairs<kAuxThreads><<<1, kAuxThreads, 0, s>>>(P->d_part, gn, P->d_sums + 4);
    // line preconditioners: w = D M^-1 r32 and rho = r32 . M^-1 r32 replace the sums
    if (w) TRY(line_setup(P, AR_F32, P->d_sums + 4));
    CTRY(cudaMemsetAsync(x, 0, v4, s));
    int iter0 = 0;
    if (resumable && !restart) {
      // reliable update: keep p~ and the iteration count
      k_resume<<<1, 1, 0, s>>>(D.d_state, P->d_sums + 4, scale / new_scale, inner_tol,
                               segment_cap(P));
      iter0 = P->h_state->iter;
      P->stats.launches += 3;
    } else {
      CTRY(cudaMemsetAsync(p0, 0, v4, s));
      CTRY(cudaMemsetAsync(p1, 0, v4, s));
      CTRY(cudaMemsetAsync(q, 0, v4, s));
      k_start<<<1, 1, 0, s>>>(D.d_state, P->d_sums + 4, (double)P->n, inner_tol, inner_maxit, 0,
                              1.0, nullptr);
      P->stats.launches += 4;
    }
    scale = new_scale;
    CTRY(cudaGetLastError());
    TRY(iterate<PF32>(P, AR_F32, iter0));
    const SolveState &hs = *P->h_state;
    P->stats.sigma = hs.sigma;
    P->stats.rr = hs.rr;
    n_inner += hs.iter - iter0;
    if (hs.status == ST_BREAKDOWN && hs.iter == iter0) {
      status = POT3D_ERR_BREAKDOWN;
      break;
    }
    resumable = (hs.status == ST_CONVERGED);
    k_refine_update<<<gn, kAuxThreads, 0, s>>>(D.d_prob, P->d_c64, x64, 1.0 / scale);
    P->stats.launches += 1;
    n_outer++;
  }
  k_unpad<<<gn, kAuxThreads, 0, s>>>(x64, P->pitch, io.phi, P->np, P->R, P->np);
  gauge_phi(P, io.phi, P->d_part, P->d_sums + 6, s);
  P->stats.launches += 1;
  CTRY(cudaGetLastError());
  if (io.phi_host)
    CTRY(cudaMemcpyAsync(phi, io.phi, P->n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CTRY(cudaStreamSynchronize(s));
  P->stats.status = status;
  P->stats.iters = n_inner;
  P->stats.outer_iters = n_outer;
  P->stats.relres = relres;
  P->stats.relres_fp64 = relres;
  P->stats.flags = 0;
  if (outer) *outer = n_outer;
  if (inner) *inner = n_inner;
  return status ? fail(status) : POT3D_OK;
}

// PCG with residual replacement (opts.verify): the recurrence residual of a
// long solve drifts from the true one (at 401x801x1601 to 1e-10 after ~33k
// iterations the FP64 result's true residual is 4.2e-10, the double-float
// one's 7.6e-9).  After each converged run the FP64 residual b - L Phi is
// recomputed; while it is above tol, PCG restarts from Phi with it (the
// use_x0 path), within the same iteration cap.
constexpr int kMaxReplacements = 10;

template <class A>
static int solve_pcg_verified(Plan *P, int ai, const double *br, double tol, double *phi,
                              int *iters) {
  const pot3d_opts_t saved = P->opts;
  const int cap = saved.max_iters > 0 ? saved.max_iters : default_maxit(P);
  int total = 0, restarts = 0, rc = POT3D_OK;
  double rel = 0.0;
  long long launches = 0;
  for (;;) {
    P->opts.max_iters = std::max(1, cap - total);
    int it = 0;
    rc = solve_pcg<A>(P, ai, br, tol, phi, &it);
    total += it;
    launches += P->stats.launches;
    if (rc != POT3D_OK) break;
    rel = P->stats.relres_fp64; // recomputed by solve_pcg from the returned Phi
    if (rel <= tol) break;
    if (restarts == kMaxReplacements || total >= cap) {
      rc = POT3D_ERR_NOT_CONVERGED;
      break;
    }
    restarts++;
    P->opts.use_x0 = 1; // Phi holds the current iterate
  }
  P->opts = saved;
  if (rc == POT3D_OK || rc == POT3D_ERR_NOT_CONVERGED) P->stats.relres = rel;
  P->stats.flags = 0;
  P->stats.status = rc;
  P->stats.iters = total;
  P->stats.outer_iters = restarts;
  P->stats.launches = launches;
  if (iters) *iters = total;
  return rc ? fail(rc) : POT3D_OK;
}

} // namespace pot3d

using namespace pot3d;

extern "C" {

int pot3d_solve(pot3d_plan_t *plan, const double *br, double tol, double *phi, int *iters) {
  if (!plan || !br || !phi || !(tol > 0.0) || !std::isfinite(tol)) return fail(POT3D_ERR_INVALID_ARG);
  Plan *P = reinterpret_cast<Plan *>(plan);
  const bool verify = P->opts.verify != 0;
  switch (P->prec) {
  case POT3D_PREC_FP64:
    return verify ? solve_pcg_verified<PF64>(P, AR_F64, br, tol, phi, iters)
                  : solve_pcg<PF64>(P, AR_F64, br, tol, phi, iters);
  case POT3D_PREC_FP64_DF:
    return verify ? solve_pcg_verified<PDF>(P, AR_DF, br, tol, phi, iters)
                  : solve_pcg<PDF>(P, AR_DF, br, tol, phi, iters);
  default: {
    int o = 0, in = 0;
    int rc = solve_mixed(P, br, tol, phi, &o, &in);
    if (iters) *iters = in;
    return rc;
  }
  }
}

int pot3d_solve_mixed(pot3d_plan_t *plan, const double *br, double tol, double *phi,
                      int *outer_iters, int *inner_iters) {
  if (!plan || !br || !phi || !(tol > 0.0) || !std::isfinite(tol)) return fail(POT3D_ERR_INVALID_ARG);
  return solve_mixed(reinterpret_cast<Plan *>(plan), br, tol, phi, outer_iters, inner_iters);
}

int pot3d_field(pot3d_plan_t *plan, const double *phi, const double *br, double *B) {
  if (!plan || !phi || !B) return fail(POT3D_ERR_INVALID_ARG);
  Plan *P = reinterpret_cast<Plan *>(plan);
  if (!br && !P->have_br) return fail(POT3D_ERR_INVALID_ARG);
  Io io;
  TRY(stage_io(P, br, const_cast<double *>(phi), B, true, io));
  const double *d_br = br ? io.br : P->d_br_last;
  cudaStream_t s = P->stream;
  if (br && P->closed) {
    // the inner face carries the balanced Br, the one a solve uses
    prepare_br(P, io.br, P->d_br_tmp, P->d_part, P->d_sums + 6, s);
    d_br = P->d_br_tmp;
  }
  k_pole_avg<kAuxThreads><<<2 * P->nr, kAuxThreads, 0, s>>>(io.phi, P->nr, P->nt, P->np,
                                                            P->d_poles);
  FieldTabs T{P->d_irs, P->d_its, P->d_irc, P->d_isd, P->d_fwt, P->d_fwp, P->d_fwpole,
              P->closed ? 1 : 0};
  const size_t tot = (size_t)(P->nr + 1) * P->nt * P->np + (size_t)P->nr * (P->nt + 1) * P->np + P->n;
  if (P->n >= (1ull << 31)) return fail(POT3D_ERR_TOO_LARGE); // 32-bit cell index
  const int gf = (int)std::min<size_t>((P->n + kFieldThreads - 1) / kFieldThreads,
                                       (size_t)8 * P->nsm);
  k_field<<<gf, kFieldThreads, 0, s>>>(io.phi, d_br, P->d_poles, T, P->nr, P->nt, P->np, io.B);
  P->stats.launches = 2;
  CTRY(cudaGetLastError());
  if (io.B_host) CTRY(cudaMemcpyAsync(B, io.B, tot * sizeof(double), cudaMemcpyDeviceToHost, s));
  CTRY(cudaStreamSynchronize(s));
  return POT3D_OK;
}

int pot3d_get_history(const pot3d_plan_t *plan, double *relres, int cap, int *n) {
  if (!plan || !relres || cap < 0 || !n) return fail(POT3D_ERR_INVALID_ARG);
  const Plan *P = reinterpret_cast<const Plan *>(plan);
  if (!P->d_hist || P->hist_n <= 0) return fail(POT3D_ERR_INVALID_ARG);
  const int m = std::min(cap, P->hist_n);
  if (m > 0) CTRY(cudaMemcpy(relres, P->d_hist, sizeof(double) * m, cudaMemcpyDeviceToHost));
  *n = m;
  return POT3D_OK;
}

int pot3d_apply(pot3d_plan_t *plan, const double *x, double *y) {
  if (!plan || !x || !y) return fail(POT3D_ERR_INVALID_ARG);
  Plan *P = reinterpret_cast<Plan *>(plan);
  const bool xh = !is_device_ptr(x), yh = !is_device_ptr(y);
  size_t need = (xh ? P->n : 0) + (yh ? P->n : 0);
  if (need) TRY(stage(P, need * sizeof(double)));
  cudaStream_t s = P->stream;
  const double *dx = x;
  double *dy = y;
  size_t off = 0;
  if (xh) {
    dx = P->d_stage;
    CTRY(cudaMemcpyAsync((void *)dx, x, P->n * sizeof(double), cudaMemcpyHostToDevice, s));
    off = P->n;
  }
  if (yh) dy = P->d_stage + off;
  const int g = aux_grid(P, P->n);
  k_op64<kAuxThreads><<<g, kAuxThreads, 0, s>>>(dx, P->np, nullptr, P->d_S, P->d_c64, P->nr, P->nt,
                                                P->np, 1, dy, P->np, P->d_part);
  CTRY(cudaGetLastError());
  if (yh) CTRY(cudaMemcpyAsync(y, dy, P->n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CTRY(cudaStreamSynchronize(s));
  return POT3D_OK;
}

int pot3d_residual(pot3d_plan_t *plan, const double *br, const double *phi, double *relres) {
  if (!plan || !br || !phi || !relres) return fail(POT3D_ERR_INVALID_ARG);
  Plan *P = reinterpret_cast<Plan *>(plan);
  Io io;
  TRY(stage_io(P, br, const_cast<double *>(phi), nullptr, true, io));
  cudaStream_t s = P->stream;
  const double *brs = io.br;
  if (P->closed) {
    // the balanced Br, the one a solve uses
    prepare_br(P, io.br, P->d_br_tmp, P->d_part, P->d_sums + 6, s);
    brs = P->d_br_tmp;
  }
  const size_t n0 = (size_t)P->nt * P->np;
  const int gb = aux_grid(P, n0);
  k_bstats<kAuxThreads><<<gb, kAuxThreads, 0, s>>>(brs, P->d_S, P->d_c64, P->nr, P->nt, P->np,
                                                   P->d_part);
  k_sum_pairs<kAuxThreads><<<1, kAuxThreads, 0, s>>>(P->d_part, gb, P->d_sums);
  const int g = aux_grid(P, P->n);
  k_op64<kAuxThreads><<<g, kAuxThreads, 0, s>>>(io.phi, P->np, brs, P->d_S, P->d_c64, P->nr,
                                                P->nt, P->np, 0, nullptr, P->np, P->d_part);
  k_sum_pairs<kAuxThreads><<<1, kAuxThreads, 0, s>>>(P->d_part, g, P->d_sums + 2);
  CTRY(cudaGetLastError());
  CTRY(cudaMemcpyAsync(P->h_sums, P->d_sums, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
  CTRY(cudaStreamSynchronize(s));
  *relres = P->h_sums[0] > 0 ? std::sqrt(P->h_sums[2]) / std::sqrt(P->h_sums[0]) : 0.0;
  return POT3D_OK;
}

} // extern "C"

// ============================================================== autotuner
namespace pot3d {
namespace {

struct TuneKey {
  int nr, nt, np, ai;
  bool operator<(const TuneKey &o) const {
    return std::tie(nr, nt, np, ai) < std::tie(o.nr, o.nt, o.np, o.ai);
  }
};
struct TuneVal {
  int var, nI, rows;
  double ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
bool g_tune_loaded = false;

// Optional persistence: POT3D_TUNE_CACHE names a text file that starts with
// the tag kTuneTag, then lines "nr nt np arith variant chunks update_rows
// matvec_ms".  A file without the tag (another format) is ignored and
// rewritten.
constexpr const char *kTuneTag = "pot3d-tune-2";
void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = getenv("POT3D_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  char tag[32] = {0};
  if (fscanf(f, "%31s", tag) != 1 || strcmp(tag, kTuneTag) != 0) {
    fclose(f);
    return;
  }
  TuneKey k;
  TuneVal v;
  while (fscanf(f, "%d %d %d %d %d %d %d %lf", &k.nr, &k.nt, &k.np, &k.ai, &v.var, &v.nI, &v.rows,
                &v.ms) == 8)
    g_tune[k] = v;
  fclose(f);
}

void tune_store_locked() {
  const char *path = getenv("POT3D_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "w");
  if (!f) return;
  fprintf(f, "%s\n", kTuneTag);
  for (const auto &kv : g_tune)
    fprintf(f, "%d %d %d %d %d %d %d %.6f\n", kv.first.nr, kv.first.nt, kv.first.np, kv.first.ai,
            kv.second.var, kv.second.nI, kv.second.rows, kv.second.ms);
  fclose(f);
}

template <class A>
int tune_arith(Plan *P, int ai, TuneVal *best) {
  TRY(ensure_arith(P, ai));
  TRY(ensure_workspace(P));
  P->line = false; // the tuner times the diagonal-scaling kernels
  P->rline = false;
  P->ilu = false;
  ArithData &D = P->ar[ai];
  const size_t es = sizeof(typename A::st);
  cudaStream_t s = P->stream;
  CTRY(cudaMemsetAsync(P->ws, 0, 5 * ((P->npad * es + 255) & ~(size_t)255), s));
  // a running iteration (k > 1, so every TMA box is loaded) on zero vectors
  SolveState fake{};
  fake.status = ST_RUNNING;
  fake.iter = 5;
  fake.alpha[0] = fake.alpha[1] = 0.5;
  fake.beta[0] = fake.beta[1] = 0.5;
  fake.rho = 1.0;
  fake.bb = 1.0;
  fake.maxit = 1 << 30;
  cudaEvent_t e0, e1;
  CTRY(cudaEventCreate(&e0));
  CTRY(cudaEventCreate(&e1));
  int nv = 0;
  const MvVariant *vs = mv_variants(ai, &nv);
  best->ms = INFINITY;
  best->rows = kRowsPerUpdateItem;
  auto prepare = [&]() -> int {
    fill_prob<A>(P, ai, ws_vec(P, 0, es), ws_vec(P, 1, es), ws_vec(P, 2, es), ws_vec(P, 3, es),
                 ws_vec(P, 4, es));
    int rc = build_tma(P, ai);
    if (rc) return rc;
    if (cudaMemcpyAsync(D.d_prob, &D.h_prob, sizeof(ProbDev), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return POT3D_ERR_CUDA;
    return POT3D_OK;
  };
  auto time_kernel = [&](bool matvec, double *avg) -> int {
    float tot = 0.f;
    const int warm = 2, reps = 5;
    for (int it = 0; it < warm + reps; it++) {
      CTRY(cudaMemcpyAsync(D.d_state, &fake, sizeof(fake), cudaMemcpyHostToDevice, s));
      CTRY(cudaEventRecord(e0, s));
      if (matvec) launch_matvec(P, ai);
      else launch_update(P, ai);
      CTRY(cudaEventRecord(e1, s));
      CTRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      CTRY(cudaEventElapsedTime(&ms, e0, e1));
      if (it >= warm) tot += ms;
    }
    *avg = tot / reps;
    return POT3D_OK;
  };
  // matvec: tile shape x r-chunks
  for (int v = 0; v < nv; v++) {
    std::vector<int> chunks = {heuristic_chunks(P, vs[v]), 1, 2, 3, 4, 6, 8};
    std::sort(chunks.begin(), chunks.end());
    chunks.erase(std::unique(chunks.begin(), chunks.end()), chunks.end());
    for (int nI : chunks) {
      if (nI > std::max(1, P->nr / 4) && nI != 1) continue;
      TRY(set_decomposition(P, ai, v, nI, best->rows));
      TRY(prepare());
      double avg = 0.0;
      TRY(time_kernel(true, &avg));
      if (avg < best->ms) {
        best->var = v;
        best->nI = nI;
        best->ms = avg;
      }
    }
  }
  // update: rows per work item, fixed sizes and sizes that make whole
  // waves of resident blocks (no partly filled last wave)
  std::vector<int> rows_c = {16, 32, 64, 128};
  const long long nres = (long long)update_occupancy(ai) * P->nsm;
  for (int k = 1; nres > 0 && k <= 3; k++)
    rows_c.push_back((int)std::max<long long>(1, ((long long)P->R + k * nres - 1) / (k * nres)));
  std::sort(rows_c.begin(), rows_c.end());
  rows_c.erase(std::unique(rows_c.begin(), rows_c.end()), rows_c.end());
  double best_up = INFINITY;
  int best_rows = kRowsPerUpdateItem;
  for (int rows : rows_c) {
    TRY(set_decomposition(P, ai, best->var, best->nI, rows));
    TRY(prepare());
    double avg = 0.0;
    TRY(time_kernel(false, &avg));
    if (avg < best_up) {
      best_up = avg;
      best_rows = rows;
    }
  }
  best->rows = best_rows;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return set_decomposition(P, ai, best->var, best->nI, best->rows);
}

} // namespace
} // namespace pot3d

extern "C" int pot3d_autotune(pot3d_plan_t *plan, int flags, int *variant, int *chunks,
                              double *ms) {
  if (!plan || flags < 0 || flags > 7) return fail(POT3D_ERR_INVALID_ARG);
  Plan *P = reinterpret_cast<Plan *>(plan);
  if (flags == 0)
    flags = P->prec == POT3D_PREC_FP64 ? 1 : (P->prec == POT3D_PREC_FP64_DF ? 2 : 4);
  TuneVal last{0, 0, 0, 0.0};
  for (int ai = 0; ai < 3; ai++) {
    if (!(flags & (1 << ai))) continue;
    const TuneKey key{P->nr, P->nt, P->np, ai};
    TuneVal got{0, 0, 0, 0.0};
    bool cached = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tune_load_locked();
      auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        got = it->second;
        cached = true;
      }
    }
    int rc;
    if (cached) {
      rc = ensure_arith(P, ai);
      if (!rc) rc = set_decomposition(P, ai, got.var, got.nI, got.rows);
    } else if (ai == AR_F64) {
      rc = tune_arith<PF64>(P, ai, &got);
    } else if (ai == AR_DF) {
      rc = tune_arith<PDF>(P, ai, &got);
    } else {
      rc = tune_arith<PF32>(P, ai, &got);
    }
    if (rc) return fail(rc);
    if (!cached) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = got;
      tune_store_locked();
    }
    last = got;
  }
  if (variant) *variant = last.var;
  if (chunks) *chunks = last.nI;
  if (ms) *ms = last.ms;
  return POT3D_OK;
}

extern "C" int pot3d_variant_info(int arith, int variant, int *tile_rows, int *tile_cols,
                                  int *stages, int *blocks_per_sm) {
  if (arith < 0 || arith > 2 || variant < 0) return fail(POT3D_ERR_INVALID_ARG);
  int nv = 0;
  const MvVariant *vs = mv_variants(arith, &nv);
  if (variant >= nv) return fail(POT3D_ERR_INVALID_ARG);
  if (tile_rows) *tile_rows = vs[variant].tj;
  if (tile_cols) *tile_cols = vs[variant].tk;
  if (stages) *stages = vs[variant].stages;
  if (blocks_per_sm) *blocks_per_sm = vs[variant].blocks_per_sm;
  return POT3D_OK;
}

extern "C" int pot3d_set_decomposition(pot3d_plan_t *plan, int arith, int variant, int chunks,
                                       int update_rows) {
  if (!plan || arith < 0 || arith > 2 || variant < 0 || chunks < 0 || update_rows < 0)
    return fail(POT3D_ERR_INVALID_ARG);
  int nv = 0;
  mv_variants(arith, &nv);
  if (variant >= nv) return fail(POT3D_ERR_INVALID_ARG);
  Plan *P = reinterpret_cast<Plan *>(plan);
  int rc = ensure_arith(P, arith);
  if (!rc) rc = set_decomposition(P, arith, variant, chunks, update_rows);
  return rc ? fail(rc) : POT3D_OK;
}
