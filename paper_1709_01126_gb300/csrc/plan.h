// Internal plan object shared by the translation units of libpot3d.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "kernels.cuh"
#include "pot3d.h"
#include "variants.h"

namespace pot3d {

enum { AR_F64 = 0, AR_DF = 1, AR_F32 = 2 };

constexpr int kAuxThreads = 256;
constexpr int kRowsPerUpdateItem = 32;

// Per-arithmetic device state of a plan.
struct ArithData {
  // work decomposition: matvec variant, tiles (theta x phi x r-chunks) and
  // update items (kRowsPerUpdateItem phi rows each)
  int var = 0;
  int nJ = 0, nK = 0, ic = 0, nI = 0, tiles_a = 0, rows_b = 0, tiles_b = 0;
  int cap_a = 0, cap_b = 0; // allocated work-list / partial capacity
  int2 *d_work_a = nullptr, *d_work_b = nullptr;
  int *d_nwork = nullptr; // [tiles_a, tiles_b]
  void *coef = nullptr; // scaled metric table [6][nr][ntp] in the arithmetic's type
  void *lcoef = nullptr; // phi-line table [6][nr][ntp] (see ensure_line)
  void *rcoef = nullptr; // radial-line table [4][nr][ntp] (see ensure_rline)
  double *part_c = nullptr; // [2 * tiles_c] radial-line partials
  int tiles_c = 0;
  void *icoef = nullptr;    // PC2 table (see ensure_ilu)
  double *part_i = nullptr; // [2 * tiles_i] PC2 partials
  int tiles_i = 0;
  int graph_pc = 0; // the preconditioner the captured graph launches (POT3D_PC_*)
  ProbDev *d_prob = nullptr;
  SolveState *d_state = nullptr;
  double *part_a = nullptr, *part_b = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_chunk = 0;
  cudaStream_t graph_stream = nullptr;
  ProbDev h_prob{};
  TmaSet *d_tma = nullptr;
  TmaSet h_tma{};
  bool ready = false;
};

struct Plan {
  int nr = 0, nt = 0, np = 0, pitch = 0, prec = 0;
  int ntp = 0; // metric-table row pitch (nt rounded up to 4)
  size_t R = 0, n = 0, npad = 0;
  // host mesh (Sec. 2.2) and tables
  std::vector<double> rf, tf, rc, tc, drc, dtc;
  double dphi = 0.0;
  std::vector<double> c64h, S, irs, its, irc, isd, fwt, fwp, fwpole;
  // device constant tables
  double *d_c64 = nullptr, *d_S = nullptr, *d_irs = nullptr, *d_its = nullptr, *d_irc = nullptr,
         *d_isd = nullptr, *d_poles = nullptr, *d_fwt = nullptr, *d_fwp = nullptr,
         *d_fwpole = nullptr;
  ArithData ar[3];
  // workspace (vectors)
  char *ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  // reductions outside the iteration
  int aux_blocks = 0;
  double *d_part = nullptr;
  double *d_sums = nullptr;
  double *h_sums = nullptr;    // pinned [8]
  SolveState *h_state = nullptr; // pinned, two snapshots: [0] is the final state of a solve
  cudaEvent_t poll_ev[2] = {nullptr, nullptr};
  double *d_br_last = nullptr; // Br of the last solve (closed wall: balanced)
  bool have_br = false;
  // closed wall (Br = 0 at r1): the operator is singular; Br is balanced to
  // zero net flux and Phi gauged to zero mean
  bool closed = false;
  double inv_area = 0.0;        // 1 / (np sum_j S_j): inner-face area
  double *d_br_tmp = nullptr;   // balanced copy of a Br given to field / residual
  double *d_stage = nullptr;
  size_t stage_bytes = 0;
  cudaStream_t stream = nullptr, own_stream = nullptr, user_stream = nullptr;
  pot3d_opts_t opts{};
  pot3d_stats_t stats{};
  int nsm = 0;
  std::vector<cudaEvent_t> ev;
  bool freeze_poll = false; // testing hook: the host re-reads a stale state snapshot
  bool line = false;         // the solve in progress runs the phi-line update
  bool rline = false;        // the solve in progress runs the radial-line kernel
  bool ilu = false;          // the solve in progress runs the PC2 kernel
  double *d_hist = nullptr;  // residual history of the last PCG run (opts.history)
  int hist_alloc = 0, hist_n = 0;
};

int fail(int code);
int cuda_status(cudaError_t e);
bool is_device_ptr(const void *p);
int plan_device_init(Plan *P);
void plan_free(Plan *P);
int ensure_arith(Plan *P, int ai);
// phi-line table of arithmetic ai (AR_F64 or AR_F32), built on first use
int ensure_line(Plan *P, int ai);
// radial-line table and partials of arithmetic ai (AR_F64 or AR_F32), built on first use
int ensure_rline(Plan *P, int ai);
// radial-line blocks of a plan (8 warps of 32 phi columns of one theta row)
int rline_tiles(const Plan *P);
// PC2 table and partials of arithmetic ai (AR_F64 or AR_F32), built on first use
int ensure_ilu(Plan *P, int ai);
// PC2 blocks of a plan (kIluThreads / 32 boxes of nr x 1 x 32 cells each)
int ilu_tiles(const Plan *P);
size_t workspace_bytes(const Plan *P);
int ensure_workspace(Plan *P);
void *ws_vec(const Plan *P, int v, size_t es);
double *ws_x64(const Plan *P);
double *ws_r64(const Plan *P);
int stage(Plan *P, size_t bytes);
void scaled_table(const Plan *P, std::vector<double> &t);
int encode3d(CUtensorMap *m, void *base, int es, const Plan *P, int bx, int by);
int encode_coef_map(CUtensorMap *m, const void *coef, int es, const Plan *P, int tj);
int set_decomposition(Plan *P, int ai, int var, int nI, int rows_b);
int heuristic_chunks(const Plan *P, const MvVariant &v);
int encode_tma_set(TmaSet *T, const ProbDev &h, const void *coef, const MvVariant &v,
                   const Plan *P);
int default_maxit(const Plan *P);
// Inner tolerance of mixed refinement when the options give none.
double default_inner_tol(const Plan *P, bool restart);
int segment_cap(const Plan *P);
// Br prepared for the right-hand side on stream s: a copy (source surface)
// or Br without its area-weighted mean (closed wall), written to out;
// part holds at least 2 * 4 * nsm doubles of block partials, sum one double pair.
void prepare_br(const Plan *P, const double *br, double *out, double *part, double *sum,
                cudaStream_t s);
// The closed-wall gauge of a dense Phi on stream s (no-op for the source surface).
void gauge_phi(const Plan *P, double *phi, double *part, double *sum, cudaStream_t s);

} // namespace pot3d
