// Batched solves: many potential-field problems of different grid sizes
// advanced together by the same persistent kernels.
//
// Every admitted solve (a "slot") runs FP32 Jacobi PCG inside FP64 iterative
// refinement, the arithmetic of pot3d_solve_mixed, with vectors carved out of
// one device arena.  A step launches a captured CUDA graph of K iterations of
// k_matvec and k_update over the concatenated (slot, tile) work list; the
// kernels read the list and its length from device memory, so the graph
// survives admissions and retirements.  Between steps the host closes the
// refinement loop of the slots whose inner solve stopped.  Each slot keeps
// its plan's tile decomposition and its own fixed-order reductions, so a
// solve returns the same bits alone or in any mix.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "aux_kernels.cuh"
#include "plan.h"

namespace pot3d {

namespace {

constexpr int kBThreads = 256;
constexpr size_t kAlign = 256;

size_t al(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over one device buffer; free blocks are coalesced.
class Arena {
 public:
  void reset(size_t cap) {
    free_.clear();
    cap_ = cap;
    if (cap) free_[0] = cap;
  }
  // offset of a block of `bytes` (multiple of kAlign), or SIZE_MAX
  size_t alloc(size_t bytes) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        used_ += bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t capacity() const { return cap_; }

 private:
  std::map<size_t, size_t> free_;
  size_t cap_ = 0, used_ = 0;
};

enum SlotPhase { PH_FREE = 0, PH_START, PH_INNER, PH_DONE };

struct Slot {
  int phase = PH_FREE;
  long long tag = 0;
  Plan *plan = nullptr;
  const double *br = nullptr;
  double *phi = nullptr;
  double tol = 0.0;
  size_t off = 0, bytes = 0;
  float *v32[6] = {}; // x~, r, p~0, p~1, q; w (phi-line preconditioner)
  double *x64 = nullptr, *r64 = nullptr, *part_a = nullptr, *part_b = nullptr, *part_aux = nullptr;
  int2 *own_work = nullptr; // phi lines: this solve's update items, for its setup launches
  int *own_nwork = nullptr;
  int outer = 0, inner = 0, status = POT3D_OK, iter0 = 0;
  bool resumable = false; // the inner PCG stopped cleanly and may continue
  double relres = INFINITY, prev = INFINITY, scale = 1.0;
};

} // namespace

} // namespace pot3d

using namespace pot3d;

struct pot3d_batch {
  size_t max_bytes = 0;
  int max_slots = 0;
  int nsm = 0;
  char *arena_base = nullptr;
  Arena arena;
  std::vector<Slot> slots;
  ProbDev *d_probs = nullptr;
  SolveState *d_states = nullptr;
  TmaSet *d_tmas = nullptr;
  double *d_sums = nullptr; // [max_slots][4]: |b|^2, Dinv b^2 | |r|^2, Dinv r^2
  double *d_isums = nullptr; // [max_slots][2]: inner-system sums
  SolveState *h_states = nullptr;
  double *h_sums = nullptr;
  std::vector<ProbDev> h_probs;
  std::vector<TmaSet> h_tmas;
  int n_var = 0;          // FP32 matvec variants
  int2 *d_work = nullptr; // [n_var + 1][cap]: matvec items per variant, then update items
  int *d_nwork = nullptr; // [n_var + 1]
  int work_cap = 0;
  unsigned var_mask = 0, graph_mask = 0; // variants with work now / in the graph
  int cap_of[8] = {};                    // grid of each list in the captured graph
  bool line = false;                     // inner solves use the phi-line preconditioner
  int ring_pitch = 0;                    // phi lines: ring buffers of the captured graph
  bool dirty = true;
  cudaStream_t stream = nullptr, own_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_k = 0;
  pot3d_opts_t opts{};
  std::vector<int> finished; // slot indices retired by the last step, not yet polled
};

namespace pot3d {
using Batch = ::pot3d_batch;

namespace {

int grid_for(const Batch *B, size_t n) {
  size_t b = (n + kBThreads - 1) / kBThreads;
  return (int)std::max<size_t>(1, std::min<size_t>(b, (size_t)4 * B->nsm));
}

// Arena bytes of one solve: FP32 x~, r, p~0, p~1, q; FP64 x64, r64; the
// partial slots of its matvec and update items and of its FP64 reductions.
size_t slot_bytes(const Plan *P, int nsm, bool line) {
  const ArithData &D = P->ar[AR_F32];
  const size_t v4 = al(P->npad * 4), v8 = al(P->npad * 8);
  // closed wall: a balanced copy of Br
  const size_t brb = P->closed ? al(sizeof(double) * P->nt * P->np) : 0;
  // phi lines: w, and the solve's own update work list and its length
  const size_t lin = line ? v4 + al(sizeof(int2) * D.tiles_b) + al(sizeof(int)) : 0;
  return 5 * v4 + 2 * v8 + al(sizeof(double) * D.tiles_a) + al(sizeof(double) * 2 * D.tiles_b) +
         al(sizeof(double) * 2 * 4 * nsm) + brb + lin;
}

// Rebuild and upload the concatenated work lists of the occupied slots:
// one matvec list per FP32 variant (each slot uses its plan's variant) and
// one update list.
int rebuild_work(Batch *B) {
  const int nl = B->n_var + 1;
  std::vector<std::vector<int2>> lists(nl);
  for (int s = 0; s < B->max_slots; s++) {
    const Slot &S = B->slots[s];
    if (S.phase == PH_FREE || S.phase == PH_DONE) continue;
    const ArithData &D = S.plan->ar[AR_F32];
    for (int t = 0; t < D.tiles_a; t++) lists[D.var].push_back(make_int2(s, t));
    for (int t = 0; t < D.tiles_b; t++) lists[B->n_var].push_back(make_int2(s, t));
  }
  size_t need = 0;
  unsigned mask = 0;
  for (int v = 0; v < nl; v++) {
    need = std::max(need, lists[v].size());
    if (v < B->n_var && !lists[v].empty()) mask |= 1u << v;
  }
  if ((int)need > B->work_cap) {
    // grow before any graph uses the old list; the graph is re-captured
    if (B->d_work) cudaFree(B->d_work);
    B->work_cap = std::max((int)need, 2 * B->work_cap);
    if (cudaMalloc(&B->d_work, sizeof(int2) * nl * B->work_cap) != cudaSuccess) {
      cudaGetLastError();
      B->work_cap = 0;
      B->d_work = nullptr;
      return POT3D_ERR_OOM;
    }
    if (B->graph) cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  std::vector<int2> all((size_t)nl * B->work_cap, make_int2(0, 0));
  std::vector<int> counts(nl);
  for (int v = 0; v < nl; v++) {
    std::copy(lists[v].begin(), lists[v].end(), all.begin() + (size_t)v * B->work_cap);
    counts[v] = (int)lists[v].size();
  }
  if (B->work_cap &&
      cudaMemcpyAsync(B->d_work, all.data(), sizeof(int2) * all.size(), cudaMemcpyHostToDevice,
                      B->stream) != cudaSuccess)
    return POT3D_ERR_CUDA;
  if (cudaMemcpyAsync(B->d_nwork, counts.data(), sizeof(int) * nl, cudaMemcpyHostToDevice,
                      B->stream) != cudaSuccess)
    return POT3D_ERR_CUDA;
  // the host vectors above are pageable and local: finish the copies here
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) return POT3D_ERR_CUDA;
  B->var_mask = mask;
  if (B->line) {
    // ring buffers for the longest ring among the running solves
    int rp = 0;
    for (int s = 0; s < B->max_slots; s++) {
      const Slot &S = B->slots[s];
      if (S.phase != PH_FREE && S.phase != PH_DONE) rp = std::max(rp, S.plan->pitch);
    }
    if (rp > B->ring_pitch) {
      B->ring_pitch = rp;
      if (B->graph) cudaGraphExecDestroy(B->graph);
      B->graph = nullptr;
    }
  }
  // a captured graph launches cap_of[v] blocks per list: grow (and
  // re-capture) when a list outgrows it, in steps to limit re-captures
  for (int v = 0; v < nl; v++) {
    if (counts[v] > B->cap_of[v]) {
      B->cap_of[v] = std::max(counts[v], 2 * B->cap_of[v]);
      if (B->graph) cudaGraphExecDestroy(B->graph);
      B->graph = nullptr;
    }
  }
  B->dirty = false;
  return POT3D_OK;
}

// One iteration of every running slot: the matvec of each variant present,
// then the update.  Grids cover the work lists' capacity (the lists and their
// lengths are read from device memory; blocks past the length exit at once).
void launch_iteration(Batch *B) {
  int nv = 0;
  const MvVariant *vs = mv_variants(AR_F32, &nv);
  for (int v = 0; v < B->n_var; v++) {
    if (!(B->graph_mask & (1u << v))) continue;
    vs[v].launch(B->d_probs, B->d_work + (size_t)v * B->work_cap, B->d_nwork + v,
                 std::max(1, B->cap_of[v]), B->stream);
  }
  if (B->line) {
    update_line_launcher(AR_F32)(B->d_probs, B->d_work + (size_t)B->n_var * B->work_cap,
                                 B->d_nwork + B->n_var, std::max(1, B->cap_of[B->n_var]),
                                 B->ring_pitch, nullptr, B->stream);
    return;
  }
  update_launcher(AR_F32)(B->d_probs, B->d_work + (size_t)B->n_var * B->work_cap,
                          B->d_nwork + B->n_var, std::max(1, B->cap_of[B->n_var]), B->stream);
}

// FP64 residual r64 = b - L x64 of slot s and its sums (into d_sums[s][2..3]).
void launch_outer_residual(Batch *B, int s) {
  Slot &S = B->slots[s];
  Plan *P = S.plan;
  const int g = grid_for(B, P->n);
  k_op64<kBThreads><<<g, kBThreads, 0, B->stream>>>(S.x64, P->pitch, S.br, P->d_S, P->d_c64, P->nr,
                                                    P->nt, P->np, 0, S.r64, P->pitch, S.part_aux);
  k_sum_pairs<kBThreads><<<1, kBThreads, 0, B->stream>>>(S.part_aux, g, B->d_sums + 4 * s + 2);
}

// Starts (or, after a clean stop, resumes with the search direction kept)
// the inner FP32 solve of slot s on new_scale * r64.
void launch_inner_start(Batch *B, int s, double new_scale) {
  Slot &S = B->slots[s];
  Plan *P = S.plan;
  const int g = grid_for(B, P->n);
  const float *dinv32 = static_cast<const float *>(P->ar[AR_F32].coef);
  k_inner_rhs<kBThreads><<<g, kBThreads, 0, B->stream>>>(S.r64, dinv32, P->nr, P->nt, P->ntp, P->np,
                                                         P->pitch, new_scale, S.v32[1], S.part_aux);
  k_sum_pairs<kBThreads><<<1, kBThreads, 0, B->stream>>>(S.part_aux, g, B->d_isums + 2 * s);
  if (B->line) {
    // w = D T^-1 r32 and rho = r32 . T^-1 r32 of this solve replace its sums
    update_line_launcher(AR_F32)(B->d_probs, S.own_work, S.own_nwork, P->ar[AR_F32].tiles_b,
                                 P->pitch, B->d_isums + 2 * s, B->stream);
  }
  const size_t v4 = al(P->npad * 4);
  const bool restart = B->opts.mixed_restart != 0;
  const double inner_tol = B->opts.inner_tol > 0 ? B->opts.inner_tol : default_inner_tol(P, restart);
  cudaMemsetAsync(S.v32[0], 0, v4, B->stream);
  if (S.resumable && !restart) {
    S.iter0 = B->h_states[s].iter;
    k_resume<<<1, 1, 0, B->stream>>>(B->d_states + s, B->d_isums + 2 * s, S.scale / new_scale,
                                     inner_tol, segment_cap(P));
  } else {
    S.iter0 = 0;
    cudaMemsetAsync(S.v32[2], 0, v4, B->stream);
    cudaMemsetAsync(S.v32[3], 0, v4, B->stream);
    cudaMemsetAsync(S.v32[4], 0, v4, B->stream);
    const int maxit = B->opts.max_iters > 0 ? B->opts.max_iters : default_maxit(P);
    k_start<<<1, 1, 0, B->stream>>>(B->d_states + s, B->d_isums + 2 * s, (double)P->n, inner_tol,
                                    maxit, 0, 1.0, nullptr);
  }
  S.scale = new_scale;
}

void release_slot(Batch *B, int s) {
  Slot &S = B->slots[s];
  B->arena.release(S.off, S.bytes);
  S = Slot{};
}

// Close the refinement loop of the newly admitted slots and (unless
// starting_only) of every slot whose inner solve stopped in the step just
// polled: FP64 residual, convergence test, next inner solve or retirement.
int advance_outer(Batch *B, bool starting_only) {
  std::vector<int> todo;
  for (int s = 0; s < B->max_slots; s++) {
    Slot &S = B->slots[s];
    if (S.phase == PH_START) {
      todo.push_back(s);
    } else if (!starting_only && S.phase == PH_INNER && B->h_states[s].status != ST_RUNNING) {
      const SolveState &hs = B->h_states[s];
      S.inner += hs.iter - S.iter0;
      S.resumable = (hs.status == ST_CONVERGED);
      if (hs.status == ST_BREAKDOWN && hs.iter == S.iter0) {
        S.status = POT3D_ERR_BREAKDOWN;
        S.phase = PH_DONE;
        continue;
      }
      k_refine_update<<<grid_for(B, S.plan->n), kBThreads, 0, B->stream>>>(
          B->d_probs + s, S.plan->d_c64, S.x64, 1.0 / S.scale);
      S.outer++;
      todo.push_back(s);
    }
  }
  if (todo.empty()) return POT3D_OK;
  for (int s : todo) launch_outer_residual(B, s);
  if (cudaGetLastError() != cudaSuccess) return POT3D_ERR_CUDA;
  if (cudaMemcpyAsync(B->h_sums, B->d_sums, sizeof(double) * 4 * B->max_slots,
                      cudaMemcpyDeviceToHost, B->stream) != cudaSuccess ||
      cudaStreamSynchronize(B->stream) != cudaSuccess)
    return POT3D_ERR_CUDA;
  const bool restart = B->opts.mixed_restart != 0;
  const int max_outer = B->opts.max_outer > 0 ? B->opts.max_outer : (restart ? 30 : 200);
  for (int s : todo) {
    Slot &S = B->slots[s];
    const double bb = B->h_sums[4 * s], rr = B->h_sums[4 * s + 2];
    const double relres = bb > 0 ? std::sqrt(rr) / std::sqrt(bb) : 0.0;
    S.relres = relres;
    bool done = false;
    if (!std::isfinite(relres)) {
      S.status = POT3D_ERR_BREAKDOWN;
      done = true;
    } else if (relres <= S.tol) {
      S.status = POT3D_OK;
      done = true;
    } else if (S.outer >= max_outer || !(relres < (restart ? 0.5 : 1.0) * S.prev)) {
      S.status = POT3D_ERR_NOT_CONVERGED;
      done = true;
    }
    if (done) {
      Plan *P = S.plan;
      k_unpad<<<grid_for(B, P->n), kBThreads, 0, B->stream>>>(S.x64, P->pitch, S.phi, P->np, P->R,
                                                              P->np);
      gauge_phi(P, S.phi, S.part_aux, B->d_isums + 2 * s, B->stream);
      S.phase = PH_DONE;
      B->dirty = true;
      B->finished.push_back(s);
      continue;
    }
    S.prev = relres;
    launch_inner_start(B, s, std::ldexp(1.0, -std::ilogb(std::sqrt(rr / (double)S.plan->n))));
    S.phase = PH_INNER;
  }
  if (cudaGetLastError() != cudaSuccess) return POT3D_ERR_CUDA;
  return POT3D_OK;
}

} // namespace
} // namespace pot3d

using namespace pot3d;

extern "C" {

pot3d_batch_t *pot3d_batch_create(size_t max_bytes, int max_slots) {
  if (max_slots < 1 || max_slots > 4096 || max_bytes < kAlign) {
    fail(POT3D_ERR_INVALID_ARG);
    return nullptr;
  }
  Batch *B = new Batch();
  B->max_bytes = max_bytes & ~(kAlign - 1);
  B->max_slots = max_slots;
  B->slots.resize(max_slots);
  B->h_probs.resize(max_slots);
  B->h_tmas.resize(max_slots);
  int dev = 0;
  bool ok = cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaStreamCreateWithFlags(&B->own_stream, cudaStreamDefault) == cudaSuccess &&
            cudaMalloc(&B->arena_base, B->max_bytes) == cudaSuccess &&
            cudaMalloc(&B->d_probs, sizeof(ProbDev) * max_slots) == cudaSuccess &&
            cudaMalloc(&B->d_states, sizeof(SolveState) * max_slots) == cudaSuccess &&
            cudaMalloc(&B->d_tmas, sizeof(TmaSet) * max_slots) == cudaSuccess &&
            cudaMalloc(&B->d_sums, sizeof(double) * 4 * max_slots) == cudaSuccess &&
            cudaMalloc(&B->d_isums, sizeof(double) * 2 * max_slots) == cudaSuccess &&
            cudaMalloc(&B->d_nwork, sizeof(int) * 8) == cudaSuccess &&
            cudaMallocHost(&B->h_states, sizeof(SolveState) * max_slots) == cudaSuccess &&
            cudaMallocHost(&B->h_sums, sizeof(double) * 4 * max_slots) == cudaSuccess;
  if (ok) {
    B->stream = B->own_stream;
    ok = cudaMemset(B->d_states, 0, sizeof(SolveState) * max_slots) == cudaSuccess &&
         cudaMemset(B->d_nwork, 0, sizeof(int) * 8) == cudaSuccess;
    int nv = 0;
    const MvVariant *vs = mv_variants(AR_F32, &nv);
    B->n_var = nv;
    for (int v = 0; v < nv && ok; v++) ok = vs[v].setup() == 0;
  }
  if (!ok) {
    cudaGetLastError();
    fail(POT3D_ERR_OOM);
    pot3d_batch_destroy(reinterpret_cast<pot3d_batch_t *>(B));
    return nullptr;
  }
  memset(B->h_states, 0, sizeof(SolveState) * max_slots);
  B->arena.reset(B->max_bytes);
  return reinterpret_cast<pot3d_batch_t *>(B);
}

void pot3d_batch_destroy(pot3d_batch_t *batch) {
  if (!batch) return;
  Batch *B = reinterpret_cast<Batch *>(batch);
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  cudaFree(B->arena_base);
  cudaFree(B->d_probs);
  cudaFree(B->d_states);
  cudaFree(B->d_tmas);
  cudaFree(B->d_sums);
  cudaFree(B->d_isums);
  cudaFree(B->d_work);
  cudaFree(B->d_nwork);
  if (B->h_states) cudaFreeHost(B->h_states);
  if (B->h_sums) cudaFreeHost(B->h_sums);
  if (B->own_stream) cudaStreamDestroy(B->own_stream);
  cudaGetLastError();
  delete B;
}

int pot3d_batch_set_stream(pot3d_batch_t *batch, void *stream) {
  if (!batch) return fail(POT3D_ERR_INVALID_ARG);
  Batch *B = reinterpret_cast<Batch *>(batch);
  B->stream = stream ? (cudaStream_t)stream : B->own_stream;
  return POT3D_OK;
}

int pot3d_batch_set_opts(pot3d_batch_t *batch, const pot3d_opts_t *o) {
  if (!batch || !o || o->inner_tol < 0 || !(o->inner_tol < 1.0) || o->max_outer < 0 ||
      o->max_iters < 0)
    return fail(POT3D_ERR_INVALID_ARG);
  if (o->precond < 0 || o->precond > 4) return fail(POT3D_ERR_INVALID_ARG);
  // the radial-line and subdomain-ILU(0) kernels work on one problem per launch
  if (o->precond == POT3D_PC_R_LINE || o->precond == POT3D_PC_LINES || o->precond == POT3D_PC_ILU)
    return fail(POT3D_ERR_UNSUPPORTED);
  Batch *B = reinterpret_cast<Batch *>(batch);
  const bool line = o->precond == POT3D_PC_PHI_LINE;
  if (line != B->line) {
    // the slot layout and the kernels depend on it: only an empty batch changes
    for (const Slot &S : B->slots)
      if (S.phase != PH_FREE) return fail(POT3D_ERR_BUSY);
    B->line = line;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  B->opts = *o;
  return POT3D_OK;
}

size_t pot3d_batch_bytes_needed(pot3d_batch_t *batch, const pot3d_plan_t *plan) {
  if (!batch || !plan) return 0;
  Plan *P = reinterpret_cast<Plan *>(const_cast<pot3d_plan_t *>(plan));
  if (ensure_arith(P, AR_F32)) return 0;
  return slot_bytes(P, reinterpret_cast<Batch *>(batch)->nsm, reinterpret_cast<Batch *>(batch)->line);
}

int pot3d_batch_submit(pot3d_batch_t *batch, pot3d_plan_t *plan, const double *br, double tol,
                       double *phi, long long tag) {
  if (!batch || !plan || !br || !phi || !(tol > 0.0) || !std::isfinite(tol))
    return fail(POT3D_ERR_INVALID_ARG);
  if (!is_device_ptr(br) || !is_device_ptr(phi)) return fail(POT3D_ERR_INVALID_ARG);
  Batch *B = reinterpret_cast<Batch *>(batch);
  Plan *P = reinterpret_cast<Plan *>(plan);
  int s = -1;
  for (int u = 0; u < B->max_slots; u++)
    if (B->slots[u].phase == PH_FREE) {
      s = u;
      break;
    }
  if (s < 0) return POT3D_ERR_BUSY;
  int rc = ensure_arith(P, AR_F32);
  if (!rc && B->line) rc = ensure_line(P, AR_F32);
  if (rc) return fail(rc);
  const ArithData &D = P->ar[AR_F32];
  const size_t bytes = slot_bytes(P, B->nsm, B->line);
  const size_t off = B->arena.alloc(bytes);
  if (off == SIZE_MAX) return POT3D_ERR_BUSY;
  Slot &S = B->slots[s];
  S = Slot{};
  S.phase = PH_START;
  S.tag = tag;
  S.plan = P;
  S.br = br;
  S.phi = phi;
  S.tol = tol;
  S.off = off;
  S.bytes = bytes;
  char *p = B->arena_base + off;
  const size_t v4 = al(P->npad * 4), v8 = al(P->npad * 8);
  for (int v = 0; v < 5; v++) S.v32[v] = reinterpret_cast<float *>(p + v * v4);
  p += 5 * v4;
  S.x64 = reinterpret_cast<double *>(p);
  S.r64 = reinterpret_cast<double *>(p + v8);
  p += 2 * v8;
  S.part_a = reinterpret_cast<double *>(p);
  p += al(sizeof(double) * D.tiles_a);
  S.part_b = reinterpret_cast<double *>(p);
  p += al(sizeof(double) * 2 * D.tiles_b);
  S.part_aux = reinterpret_cast<double *>(p);
  p += al(sizeof(double) * 2 * 4 * B->nsm);
  if (P->closed) {
    // the balanced Br this solve uses (zero net flux)
    double *brb = reinterpret_cast<double *>(p);
    prepare_br(P, br, brb, S.part_aux, B->d_isums + 2 * s, B->stream);
    S.br = brb;
    p += al(sizeof(double) * P->nt * P->np);
  }
  if (B->line) {
    S.v32[5] = reinterpret_cast<float *>(p);
    p += v4;
    S.own_work = reinterpret_cast<int2 *>(p);
    p += al(sizeof(int2) * D.tiles_b);
    S.own_nwork = reinterpret_cast<int *>(p);
    std::vector<int2> ow(D.tiles_b);
    for (int t = 0; t < D.tiles_b; t++) ow[t] = make_int2(s, t);
    const int cnt = D.tiles_b;
    // pageable sources: these copies complete before the calls return
    if (cudaMemcpyAsync(S.own_work, ow.data(), sizeof(int2) * ow.size(), cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess ||
        cudaMemcpyAsync(S.own_nwork, &cnt, sizeof(int), cudaMemcpyHostToDevice, B->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(B->stream) != cudaSuccess) {
      release_slot(B, s);
      return fail(POT3D_ERR_CUDA);
    }
  }
  // descriptor and TMA maps of the slot
  ProbDev &h = B->h_probs[s];
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
  h.x = S.v32[0];
  h.r = S.v32[1];
  h.p0 = S.v32[2];
  h.p1 = S.v32[3];
  h.q = S.v32[4];
  h.coef = P->ar[AR_F32].coef;
  h.part_a = S.part_a;
  h.part_b = S.part_b;
  h.st = B->d_states + s;
  h.tma = B->d_tmas + s;
  h.w = B->line ? S.v32[5] : nullptr;
  h.lcoef = B->line ? P->ar[AR_F32].lcoef : nullptr;
  TmaSet &T = B->h_tmas[s];
  int nv = 0;
  rc = encode_tma_set(&T, h, h.coef, mv_variants(AR_F32, &nv)[D.var], P);
  cudaStream_t st = B->stream;
  if (!rc && (cudaMemcpyAsync(B->d_probs + s, &h, sizeof(ProbDev), cudaMemcpyHostToDevice, st) !=
                  cudaSuccess ||
              cudaMemcpyAsync(B->d_tmas + s, &T, sizeof(TmaSet), cudaMemcpyHostToDevice, st) !=
                  cudaSuccess))
    rc = POT3D_ERR_CUDA;
  if (rc) {
    release_slot(B, s);
    return fail(rc);
  }
  // x64 = 0 and zeroed FP32 vectors (padding included); ||b||^2 for the
  // refinement test
  cudaMemsetAsync(B->arena_base + off, 0, 5 * v4 + 2 * v8, st);
  if (B->line) cudaMemsetAsync(S.v32[5], 0, v4, st);
  const size_t n0 = (size_t)P->nt * P->np;
  const int gb = grid_for(B, n0);
  k_bstats<kBThreads><<<gb, kBThreads, 0, st>>>(S.br, P->d_S, P->d_c64, P->nr, P->nt, P->np,
                                                S.part_aux);
  k_sum_pairs<kBThreads><<<1, kBThreads, 0, st>>>(S.part_aux, gb, B->d_sums + 4 * s);
  SolveState idle{};
  idle.status = ST_CONVERGED; // not iterating until its first inner start
  cudaMemcpyAsync(B->d_states + s, &idle, sizeof(SolveState), cudaMemcpyHostToDevice, st);
  if (cudaGetLastError() != cudaSuccess) {
    release_slot(B, s);
    return fail(POT3D_ERR_CUDA);
  }
  B->dirty = true;
  return POT3D_OK;
}

// Advances every admitted solve by up to k inner iterations, then closes the
// refinement loop where an inner solve stopped.  Returns the number of solves
// still running (>= 0) or an error.
int pot3d_batch_step(pot3d_batch_t *batch, int k) {
  if (!batch || k < 1 || k > 4096) return fail(POT3D_ERR_INVALID_ARG);
  Batch *B = reinterpret_cast<Batch *>(batch);
  // newly admitted slots get their first FP64 residual and inner start
  int rc = advance_outer(B, true);
  if (rc) return fail(rc);
  if (B->dirty) {
    rc = rebuild_work(B);
    if (rc) return fail(rc);
  }
  int running = 0;
  for (const Slot &S : B->slots) running += (S.phase == PH_INNER);
  if (running) {
    if (!B->graph || B->graph_k != k || B->graph_mask != B->var_mask) {
      B->graph_mask = B->var_mask;
      if (B->graph) cudaGraphExecDestroy(B->graph);
      B->graph = nullptr;
      cudaGraph_t g;
      if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(POT3D_ERR_CUDA);
      for (int c = 0; c < k; c++) launch_iteration(B);
      if (cudaStreamEndCapture(B->stream, &g) != cudaSuccess) return fail(POT3D_ERR_CUDA);
      cudaError_t e = cudaGraphInstantiate(&B->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_status(e);
      B->graph_k = k;
    }
    if (cudaGraphLaunch(B->graph, B->stream) != cudaSuccess) return fail(POT3D_ERR_CUDA);
  }
  if (cudaMemcpyAsync(B->h_states, B->d_states, sizeof(SolveState) * B->max_slots,
                      cudaMemcpyDeviceToHost, B->stream) != cudaSuccess ||
      cudaStreamSynchronize(B->stream) != cudaSuccess)
    return fail(POT3D_ERR_CUDA);
  for (int s = 0; s < B->max_slots; s++) {
    if (B->slots[s].phase == PH_INNER && B->h_states[s].status == ST_TIMEOUT)
      return fail(POT3D_ERR_TIMEOUT);
  }
  rc = advance_outer(B, false);
  if (rc) return fail(rc);
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) return fail(POT3D_ERR_CUDA);
  running = 0;
  for (const Slot &S : B->slots) running += (S.phase == PH_INNER || S.phase == PH_START);
  return running;
}

// Retires finished solves: writes up to max entries and frees their memory.
int pot3d_batch_poll(pot3d_batch_t *batch, long long *tags, int *status, int *outer, int *inner,
                     double *relres, int max, int *n_done) {
  if (!batch || !n_done || max < 0) return fail(POT3D_ERR_INVALID_ARG);
  Batch *B = reinterpret_cast<Batch *>(batch);
  int n = 0;
  std::vector<int> keep;
  for (int s : B->finished) {
    if (n >= max) {
      keep.push_back(s);
      continue;
    }
    const Slot &S = B->slots[s];
    if (tags) tags[n] = S.tag;
    if (status) status[n] = S.status;
    if (outer) outer[n] = S.outer;
    if (inner) inner[n] = S.inner;
    if (relres) relres[n] = S.relres;
    release_slot(B, s);
    n++;
  }
  B->finished.swap(keep);
  *n_done = n;
  return POT3D_OK;
}

int pot3d_batch_info(pot3d_batch_t *batch, int *active, size_t *bytes_used, size_t *bytes_cap) {
  if (!batch) return fail(POT3D_ERR_INVALID_ARG);
  Batch *B = reinterpret_cast<Batch *>(batch);
  int a = 0;
  for (const Slot &S : B->slots) a += (S.phase != PH_FREE);
  if (active) *active = a;
  if (bytes_used) *bytes_used = B->arena.used();
  if (bytes_cap) *bytes_cap = B->arena.capacity();
  return POT3D_OK;
}

} // extern "C"
