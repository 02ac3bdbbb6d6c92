/*
 * pot3d.h — C ABI of the GB300 potential-field solver (libpot3d.so).
 *
 * Solves the finite-difference spherical Laplace equation for a coronal
 * potential field (arXiv:1709.01126):
 *   - Sec. 2.1, Eq. 1: Laplace equation for the scalar potential Phi,
 *     B = grad Phi.
 *   - Sec. 2.1, Eq. 2: inner boundary dPhi/dr = Br at r = r0 (the photosphere).
 *   - Sec. 2.1: outer boundary "source surface" Phi = 0 at r = r1, or the
 *     closed wall Br = 0 there; phi periodic.
 *   - Sec. 2.1, Eq. 3: polar boundary value = phi-average of Phi half a cell
 *     from the pole.
 *   - Sec. 2.2 and Eq. 4: second-order 7-point finite-difference operator on
 *     a logically rectangular grid, nonuniform in r and theta, here in its
 *     symmetric volume-weighted form (the r^2 metric factors restored).
 *   - Sec. 2.3: preconditioned conjugate gradient with point-Jacobi /
 *     diagonal scaling (PC1) or with the non-overlapping domain
 *     decomposition with ILU(0) per subdomain (PC2); line preconditioners
 *     beside them, of the vectorisable kind Sec. 6 asks for.
 *
 * Grid convention: Phi is cell-centred in r, theta and phi.  Unknowns are
 * Phi[i][j][k], i < nr (r), j < nt (theta, from the north pole), k < np
 * (phi), stored densely in C order with k fastest (element (i*nt + j)*np + k).
 *
 * Pointers.  Array arguments marked "dev or host" may be device pointers
 * (cudaMalloc / torch CUDA tensors; no copy) or host pointers (staged
 * through device memory inside the call; pinned host memory makes those
 * copies asynchronous).  All GPU work runs on the plan's stream (set with
 * pot3d_set_stream; default: a blocking stream the plan creates, ordered
 * with the legacy default stream).  A call that
 * returns a result on the host (iteration counts, residuals) synchronises
 * that stream before returning.
 *
 * Errors.  Functions return POT3D_OK (0) or a negative POT3D_ERR_* code;
 * pot3d_plan returns NULL and records the code for pot3d_last_error().
 * pot3d_strerror maps a code to a static string.  No call aborts the
 * process; device-side waits are bounded and report POT3D_ERR_TIMEOUT.
 *
 * Threads.  One plan must not be used from two host threads at once.
 * Different plans are independent.
 */
#ifndef POT3D_H
#define POT3D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define POT3D_OK 0
#define POT3D_ERR_INVALID_ARG (-1)  /* bad dimension, pointer, tolerance or option */
#define POT3D_ERR_OOM (-2)          /* device or host allocation failed            */
#define POT3D_ERR_CUDA (-3)         /* a CUDA runtime call failed                  */
#define POT3D_ERR_NOT_CONVERGED (-4)/* iteration cap reached; phi = last iterate   */
#define POT3D_ERR_BREAKDOWN (-5)    /* PCG breakdown: p.Ap <= 0 or not finite      */
#define POT3D_ERR_TIMEOUT (-6)      /* a bounded device-side wait gave up          */
#define POT3D_ERR_UNSUPPORTED (-7)  /* option not implemented                      */
#define POT3D_ERR_BUSY (-8)         /* batch full / no memory to admit now         */
#define POT3D_ERR_TOO_LARGE (-9)    /* request needs more than a fixed-size buffer */

/* ---- arithmetic of the PCG iteration ------------------------------- */
#define POT3D_PREC_FP64 0    /* every operation in native FP64                      */
#define POT3D_PREC_FP64_DF 1 /* FP64-class: vectors as (hi, lo) float pairs, every  */
                             /* operation in double-float arithmetic on FP32 units  */
#define POT3D_PREC_MIXED 2   /* FP32 inner PCG inside FP64 iterative refinement     */

/* ---- preconditioner of the PCG iteration ------------------------------ */
#define POT3D_PC_JACOBI 0   /* diagonal scaling z = D^-1 r (PC1, Sec. 2.3)             */
#define POT3D_PC_PHI_LINE 1 /* phi-line Jacobi: z = T^-1 r with T the part of L that
                               couples the cells of one (r, theta) ring (diagonal and
                               both phi neighbours, periodic): a cyclic tridiagonal
                               solve per ring, the stronger line preconditioner of
                               the kind Sec. 6 calls for.  FP64 and MIXED plans       */
#define POT3D_PC_R_LINE 2   /* radial-line Jacobi: z = T_r^-1 r with T_r the part of L
                               inside each radial column (diagonal and both r
                               neighbours): one tridiagonal solve per (theta, phi)
                               column.  Radial couplings dominate where the r mesh is
                               stretched (thin cells near r0).  FP64 and MIXED plans  */
#define POT3D_PC_LINES 3    /* both line directions, additively:
                               M^-1 = T_r^-1 + T_phi^-1 - D^-1.  It is SPD: scaled
                               by D^1/2 on both sides it is I + f(K_r) + f(K_phi),
                               f(K) = K (I - K)^-1 with K one direction's scaled
                               couplings (eigenvalues in (-1, 1)), and each f(K) has
                               eigenvalues above -1/2.  FP64 and MIXED plans          */
#define POT3D_PC_ILU 4      /* PC2 of Sec. 2.3: non-overlapping domain decomposition
                               with a zero-fill incomplete LU factorisation (ILU(0))
                               of every subdomain's block of L, couplings between
                               subdomains dropped.  The subdomains are boxes of every
                               r cell x 1 theta row x 32 phi columns (the last box of
                               a row takes the remainder; a box never closes the phi
                               ring, so np must exceed 32, else the solve returns
                               POT3D_ERR_UNSUPPORTED).  For the 7-point pattern
                               ILU(0) keeps L's couplings and changes only the
                               diagonal, so M = (P + E) P^-1 (P + E^T), E the strict
                               lower part of the box block and P the pivots.  FP64
                               and MIXED plans                                        */

/* ---- boundary conditions (Sec. 2.1) ---------------------------------- */
#define POT3D_OUTER_SOURCE_SURFACE 0 /* Phi = 0 at r = r1                              */
#define POT3D_OUTER_CLOSED_WALL 1    /* Br = dPhi/dr = 0 at r = r1.  The operator is then
                                        singular (constants are its null space): every
                                        call that forms the right-hand side first removes
                                        Br's area-weighted mean over the inner face (zero
                                        net flux), and every returned Phi has zero mean
                                        over the cells                                  */
#define POT3D_POLE_AVERAGE 0         /* Eq. 3                                          */

typedef struct pot3d_plan pot3d_plan_t;

/* Grid description (Sec. 2.2).  nr >= 2, nt >= 2, np >= 3.
 * Radial faces: r_faces[nr+1] (host, strictly increasing) if non-NULL, else
 * from r0 to r1 with cell widths dr_i = dr_1 * r_ratio^(i-1) (r_ratio = 1:
 * uniform).  Colatitude faces: t_faces[nt+1] (host, 0 .. pi, strictly
 * increasing) if non-NULL, else uniform j*pi/nt.  phi faces are uniform.
 * The face arrays are copied; the caller keeps ownership. */
typedef struct {
  int nr, nt, np;
  double r0, r1;
  double r_ratio;
  const double *r_faces;
  const double *t_faces;
  int precision; /* POT3D_PREC_* */
} pot3d_grid_t;

typedef struct {
  int outer; /* POT3D_OUTER_* */
  int pole;  /* POT3D_POLE_* */
} pot3d_bc_t;

/* Solver options; zero-initialised fields take the defaults. */
typedef struct {
  int max_iters;      /* PCG iteration cap (inner cap for MIXED); 0: 100*(nr+nt+np) */
  int use_x0;         /* 1: phi holds the initial guess on entry of pot3d_solve      */
  int chunk;          /* iterations enqueued between host polls; 0: automatic        */
  int use_graphs;     /* 0: automatic (graphs on), 1: on, -1: off                    */
  int time_kernels;   /* 1: time every iteration kernel with CUDA events (no graphs) */
  double inner_tol;   /* MIXED: the inner FP32 PCG hands over to an FP64 refinement
                         step once its residual fell by this factor (0: with
                         mixed_restart = 0, 0.5 for grids of 8M unknowns or more
                         and 0.1 below; with mixed_restart = 1, 1e-4)           */
  int max_outer;      /* MIXED: refinement cap (0: 30 restarts, 200 replacements)    */
  int mixed_restart;  /* MIXED: 0 = after each FP64 step the inner PCG continues on
                         the replaced residual with its search direction kept
                         (reliable updates; a segment that needs more than
                         20*(nr+nt+np) iterations ends and the next one
                         restarts); 1 = it always restarts from zero (plain
                         defect correction)                                      */
  int verify;         /* FP64 and FP64_DF: 0 = stop when the PCG recurrence residual
                         reaches tol (the paper's stopping rule); 1 = then also
                         recompute ||b - L Phi|| / ||b|| in FP64 and, while it is
                         above tol, restart PCG from Phi with that residual (at
                         most 10 restarts, within max_iters in total).  stats
                         report the FP64 residual and the restarts (outer_iters).
                         MIXED always stops on the FP64 residual.                */
  int precond;        /* POT3D_PC_*: the preconditioner.  The line preconditioners
                         and PC2 run with FP64 or MIXED plans (a FP64_DF solve
                         returns POT3D_ERR_UNSUPPORTED); batches take POT3D_PC_JACOBI and
                         POT3D_PC_PHI_LINE (pot3d_batch_set_opts returns
                         POT3D_ERR_UNSUPPORTED for the others)                  */
  int history;        /* FP64 and FP64_DF: 1 = record the recurrence residual
                         ||r_k|| / ||b|| of every iteration k = 0 .. iters of the
                         next solves (with verify: of the last restart), read back
                         with pot3d_get_history; 0 = off                          */
} pot3d_opts_t;

/* pot3d_stats_t.flags bits */
#define POT3D_FLAG_ABOVE_TOL 1 /* the recomputed FP64 residual of the returned Phi
                                  is above tol although the PCG recurrence
                                  residual met it (the solve still returns
                                  POT3D_OK: the paper's stopping rule)          */

/* Residual history of the last FP64 / FP64_DF solve run with opts.history:
 * copies min(cap, iters + 1) values ||r_k|| / ||b||, k = 0, 1, ..., into
 * relres (host) and their count into *n.  POT3D_ERR_INVALID_ARG when no
 * history was recorded. */
int pot3d_get_history(const pot3d_plan_t *plan, double *relres, int cap, int *n);

/* Statistics of the last solve on a plan. */
typedef struct {
  int status;          /* return code of the last solve                         */
  int iters;           /* PCG iterations (MIXED: total inner FP32 iterations)   */
  int outer_iters;     /* MIXED: refinement steps; verify: restarts (else 0)    */
  double relres;       /* final ||r||/||b||: PCG recurrence residual (FP64, DF)
                          or the recomputed FP64 residual (MIXED, verify)       */
  double kernel_ms[4]; /* with time_kernels: summed event time of the matvec     */
                       /* kernel, the update kernel, and their launch counts     */
  long long launches;  /* kernels the last solve or field call launched          */
  double relres_fp64;  /* ||b - L Phi|| / ||b|| of the returned Phi, recomputed
                          in FP64 after every solve (one operator application)  */
  int flags;           /* POT3D_FLAG_* bits                                      */
  double sigma;        /* p.Ap of the last PCG iteration, as the device summed it
                          (inner FP32 system for MIXED: scaled units)           */
  double rr;           /* ||r||^2 of the last PCG iteration, as summed (same)    */
} pot3d_stats_t;

/* Static facts about a plan (for measurement and sizing). */
typedef struct {
  long long n;               /* unknowns nr*nt*np                                */
  int pitch;                 /* padded phi length of the internal vectors        */
  int tiles_matvec;          /* work items of the matvec kernel                  */
  int tiles_update;          /* work items of the update kernel                  */
  size_t workspace_bytes;    /* device workspace a solve needs                   */
  double bytes_matvec;       /* algorithmic HBM bytes per matvec-kernel launch   */
  double bytes_update;       /* algorithmic HBM bytes per update-kernel launch   */
} pot3d_info_t;

/* Builds the mesh, the per-(r,theta) metric and diagonal tables and uploads
 * them (device memory owned by the plan).  Returns NULL on error
 * (pot3d_last_error()). */
pot3d_plan_t *pot3d_plan(const pot3d_grid_t *grid, const pot3d_bc_t *bc);

/* Frees everything the plan owns (not a workspace given by the caller). */
void pot3d_destroy(pot3d_plan_t *plan);

int pot3d_set_stream(pot3d_plan_t *plan, void *cuda_stream);
int pot3d_set_opts(pot3d_plan_t *plan, const pot3d_opts_t *opts);
int pot3d_get_info(const pot3d_plan_t *plan, pot3d_info_t *info);
int pot3d_last_stats(const pot3d_plan_t *plan, pot3d_stats_t *stats);

/* Autotuner: times every matvec tile-shape variant and r-chunk count, then
 * the update kernel's rows per work item (16, 32, 64, 128), of the selected
 * arithmetics on this plan's problem (a few launches each, on the plan's
 * stream, with the plan's workspace) and keeps the fastest for later
 * solves (pot3d_get_info reports the resulting work-item counts).  flags: bit 0 FP64, bit 1 double-float, bit 2 FP32 (the inner
 * solve of refinement and batches); 0 = the plan's own precision.  Results
 * are cached per (nr, nt, np, arithmetic) for the process and, when the
 * environment names a file in POT3D_TUNE_CACHE, across processes.
 * variant / chunks / ms (may be NULL) receive the choice for the last
 * arithmetic tuned: variant index, r-chunks per tile column, and the matvec
 * time in ms measured when the choice was made. */
int pot3d_autotune(pot3d_plan_t *plan, int flags, int *variant, int *chunks, double *ms);

/* Matvec kernel variants of arithmetic `arith` (0 FP64, 1 double-float,
 * 2 FP32): for variant index `variant`, the tile shape (theta rows x phi
 * columns), the number of TMA stages and the blocks per SM the kernel's
 * register budget targets.  Output pointers may be NULL.  Returns
 * POT3D_ERR_INVALID_ARG when `arith` or `variant` is out of range, so a
 * caller can enumerate variants 0, 1, ... until it fails. */
int pot3d_variant_info(int arith, int variant, int *tile_rows, int *tile_cols, int *stages,
                       int *blocks_per_sm);

/* Manual kernel configuration of arithmetic `arith` on this plan, instead of
 * pot3d_autotune: matvec variant, r-chunks per tile column (0: heuristic,
 * clamped to nr) and update rows per work item (0: 32).  Later solves use
 * it until the next pot3d_autotune or pot3d_set_decomposition.  Every
 * configuration computes the same operator and iteration; only the
 * rounding order of the block reductions differs.  POT3D_ERR_INVALID_ARG
 * for an unknown arithmetic or variant or a negative count. */
int pot3d_set_decomposition(pot3d_plan_t *plan, int arith, int variant, int chunks,
                            int update_rows);

/* Device workspace.  By default the plan allocates it with cudaMalloc at
 * the first solve.  A caller that manages device memory itself passes a
 * buffer of at least pot3d_workspace_bytes() bytes, 256-byte aligned; it
 * stays owned by the caller and must outlive the plan's use of it. */
size_t pot3d_workspace_bytes(const pot3d_plan_t *plan);
int pot3d_set_workspace(pot3d_plan_t *plan, void *dev_ptr, size_t bytes);

/* Solves L Phi = b(Br) to ||r||/||b|| <= tol (Sec. 2.3 with PC1; stopping
 * rule checked after every iteration, x0 = 0 unless opts.use_x0).
 *   br   [nt*np]      dev or host, read      inner-boundary Br (Eq. 2)
 *   phi  [nr*nt*np]   dev or host, written   the solution (initial guess
 *                                            when opts.use_x0)
 *   iters             host, may be NULL      iterations taken
 * Returns POT3D_OK, POT3D_ERR_NOT_CONVERGED (phi = last iterate),
 * POT3D_ERR_BREAKDOWN, or an argument / CUDA error.  The arithmetic is the
 * plan's precision. */
int pot3d_solve(pot3d_plan_t *plan, const double *br, double tol, double *phi, int *iters);

/* FP64 iterative refinement around FP32 PCG (any plan precision):
 * outer_iters / inner_iters (host, may be NULL) receive the refinement
 * steps and the total inner iterations.  Stops when the FP64 residual
 * ||b - L phi|| / ||b|| <= tol. */
int pot3d_solve_mixed(pot3d_plan_t *plan, const double *br, double tol, double *phi,
                      int *outer_iters, int *inner_iters);

/* Field B = grad Phi on staggered faces (Sec. 2.1; poles by Eq. 3).
 *   phi [nr*nt*np]    dev or host, read
 *   br  [nt*np]       dev or host, read; NULL = the Br of the last solve
 *   B                 dev or host, written: three contiguous blocks
 *       Br  [(nr+1)*nt*np]   radial faces, inner face first (= input Br)
 *       Bth [nr*(nt+1)*np]   colatitude faces, north pole face first
 *       Bph [nr*nt*np]       phi faces between k and k+1 (periodic)   */
int pot3d_field(pot3d_plan_t *plan, const double *phi, const double *br, double *B);

/* y = L x with the FP64 operator of Eq. 4 (no boundary right-hand side).
 *   x, y [nr*nt*np]  dev or host.  */
int pot3d_apply(pot3d_plan_t *plan, const double *x, double *y);

/* FP64 relative residual ||b(Br) - L phi|| / ||b(Br)||. br, phi dev or host. */
int pot3d_residual(pot3d_plan_t *plan, const double *br, const double *phi, double *relres);

/* The same residual as pot3d_residual for callers that cannot allocate
 * device memory during the call (device memory owned by another allocator,
 * a fixed memory budget, or code where an allocation would synchronise the
 * device).  The paper has no counterpart; this is a library convenience.
 *   br [nt*np], phi [nr*nt*np]   device pointers only (host arrays would need
 *                                a staging copy: POT3D_ERR_INVALID_ARG)
 *   relres                       host, written
 * Allocates nothing: the plan (created beforehand) supplies its tables (and,
 * with the closed wall, its own buffer for the balanced Br), and the
 * per-block partial sums go to a 32 KiB scratch array compiled into the
 * library (4096 doubles, room for 2046 blocks; the call launches at most
 * 4 x SMs blocks and returns POT3D_ERR_TOO_LARGE if that exceeds the room).
 * Every GPU that loads the library holds the array until the process exits.
 * The first call on each device (each device context) looks up the array's
 * device address, so it should come before any stream capture.  The call
 * reads its result back to the host and synchronises the plan's stream
 * before it returns.  All calls share the array and every slot a call reads
 * is written earlier in the same call: calls whose kernels overlap on the
 * GPU race; order them on one stream.  The result agrees with
 * pot3d_residual to rounding. */
int pot3d_residual_noalloc(pot3d_plan_t *plan, const double *br, const double *phi,
                           double *relres);

/* Self-test of the device-side wait limit (failure detection without a
 * fault): one block waits, through the same bounded mbarrier wait the
 * iteration kernels use, on a barrier that nothing completes, for
 * limit_s seconds (0 < limit_s <= 10).  *device_status receives the status
 * the kernel reported, POT3D_ERR_TIMEOUT when the wait gave up as designed;
 * *elapsed_s (may be NULL) the device time the wait took.  Runs on the legacy
 * default stream and synchronises it.  Returns POT3D_OK if the test ran. */
int pot3d_selftest_wait(double limit_s, int *device_status, double *elapsed_s);

/* Measurement helper: the native FP64 fused multiply-add rate of the current
 * device, the roofline denominator of the FP64 iteration (no counterpart in
 * the paper).  Runs a kernel of independent DFMA chains on every SM for at
 * least min_seconds of device time (0 < min_seconds <= 5) on the legacy
 * default stream and synchronises it.  *fma_per_s receives the measured
 * DFMA per second (one DFMA = 2 flop); *elapsed_s (may be NULL) the timed
 * device seconds.  Returns POT3D_OK, or POT3D_ERR_INVALID_ARG / a CUDA error. */
int pot3d_probe_fp64_fma(double min_seconds, double *fma_per_s, double *elapsed_s);

/* Testing hook for the host-side progress guard (failure detection without
 * a fault): with on = 1 the host keeps re-reading the first solver-state
 * snapshot of a solve, as if the device state had stopped advancing, so the
 * guard ends the solve with POT3D_ERR_TIMEOUT after two polls.  The kernels
 * already queued run to completion before the call returns; the plan stays
 * usable.  on = 0 restores normal polling. */
int pot3d_test_freeze_poll(pot3d_plan_t *plan, int on);

/* ---- batched solves (continuous batching) ------------------------------
 * Many solves of different grids advance together in the same persistent
 * kernels: each admitted solve runs the arithmetic of pot3d_solve_mixed
 * (FP32 PCG inside FP64 refinement, the plan's tile decomposition and its own
 * fixed-order reductions, so its result is bitwise the same as
 * pot3d_solve_mixed on the same plan, alone or in any mix).
 * pot3d_batch_create: max_bytes of device arena (allocated once) and up to
 *   max_slots concurrent solves.  NULL on error (pot3d_last_error()).
 * pot3d_batch_submit: admits a solve if a slot and arena memory are free
 *   (else POT3D_ERR_BUSY, nothing changed).  br [nt*np] and phi [nr*nt*np]
 *   are device pointers that must stay valid until the solve is polled;
 *   phi receives the solution.  The plan may be shared by many solves.
 * pot3d_batch_step: advances every admitted solve by up to k inner
 *   iterations (one CUDA graph of k iterations) and runs the refinement
 *   step of those whose inner solve stopped.  Returns the number of solves
 *   still running, or an error.
 * pot3d_batch_poll: retires up to max finished solves, writing their tag,
 *   status, refinement steps, inner iterations and final FP64 relative
 *   residual (any output pointer may be NULL), and frees their memory.
 * One batch must not be used from two host threads at once. */
typedef struct pot3d_batch pot3d_batch_t;
pot3d_batch_t *pot3d_batch_create(size_t max_bytes, int max_slots);
void pot3d_batch_destroy(pot3d_batch_t *batch);
int pot3d_batch_set_stream(pot3d_batch_t *batch, void *cuda_stream);
int pot3d_batch_set_opts(pot3d_batch_t *batch, const pot3d_opts_t *opts);
size_t pot3d_batch_bytes_needed(pot3d_batch_t *batch, const pot3d_plan_t *plan);
int pot3d_batch_submit(pot3d_batch_t *batch, pot3d_plan_t *plan, const double *br, double tol,
                       double *phi, long long tag);
int pot3d_batch_step(pot3d_batch_t *batch, int k);
int pot3d_batch_poll(pot3d_batch_t *batch, long long *tags, int *status, int *outer_iters,
                     int *inner_iters, double *relres, int max, int *n_done);
int pot3d_batch_info(pot3d_batch_t *batch, int *active, size_t *bytes_used, size_t *bytes_cap);

int pot3d_last_error(void);
const char *pot3d_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* POT3D_H */
