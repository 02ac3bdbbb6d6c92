/*
 * Plain FP64 CPU oracle for the POT3D potential-field solve (arXiv:1709.01126).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The GPU
 * library shares no code, header, table or constant generator with this file.
 *
 * Everything here is written for a reader checking it against the paper:
 * each step is a separate loop, written in the order the method states it,
 * with no fusion or blocking.  OpenMP only splits loops over points; every
 * reduction is combined in a fixed order (per-thread partials summed in
 * thread order), so results are deterministic for a given thread count.
 *
 * Discretisation (Sec. 2.1 Eqs. 1-3, Sec. 2.2 stencil, Eq. 4):
 *   - Phi is cell-centred in r, theta and phi: unknowns Phi[i][j][k],
 *     i<nr, j<nt, k<np, stored in C order with phi fastest.
 *   - The operator is the finite-volume form of the spherical Laplacian,
 *     multiplied by the cell volume r_i^2 dr_i sin(th_j) dth_j dphi and
 *     negated, which makes it symmetric positive definite:
 *        (L x)_c = sum over faces f of c_f * (x_c - x_nb(f))
 *     with face coefficients
 *        c^r  (face r_{i+1/2})  = r_{i+1/2}^2 sin(th_j) dth_j dphi / (r_{i+1}-r_i)
 *        c^th (face th_{j+1/2}) = dr_i sin(th_{j+1/2}) dphi / (th_{j+1}-th_j)
 *        c^ph (both phi faces)  = dr_i dth_j / (sin(th_j) dphi)
 *     The paper's printed stencil omits the r^2 and 1/r^2 metric factors;
 *     this file restores them (the only reading that is symmetric, as
 *     Sec. 2.3 says A is).
 *   - Inner boundary r=R_sun (Eq. 2): dPhi/dr = Br is a prescribed flux; the
 *     face carries no coupling and moves to the right-hand side
 *        b_c = -r_{1/2}^2 sin(th_j) dth_j dphi Br[j][k]   (i = 0 only).
 *   - Outer boundary r=R_1, source surface Phi=0 (Sec. 2.1): mirror ghost
 *     Phi_ghost = -Phi_c at spacing 2 (R_1 - r_last), i.e. a coupling
 *     2 c^r_outer x_c on the last radial layer.
 *   - Outer boundary alternative, closed wall Br = dPhi/dr = 0 at R_1
 *     (Sec. 2.1, orc_set_outer(1)): the outer face carries no flux, like the
 *     inner face without its Br.  L is then singular (constants are its null
 *     space); the right-hand side must have zero net flux, so the inner Br
 *     loses its area-weighted mean (the discrete monopole) before b is
 *     formed, and a solution is defined up to a constant: orc_remove_mean
 *     gives the representative with zero mean over the cells.
 *   - Poles (Eq. 3): the pole faces have sin(0) = sin(pi) = 0 area, so they
 *     carry no coupling in L; Eq. 3 enters through the field evaluation,
 *     where the ghost cell across the pole is set so that the face value is
 *     the phi-average of the first ring (half a cell from the pole).
 *   - phi is periodic: k-1 and k+1 wrap modulo np.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* status codes returned by orc_pcg */
#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_BREAKDOWN 2
#define ORC_BAD_ARG 3

typedef struct {
  int nr, nt, np;
  double dphi;
  double *rf, *rc, *dr; /* r faces [nr+1], centres [nr], widths [nr]    */
  double *tf, *tc, *dt; /* th faces [nt+1], centres [nt], widths [nt]   */
  double *cr;           /* c^r on face r_{i+1/2}, i = 0..nr-1 (last = outer face) : [nr*nt] */
  double *ct;           /* c^th on face th_{j+1/2}, j = 0..nt-2 : [nr*(nt-1)]               */
  double *cp;           /* c^ph : [nr*nt]                                                      */
  double *diag;         /* diagonal of L : [nr*nt] (independent of k)                          */
} orc_op;

static int g_threads = 0;
static int g_outer_closed = 0; /* 0: source surface Phi = 0; 1: closed wall Br = 0 */
static int g_precond = 0; /* 0: point Jacobi (PC1); 1: radial lines; 2: phi lines;
                            3: both line directions; 4: subdomain ILU(0) (PC2) */
/* PC2 subdomain box: cells in r, theta, phi (0 = the whole extent) */
static int g_blk[3] = {0, 1, 32};

/* Preconditioner of orc_pcg (line preconditioners are of the kind Sec. 6
 * asks for: stronger than diagonal scaling, yet every line independent):
 *   0 = diagonal scaling (PC1 of Sec. 2.3);
 *   1 = radial-line Jacobi: M is the part of L that couples cells of one
 *       (theta, phi) column (the full diagonal and the two radial
 *       neighbours); z = M^-1 r is one tridiagonal solve per column;
 *   2 = phi-line Jacobi: M is the part of L that couples cells of one
 *       (r, theta) ring (the full diagonal and the two periodic phi
 *       neighbours); z = M^-1 r is one cyclic tridiagonal solve per ring;
 *   3 = both line directions, added: M^-1 = T_r^-1 + T_phi^-1 - D^-1 with
 *       T_r, T_phi the radial-line and phi-line parts above and D the
 *       diagonal.  It is symmetric positive definite: scaled by D^1/2 on
 *       both sides it is I + f(K_r) + f(K_phi), f(K) = K (I - K)^-1, where
 *       K = D^-1/2 C D^-1/2 holds one line direction's couplings C; the
 *       eigenvalues l of K lie in (-1, 1), so those of f(K), l / (1 - l),
 *       exceed -1/2, and the sum stays above 0;
 *   4 = PC2 of Sec. 2.3: non-overlapping domain decomposition with a
 *       zero-fill incomplete LU factorisation (ILU(0)) of each subdomain's
 *       block of L.  The subdomains are boxes of g_blk cells (orc_set_blocks;
 *       the last box of each direction holds the remainder); couplings
 *       between boxes are dropped (block Jacobi over the subdomains), a box
 *       that spans the whole phi ring keeps the periodic coupling inside
 *       it.  Within a box the unknowns are numbered in C order (r slowest,
 *       phi fastest).  For the 7-point pattern any lexicographic numbering
 *       with every axis ascending orients each coupling the same way (the
 *       cell with the larger r, theta or phi index comes later), so the
 *       paper's r-fastest FORTRAN numbering gives the same factors. */
int orc_set_precond(int kind) {
  if (kind < 0 || kind > 4) return 3;
  g_precond = kind;
  return 0;
}

/* Box of the PC2 subdomains: bi x bj x bk cells (0 = the whole extent). */
int orc_set_blocks(int bi, int bj, int bk) {
  if (bi < 0 || bj < 0 || bk < 0) return 3;
  g_blk[0] = bi;
  g_blk[1] = bj;
  g_blk[2] = bk;
  return 0;
}

/* Outer boundary condition used by every later call: 0 = source surface,
 * 1 = closed wall. */
int orc_set_outer(int kind) {
  if (kind != 0 && kind != 1) return 3;
  g_outer_closed = kind;
  return 0;
}

void orc_set_threads(int n) {
  g_threads = n;
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------- mesh */

/* Radial faces from r0 to r1.  ratio == 1: uniform.  Otherwise geometric:
 * cell widths dr_i = dr_1 ratio^(i-1) summing to r1 - r0 (Sec. 2.2:
 * the grid is nonuniform in r). */
int orc_r_faces(int nr, double r0, double r1, double ratio, double *rf) {
  if (nr < 1 || !(r1 > r0) || !(ratio > 0)) return ORC_BAD_ARG;
  if (ratio == 1.0) {
    for (int i = 0; i <= nr; i++) rf[i] = r0 + (r1 - r0) * (double)i / (double)nr;
  } else {
    double dr1 = (r1 - r0) * (ratio - 1.0) / (pow(ratio, (double)nr) - 1.0);
    for (int i = 0; i <= nr; i++) rf[i] = r0 + dr1 * (pow(ratio, (double)i) - 1.0) / (ratio - 1.0);
  }
  rf[0] = r0;
  rf[nr] = r1;
  return ORC_OK;
}

/* Uniform theta faces j*pi/nt, j = 0..nt. */
int orc_t_faces(int nt, double *tf) {
  if (nt < 1) return ORC_BAD_ARG;
  for (int j = 0; j <= nt; j++) tf[j] = ORC_PI * (double)j / (double)nt;
  tf[0] = 0.0;
  tf[nt] = ORC_PI;
  return ORC_OK;
}

static void op_free(orc_op *op) {
  free(op->rf); free(op->rc); free(op->dr);
  free(op->tf); free(op->tc); free(op->dt);
  free(op->cr); free(op->ct); free(op->cp); free(op->diag);
}

/* sin of a theta face; the two pole faces are exactly zero (Eq. 3 reading:
 * the pole face has no area). */
static double sin_face(const orc_op *op, int jf) {
  if (jf == 0 || jf == op->nt) return 0.0;
  return sin(op->tf[jf]);
}

static int op_build(orc_op *op, int nr, int nt, int np, const double *rf, const double *tf) {
  memset(op, 0, sizeof(*op));
  if (nr < 1 || nt < 2 || np < 2) return ORC_BAD_ARG;
  op->nr = nr; op->nt = nt; op->np = np;
  op->dphi = 2.0 * ORC_PI / (double)np;
  op->rf = malloc(sizeof(double) * (nr + 1));
  op->rc = malloc(sizeof(double) * nr);
  op->dr = malloc(sizeof(double) * nr);
  op->tf = malloc(sizeof(double) * (nt + 1));
  op->tc = malloc(sizeof(double) * nt);
  op->dt = malloc(sizeof(double) * nt);
  op->cr = malloc(sizeof(double) * nr * nt);
  op->ct = malloc(sizeof(double) * nr * (nt > 1 ? nt - 1 : 1));
  op->cp = malloc(sizeof(double) * nr * nt);
  op->diag = malloc(sizeof(double) * nr * nt);
  if (!op->rf || !op->rc || !op->dr || !op->tf || !op->tc || !op->dt || !op->cr || !op->ct ||
      !op->cp || !op->diag) {
    op_free(op);
    return ORC_BAD_ARG;
  }
  memcpy(op->rf, rf, sizeof(double) * (nr + 1));
  memcpy(op->tf, tf, sizeof(double) * (nt + 1));
  for (int i = 0; i < nr; i++) {
    op->rc[i] = 0.5 * (rf[i] + rf[i + 1]);
    op->dr[i] = rf[i + 1] - rf[i];
  }
  for (int j = 0; j < nt; j++) {
    op->tc[j] = 0.5 * (tf[j] + tf[j + 1]);
    op->dt[j] = tf[j + 1] - tf[j];
  }
  const double dphi = op->dphi;
  for (int i = 0; i < nr; i++) {
    for (int j = 0; j < nt; j++) {
      /* radial face r_{i+1/2}: between centres i and i+1, or (outer face)
         between centre nr-1 and its mirror ghost at 2 R_1 - r_{nr-1}. */
      double rface = rf[i + 1];
      double spacing = (i < nr - 1) ? (op->rc[i + 1] - op->rc[i]) : 2.0 * (rf[nr] - op->rc[nr - 1]);
      op->cr[i * nt + j] = rface * rface * sin(op->tc[j]) * op->dt[j] * dphi / spacing;
      /* closed wall: no flux through the outer face */
      if (i == nr - 1 && g_outer_closed) op->cr[i * nt + j] = 0.0;
      op->cp[i * nt + j] = op->dr[i] * op->dt[j] / (sin(op->tc[j]) * dphi);
    }
    for (int j = 0; j + 1 < nt; j++) {
      op->ct[i * (nt - 1) + j] =
          op->dr[i] * sin_face(op, j + 1) * dphi / (op->tc[j + 1] - op->tc[j]);
    }
  }
  /* diagonal: L applied to a unit vector at c, read back at c */
  for (int i = 0; i < nr; i++) {
    for (int j = 0; j < nt; j++) {
      double d = 0.0;
      if (i < nr - 1) d += op->cr[i * nt + j];
      else d += 2.0 * op->cr[i * nt + j];
      if (i > 0) d += op->cr[(i - 1) * nt + j];
      if (j < nt - 1) d += op->ct[i * (nt - 1) + j];
      if (j > 0) d += op->ct[i * (nt - 1) + j - 1];
      d += 2.0 * op->cp[i * nt + j];
      op->diag[i * nt + j] = d;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------ operator */

static void op_apply(const orc_op *op, const double *x, double *y) {
  const int nr = op->nr, nt = op->nt, np = op->np;
  const long plane = (long)nt * np;
#pragma omp parallel for schedule(static)
  for (long rowid = 0; rowid < (long)nr * nt; rowid++) {
    int i = (int)(rowid / nt), j = (int)(rowid % nt);
    const double cr_out = op->cr[i * nt + j];
    const double cr_in = (i > 0) ? op->cr[(i - 1) * nt + j] : 0.0;
    const double ct_n = (j < nt - 1) ? op->ct[i * (nt - 1) + j] : 0.0;
    const double ct_s = (j > 0) ? op->ct[i * (nt - 1) + j - 1] : 0.0;
    const double cphi = op->cp[i * nt + j];
    for (int k = 0; k < np; k++) {
      long c = rowid * np + k;
      double xc = x[c];
      double s = 0.0;
      if (i < nr - 1) s += cr_out * (xc - x[c + plane]);
      else s += cr_out * (xc - (-xc)); /* source surface: mirror ghost */
      if (i > 0) s += cr_in * (xc - x[c - plane]);
      /* i == 0: prescribed-flux face, handled by the right-hand side */
      if (j < nt - 1) s += ct_n * (xc - x[c + np]);
      if (j > 0) s += ct_s * (xc - x[c - np]);
      /* pole faces: zero area, no coupling */
      int kp = (k + 1) % np, km = (k + np - 1) % np;
      s += cphi * (xc - x[rowid * np + kp]);
      s += cphi * (xc - x[rowid * np + km]);
      y[c] = s;
    }
  }
}

/* ------------------------------------------------------ preconditioner */

/* z = M^-1 r.  PC1: z = r / diag.  Radial lines: for each column (j, k) the
 * tridiagonal system with diagonal diag[i][j], sub- and super-diagonal
 * -cr[i][j] between cells i and i+1, solved by Gaussian elimination without
 * pivoting (the Thomas algorithm: forward elimination, back substitution;
 * the matrix is symmetric and diagonally dominant, so no pivoting is
 * needed). */
/* Tridiagonal solve (Thomas algorithm) of rows i = 0..n-1:
 * a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i, a_0 and c_{n-1} unused;
 * cp, dp: n doubles of workspace. */
static void thomas(int n, const double *a, const double *b, const double *c, const double *d,
                   double *x, double *cp, double *dp) {
  cp[0] = c[0] / b[0];
  dp[0] = d[0] / b[0];
  for (int i = 1; i < n; i++) {
    const double m = b[i] - a[i] * cp[i - 1];
    cp[i] = c[i] / m;
    dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; i--) x[i] = dp[i] - cp[i] * x[i + 1];
}

/* Cyclic tridiagonal solve, diagonal dg, both off-diagonals (including the
 * two corners that close the ring) equal to off: the Sherman-Morrison
 * formula around one tridiagonal matrix B (A = B + u v^T with
 * u = (g, 0, .., 0, off), v = (1, 0, .., 0, off / g), g = -dg), two Thomas
 * solves B y = d and B w = u, then x = y - (v.y) / (1 + v.w) w.
 * n >= 3; work: 7 n doubles. */
static void cyclic_solve(int n, double dg, double off, const double *d, double *x, double *work) {
  double *a = work, *b = work + n, *c = work + 2 * n, *u = work + 3 * n, *w = work + 4 * n;
  double *cp = work + 5 * n, *dp = work + 6 * n;
  const double g = -dg;
  for (int i = 0; i < n; i++) {
    a[i] = off;
    b[i] = dg;
    c[i] = off;
    u[i] = 0.0;
  }
  b[0] = dg - g;
  b[n - 1] = dg - off * off / g;
  u[0] = g;
  u[n - 1] = off;
  thomas(n, a, b, c, d, x, cp, dp);
  thomas(n, a, b, c, u, w, cp, dp);
  const double vy = x[0] + (off / g) * x[n - 1];
  const double vw = w[0] + (off / g) * w[n - 1];
  const double f = vy / (1.0 + vw);
  for (int i = 0; i < n; i++) x[i] -= f * w[i];
}

static void precond_jacobi(const orc_op *op, const double *r, double *z) {
  const long n = (long)op->nr * op->nt * op->np;
  const int np = op->np;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < n; c++) z[c] = r[c] / op->diag[c / np];
}

static void precond_philine(const orc_op *op, const double *r, double *z) {
  const int nr = op->nr, nt = op->nt, np = op->np;
#pragma omp parallel
  {
    double *work = malloc(sizeof(double) * 7 * (np > 3 ? np : 3));
#pragma omp for schedule(static)
    for (long row = 0; row < (long)nr * nt; row++) {
      const double dg = op->diag[row], off = -op->cp[row];
      const double *rr = r + row * np;
      double *zz = z + row * np;
      if (np == 2) {
        /* both phi faces couple to the one other cell: [[dg, 2 off], [2 off, dg]] */
        const double det = dg * dg - 4.0 * off * off;
        zz[0] = (dg * rr[0] - 2.0 * off * rr[1]) / det;
        zz[1] = (dg * rr[1] - 2.0 * off * rr[0]) / det;
      } else {
        cyclic_solve(np, dg, off, rr, zz, work);
      }
    }
    free(work);
  }
}

static void precond_rline(const orc_op *op, const double *r, double *z) {
  const int nr = op->nr, nt = op->nt, np = op->np;
  const long plane = (long)nt * np;
  /* The coefficients of a column depend on (i, j) only, so the columns of
     one theta row are eliminated together, plane by plane (contiguous
     accesses); each column still goes through the same operations in the
     same order as a column-by-column Thomas solve. */
#pragma omp parallel
  {
    double *cp = malloc(sizeof(double) * nr);            /* modified super-diagonal */
    double *dp = malloc(sizeof(double) * (long)nr * np); /* modified right-hand sides */
#pragma omp for schedule(static)
    for (int j = 0; j < nt; j++) {
      /* row i: a_i z_{i-1} + b_i z_i + c_i z_{i+1} = r_i with
         a_i = -cr[i-1][j], b_i = diag[i][j], c_i = -cr[i][j] */
      for (int i = 0; i < nr; i++) {
        const double a = (i > 0) ? -op->cr[(i - 1) * nt + j] : 0.0;
        const double b = op->diag[i * nt + j];
        const double c = (i < nr - 1) ? -op->cr[i * nt + j] : 0.0;
        const double *ri = r + (long)i * plane + (long)j * np;
        double *di = dp + (long)i * np;
        if (i == 0) {
          cp[0] = c / b;
          for (int k = 0; k < np; k++) di[k] = ri[k] / b;
        } else {
          const double m = b - a * cp[i - 1];
          cp[i] = c / m;
          const double *dm = dp + (long)(i - 1) * np;
          for (int k = 0; k < np; k++) di[k] = (ri[k] - a * dm[k]) / m;
        }
      }
      double *zl = z + (long)(nr - 1) * plane + (long)j * np;
      for (int k = 0; k < np; k++) zl[k] = dp[(long)(nr - 1) * np + k];
      for (int i = nr - 2; i >= 0; i--) {
        double *zi = z + (long)i * plane + (long)j * np;
        const double *zn = zi + plane;
        for (int k = 0; k < np; k++) zi[k] = dp[(long)i * np + k] - cp[i] * zn[k];
      }
    }
    free(cp);
    free(dp);
  }
}

/* ------------------------------------------------- PC2: subdomain ILU(0) */

/* The block-diagonal matrix of the subdomain blocks of L in box order
 * (box by box, C order inside a box), stored in CSR with sorted columns,
 * factored in place by ILU(0): below the diagonal the multipliers of the
 * unit lower factor, on and above it the upper factor. */
typedef struct {
  long n, nbox;
  long *perm;   /* perm[m]: unknown index (C order of the grid) of box-order row m */
  long *bstart; /* [nbox + 1]: first box-order row of each box */
  long *rowptr; /* [n + 1] */
  long *col;    /* box-order column indices */
  double *val;
  long *dpos;   /* position of each row's diagonal entry */
} orc_ilu;

static void ilu_free(orc_ilu *f) {
  free(f->perm); free(f->bstart); free(f->rowptr); free(f->col); free(f->val); free(f->dpos);
  memset(f, 0, sizeof(*f));
}

/* number of boxes of extent b (0: one box) along an axis of n cells */
static int nboxes(int n, int b) { return (b <= 0 || b >= n) ? 1 : (n + b - 1) / b; }
static int boxlen(int n, int b) { return (b <= 0 || b >= n) ? n : b; }

/* Assemble the subdomain blocks of L and factor each by ILU(0), Saad,
 * Iterative Methods for Sparse Linear Systems, Algorithm 10.4 (IKJ form):
 *   for each row i, for each k < i with (i, k) in NZ(A), in column order:
 *     a_ik := a_ik / a_kk;
 *     for each j > k with (i, j) in NZ(A):  a_ij := a_ij - a_ik a_kj
 * (a_kj taken as 0 where (k, j) is not in NZ(A): no fill).  Returns ORC_OK,
 * ORC_BREAKDOWN when a pivot is not positive, ORC_BAD_ARG on allocation
 * failure. */
static int ilu_build(const orc_op *op, orc_ilu *f) {
  memset(f, 0, sizeof(*f));
  const int nr = op->nr, nt = op->nt, np = op->np;
  const long n = (long)nr * nt * np, plane = (long)nt * np;
  const int Li = boxlen(nr, g_blk[0]), Lj = boxlen(nt, g_blk[1]), Lk = boxlen(np, g_blk[2]);
  const int Bi = nboxes(nr, g_blk[0]), Bj = nboxes(nt, g_blk[1]), Bk = nboxes(np, g_blk[2]);
  f->n = n;
  f->nbox = (long)Bi * Bj * Bk;
  f->perm = malloc(sizeof(long) * n);
  f->bstart = malloc(sizeof(long) * (f->nbox + 1));
  f->rowptr = malloc(sizeof(long) * (n + 1));
  f->col = malloc(sizeof(long) * 7 * n);
  f->val = malloc(sizeof(double) * 7 * n);
  f->dpos = malloc(sizeof(long) * n);
  long *inv = malloc(sizeof(long) * n);
  if (!f->perm || !f->bstart || !f->rowptr || !f->col || !f->val || !f->dpos || !inv) {
    free(inv);
    ilu_free(f);
    return ORC_BAD_ARG;
  }
  /* box order: boxes in C order of their box indices, cells in C order */
  long m = 0, b = 0;
  for (int bi = 0; bi < Bi; bi++)
    for (int bj = 0; bj < Bj; bj++)
      for (int bk = 0; bk < Bk; bk++) {
        f->bstart[b++] = m;
        for (int i = bi * Li; i < nr && i < (bi + 1) * Li; i++)
          for (int j = bj * Lj; j < nt && j < (bj + 1) * Lj; j++)
            for (int k = bk * Lk; k < np && k < (bk + 1) * Lk; k++) {
              const long c = (long)i * plane + (long)j * np + k;
              f->perm[m] = c;
              inv[c] = m;
              m++;
            }
      }
  f->bstart[f->nbox] = n;
  /* rows: the couplings of L whose two cells lie in the same box */
  long nnz = 0;
  f->rowptr[0] = 0;
  for (long row = 0; row < n; row++) {
    const long c = f->perm[row];
    const int i = (int)(c / plane), j = (int)((c / np) % nt), k = (int)(c % np);
    const long box = ((long)(i / Li) * Bj + j / Lj) * Bk + k / Lk;
    long cols[8];
    double vals[8];
    int cnt = 0;
    cols[cnt] = row; vals[cnt] = op->diag[i * nt + j]; cnt++;
    /* neighbour (ii, jj, kk) with coupling -coef, kept if in the same box */
#define ORC_NB(ii, jj, kk, coef)                                                              \
  do {                                                                                       \
    const long nbbox = ((long)((ii) / Li) * Bj + (jj) / Lj) * Bk + (kk) / Lk;               \
    if (nbbox == box) {                                                                      \
      cols[cnt] = inv[(long)(ii) * plane + (long)(jj) * np + (kk)];                          \
      vals[cnt] = -(coef);                                                                   \
      cnt++;                                                                                 \
    }                                                                                        \
  } while (0)
    if (i < nr - 1) ORC_NB(i + 1, j, k, op->cr[i * nt + j]);
    if (i > 0) ORC_NB(i - 1, j, k, op->cr[(i - 1) * nt + j]);
    if (j < nt - 1) ORC_NB(i, j + 1, k, op->ct[i * (nt - 1) + j]);
    if (j > 0) ORC_NB(i, j - 1, k, op->ct[i * (nt - 1) + j - 1]);
    const int kp = (k + 1) % np, km = (k + np - 1) % np;
    if (kp == km) {
      /* np == 2: both phi faces couple to the one other cell */
      ORC_NB(i, j, kp, 2.0 * op->cp[i * nt + j]);
    } else {
      ORC_NB(i, j, kp, op->cp[i * nt + j]);
      ORC_NB(i, j, km, op->cp[i * nt + j]);
    }
#undef ORC_NB
    for (int a = 1; a < cnt; a++) {
      long cc = cols[a]; double vv = vals[a]; int q = a - 1;
      while (q >= 0 && cols[q] > cc) { cols[q + 1] = cols[q]; vals[q + 1] = vals[q]; q--; }
      cols[q + 1] = cc; vals[q + 1] = vv;
    }
    for (int a = 0; a < cnt; a++) {
      if (cols[a] == row) f->dpos[row] = nnz;
      f->col[nnz] = cols[a];
      f->val[nnz] = vals[a];
      nnz++;
    }
    f->rowptr[row + 1] = nnz;
  }
  free(inv);
  /* ILU(0), box by box (no coupling crosses a box) */
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (long bx = 0; bx < f->nbox; bx++) {
    for (long i = f->bstart[bx]; i < f->bstart[bx + 1]; i++) {
      for (long e = f->rowptr[i]; e < f->rowptr[i + 1] && f->col[e] < i; e++) {
        const long k = f->col[e];
        const double piv = f->val[f->dpos[k]];
        if (!(piv > 0.0)) { bad = 1; break; }
        f->val[e] /= piv;
        for (long g = e + 1; g < f->rowptr[i + 1]; g++) {
          const long jcol = f->col[g];
          for (long h = f->rowptr[k]; h < f->rowptr[k + 1]; h++) {
            if (f->col[h] == jcol) { f->val[g] -= f->val[e] * f->val[h]; break; }
          }
        }
      }
      if (!(f->val[f->dpos[i]] > 0.0)) bad = 1;
    }
  }
  if (bad) {
    ilu_free(f);
    return ORC_BREAKDOWN;
  }
  return ORC_OK;
}

/* z = (LU)^-1 r box by box: forward substitution with the unit lower
 * factor, then back substitution with the upper factor. */
static void precond_ilu(const orc_ilu *f, const double *r, double *z) {
#pragma omp parallel
  {
    long cap = 0;
    double *y = NULL;
#pragma omp for schedule(dynamic, 16)
    for (long bx = 0; bx < f->nbox; bx++) {
      const long b0 = f->bstart[bx], b1 = f->bstart[bx + 1];
      if (b1 - b0 > cap) {
        free(y);
        cap = b1 - b0;
        y = malloc(sizeof(double) * cap);
      }
      /* L y = r:  y_i = r_i - sum_{k<i} l_ik y_k */
      for (long i = b0; i < b1; i++) {
        double s = r[f->perm[i]];
        for (long e = f->rowptr[i]; e < f->dpos[i]; e++) s -= f->val[e] * y[f->col[e] - b0];
        y[i - b0] = s;
      }
      /* U z = y:  z_i = (y_i - sum_{j>i} u_ij z_j) / u_ii, stored in y */
      for (long i = b1 - 1; i >= b0; i--) {
        double s = y[i - b0];
        for (long e = f->dpos[i] + 1; e < f->rowptr[i + 1]; e++) s -= f->val[e] * y[f->col[e] - b0];
        y[i - b0] = s / f->val[f->dpos[i]];
      }
      for (long i = b0; i < b1; i++) z[f->perm[i]] = y[i - b0];
    }
    free(y);
  }
}

static void precond_apply(const orc_op *op, const orc_ilu *ilu, const double *r, double *z) {
  if (g_precond == 4) {
    precond_ilu(ilu, r, z);
  } else if (g_precond == 0) {
    precond_jacobi(op, r, z);
  } else if (g_precond == 1) {
    precond_rline(op, r, z);
  } else if (g_precond == 2) {
    precond_philine(op, r, z);
  } else {
    /* both line directions: z = T_r^-1 r + T_phi^-1 r - D^-1 r */
    const long n = (long)op->nr * op->nt * op->np;
    double *t = malloc(sizeof(double) * n);
    double *d = malloc(sizeof(double) * n);
    precond_rline(op, r, z);
    precond_philine(op, r, t);
    precond_jacobi(op, r, d);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; c++) z[c] = z[c] + t[c] - d[c];
    free(t);
    free(d);
  }
}

/* ------------------------------------------------------ vector helpers */

static double dot(long n, const double *a, const double *b) {
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  double *part = calloc((size_t)nth, sizeof(double));
#pragma omp parallel num_threads(nth)
  {
    int t = 0, T = 1;
#ifdef _OPENMP
    t = omp_get_thread_num();
    T = omp_get_num_threads();
#endif
    long lo = n * t / T, hi = n * (t + 1) / T;
    double s = 0.0;
    for (long q = lo; q < hi; q++) s += a[q] * b[q];
    part[t] = s;
  }
  double s = 0.0;
  for (int t = 0; t < nth; t++) s += part[t];
  free(part);
  return s;
}

/* ----------------------------------------------------------- public API */

int orc_apply(int nr, int nt, int np, const double *rf, const double *tf, const double *x,
              double *y) {
  orc_op op;
  int st = op_build(&op, nr, nt, np, rf, tf);
  if (st) return st;
  op_apply(&op, x, y);
  op_free(&op);
  return ORC_OK;
}

/* z = M^-1 r with the preconditioner of orc_set_precond (exposed for the
 * tests). */
int orc_precond(int nr, int nt, int np, const double *rf, const double *tf, const double *r,
                double *z) {
  orc_op op;
  int st = op_build(&op, nr, nt, np, rf, tf);
  if (st) return st;
  orc_ilu ilu;
  memset(&ilu, 0, sizeof(ilu));
  if (g_precond == 4 && (st = ilu_build(&op, &ilu)) != ORC_OK) {
    op_free(&op);
    return st;
  }
  precond_apply(&op, &ilu, r, z);
  ilu_free(&ilu);
  op_free(&op);
  return ORC_OK;
}

/* Diagonal of L per (i, j) row; the same for every k. */
int orc_diag(int nr, int nt, int np, const double *rf, const double *tf, double *d) {
  orc_op op;
  int st = op_build(&op, nr, nt, np, rf, tf);
  if (st) return st;
  memcpy(d, op.diag, sizeof(double) * nr * nt);
  op_free(&op);
  return ORC_OK;
}

/* Face coefficient tables, exposed for the tests: cr [nr*nt], ct [nr*(nt-1)], cp [nr*nt]. */
int orc_coeffs(int nr, int nt, int np, const double *rf, const double *tf, double *cr, double *ct,
               double *cp) {
  orc_op op;
  int st = op_build(&op, nr, nt, np, rf, tf);
  if (st) return st;
  memcpy(cr, op.cr, sizeof(double) * nr * nt);
  if (nt > 1) memcpy(ct, op.ct, sizeof(double) * nr * (nt - 1));
  memcpy(cp, op.cp, sizeof(double) * nr * nt);
  op_free(&op);
  return ORC_OK;
}

/* Closed wall: Br minus its area-weighted mean over the inner face (the
 * discrete monopole), so that the right-hand side has zero net flux.  With
 * the source surface Br is copied unchanged. */
int orc_balance_br(int nr, int nt, int np, const double *rf, const double *tf, const double *br,
                   double *out) {
  orc_op op;
  int st = op_build(&op, nr, nt, np, rf, tf);
  if (st) return st;
  double mono = 0.0;
  if (g_outer_closed) {
    double fl = 0.0, ar = 0.0;
    for (int j = 0; j < nt; j++) {
      double area = rf[0] * rf[0] * sin(op.tc[j]) * op.dt[j] * op.dphi;
      for (int k = 0; k < np; k++) {
        fl += area * br[(long)j * np + k];
        ar += area;
      }
    }
    mono = fl / ar;
  }
  for (long e = 0; e < (long)nt * np; e++) out[e] = br[e] - mono;
  op_free(&op);
  return ORC_OK;
}

/* Right-hand side from the inner-boundary Br map (Eq. 2). */
int orc_rhs(int nr, int nt, int np, const double *rf, const double *tf, const double *br,
            double *b) {
  orc_op op;
  int st = op_build(&op, nr, nt, np, rf, tf);
  if (st) return st;
  long n = (long)nr * nt * np;
  memset(b, 0, sizeof(double) * n);
  /* closed wall: subtract the area-weighted mean of Br (zero net flux) */
  double mono = 0.0;
  if (g_outer_closed) {
    double fl = 0.0, ar = 0.0;
    for (int j = 0; j < nt; j++) {
      double area = rf[0] * rf[0] * sin(op.tc[j]) * op.dt[j] * op.dphi;
      for (int k = 0; k < np; k++) {
        fl += area * br[(long)j * np + k];
        ar += area;
      }
    }
    mono = fl / ar;
  }
  for (int j = 0; j < nt; j++) {
    double area = rf[0] * rf[0] * sin(op.tc[j]) * op.dt[j] * op.dphi;
    for (int k = 0; k < np; k++) b[(long)j * np + k] = -area * (br[(long)j * np + k] - mono);
  }
  op_free(&op);
  return ORC_OK;
}

/* Textbook preconditioned conjugate gradient (Saad, Iterative Methods,
 * Algorithm 9.1) with the preconditioner of orc_set_precond: point Jacobi
 * (diagonal scaling, PC1 of Sec. 2.3) by default, a line preconditioner, or
 * the subdomain ILU(0) (PC2 of Sec. 2.3, factored once per call).  x holds
 * the initial guess when x0_given != 0, else it is
 * zeroed.  Stops after iteration k when ||r_k||_2 / ||b||_2 <= tol.
 * relres (optional, length maxit+1) receives ||r_k||/||b|| for k = 0..iters.
 * Returns ORC_OK, ORC_NOT_CONVERGED (iters == maxit, x = last iterate) or
 * ORC_BREAKDOWN (p.Ap <= 0 or not finite). */
int orc_pcg(int nr, int nt, int np, const double *rf, const double *tf, const double *b,
            double tol, int maxit, int x0_given, double *x, int *iters, double *relres) {
  orc_op op;
  int st = op_build(&op, nr, nt, np, rf, tf);
  if (st) return st;
  const long n = (long)nr * nt * np;
  double *r = malloc(sizeof(double) * n);
  double *z = malloc(sizeof(double) * n);
  double *p = malloc(sizeof(double) * n);
  double *q = malloc(sizeof(double) * n);
  if (!r || !z || !p || !q) {
    free(r); free(z); free(p); free(q);
    op_free(&op);
    return ORC_BAD_ARG;
  }
  /* r_0 = b - L x_0 */
  if (x0_given) {
    op_apply(&op, x, q);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; c++) r[c] = b[c] - q[c];
  } else {
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; c++) { x[c] = 0.0; r[c] = b[c]; }
  }
  const double bnorm = sqrt(dot(n, b, b));
  /* PC2: the subdomain ILU(0) factors, once per solve */
  orc_ilu ilu;
  memset(&ilu, 0, sizeof(ilu));
  if (g_precond == 4 && (st = ilu_build(&op, &ilu)) != ORC_OK) {
    free(r); free(z); free(p); free(q);
    op_free(&op);
    return st;
  }
  /* z_0 = M^-1 r_0 */
  precond_apply(&op, &ilu, r, z);
  /* p_0 = z_0 */
#pragma omp parallel for schedule(static)
  for (long c = 0; c < n; c++) p[c] = z[c];
  double rho = dot(n, r, z);
  double rn = sqrt(dot(n, r, r));
  if (relres) relres[0] = (bnorm > 0) ? rn / bnorm : 0.0;
  int k = 0;
  int status = ORC_NOT_CONVERGED;
  if (bnorm == 0.0 || rn / bnorm <= tol) status = ORC_OK;
  while (status == ORC_NOT_CONVERGED && k < maxit) {
    k++;
    /* q = L p */
    op_apply(&op, p, q);
    /* sigma = p . q ; alpha = rho / sigma */
    double sigma = dot(n, p, q);
    if (!(sigma > 0.0) || !isfinite(sigma)) { status = ORC_BREAKDOWN; break; }
    double alpha = rho / sigma;
    /* x = x + alpha p */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; c++) x[c] = x[c] + alpha * p[c];
    /* r = r - alpha q */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; c++) r[c] = r[c] - alpha * q[c];
    /* convergence: ||r|| / ||b|| <= tol */
    rn = sqrt(dot(n, r, r));
    if (relres) relres[k] = rn / bnorm;
    if (rn / bnorm <= tol) { status = ORC_OK; break; }
    /* z = M^-1 r */
    precond_apply(&op, &ilu, r, z);
    /* beta = (r_new . z_new) / (r_old . z_old) */
    double rho_new = dot(n, r, z);
    double beta = rho_new / rho;
    rho = rho_new;
    /* p = z + beta p */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; c++) p[c] = z[c] + beta * p[c];
  }
  *iters = k;
  free(r); free(z); free(p); free(q);
  ilu_free(&ilu);
  op_free(&op);
  return status;
}

/* Subtracts the arithmetic mean over all n cells from x: the gauge of the
 * closed-wall problem, whose solution is defined up to a constant. */
void orc_remove_mean(long n, double *x) {
  double s = 0.0;
  for (long c = 0; c < n; c++) s += x[c];
  const double m = s / (double)n;
  for (long c = 0; c < n; c++) x[c] -= m;
}

/* Pole averages (Eq. 3): mean over phi of the first ring at each radius.
 * north[i] uses j = 0, south[i] uses j = nt-1. */
int orc_pole_avg(int nr, int nt, int np, const double *phi, double *north, double *south) {
  for (int i = 0; i < nr; i++) {
    double sn = 0.0, ss = 0.0;
    for (int k = 0; k < np; k++) {
      sn += phi[((long)i * nt + 0) * np + k];
      ss += phi[((long)i * nt + (nt - 1)) * np + k];
    }
    north[i] = sn / (double)np;
    south[i] = ss / (double)np;
  }
  return ORC_OK;
}

/* Field B = grad Phi on the staggered faces (Sec. 2.1: B = grad Phi).
 * Output B is three contiguous blocks:
 *   Br  [(nr+1) * nt * np]  on r faces  r_{i+1/2}, i = -1..nr-1 (face index 0..nr)
 *   Bth [nr * (nt+1) * np]  on th faces th_{j+1/2}, j = -1..nt-1 (face index 0..nt)
 *   Bph [nr * nt * np]      on phi faces between k and k+1 (wrapping)
 * Ghosts: inner Phi_g = Phi_0 - Br dr1 (so the inner face gets Br exactly;
 * for the closed wall pass the balanced Br of orc_balance_br, the one the
 * solve used); outer Phi_g = -Phi_last (Phi = 0 on the source surface) or
 * Phi_last (closed wall, Br = 0); across a pole
 * Phi_g = 2 avg - Phi_ring, so the pole face value is the ring's phi-average
 * (Eq. 3 with epsilon = half the first cell). */
int orc_field(int nr, int nt, int np, const double *rf, const double *tf, const double *phi,
              const double *br, double *B) {
  orc_op op;
  int st = op_build(&op, nr, nt, np, rf, tf);
  if (st) return st;
  double *north = malloc(sizeof(double) * nr), *south = malloc(sizeof(double) * nr);
  orc_pole_avg(nr, nt, np, phi, north, south);
  const long n = (long)nr * nt * np;
  double *Br = B, *Bt = B + (long)(nr + 1) * nt * np, *Bp = Bt + (long)nr * (nt + 1) * np;
  (void)n;
  /* Br on radial faces */
  for (int f = 0; f <= nr; f++) {
    for (int j = 0; j < nt; j++) {
      for (int k = 0; k < np; k++) {
        long o = ((long)f * nt + j) * np + k;
        if (f == 0) {
          /* inner ghost: (Phi_0 - (Phi_0 - Br dr1)) / dr1 = Br */
          Br[o] = br[(long)j * np + k];
        } else if (f == nr) {
          double pl = phi[((long)(nr - 1) * nt + j) * np + k];
          /* source surface: ghost -Phi; closed wall: ghost Phi (Br = 0) */
          double ghost = g_outer_closed ? pl : -pl;
          double spacing = 2.0 * (rf[nr] - op.rc[nr - 1]);
          Br[o] = (ghost - pl) / spacing;
        } else {
          double lo = phi[((long)(f - 1) * nt + j) * np + k];
          double hi = phi[((long)f * nt + j) * np + k];
          Br[o] = (hi - lo) / (op.rc[f] - op.rc[f - 1]);
        }
      }
    }
  }
  /* Btheta on theta faces */
  for (int i = 0; i < nr; i++) {
    for (int f = 0; f <= nt; f++) {
      for (int k = 0; k < np; k++) {
        long o = ((long)i * (nt + 1) + f) * np + k;
        double v;
        if (f == 0) {
          double p0 = phi[((long)i * nt + 0) * np + k];
          double ghost = 2.0 * north[i] - p0;
          double spacing = 2.0 * (op.tc[0] - tf[0]); /* mirror across theta = 0 */
          v = (p0 - ghost) / (op.rc[i] * spacing);
        } else if (f == nt) {
          double pl = phi[((long)i * nt + nt - 1) * np + k];
          double ghost = 2.0 * south[i] - pl;
          double spacing = 2.0 * (tf[nt] - op.tc[nt - 1]); /* mirror across theta = pi */
          v = (ghost - pl) / (op.rc[i] * spacing);
        } else {
          double lo = phi[((long)i * nt + f - 1) * np + k];
          double hi = phi[((long)i * nt + f) * np + k];
          v = (hi - lo) / (op.rc[i] * (op.tc[f] - op.tc[f - 1]));
        }
        Bt[o] = v;
      }
    }
  }
  /* Bphi on phi faces between k and k+1 (periodic) */
  for (int i = 0; i < nr; i++) {
    for (int j = 0; j < nt; j++) {
      for (int k = 0; k < np; k++) {
        long c = ((long)i * nt + j) * np;
        double lo = phi[c + k], hi = phi[c + (k + 1) % np];
        Bp[c + k] = (hi - lo) / (op.rc[i] * sin(op.tc[j]) * op.dphi);
      }
    }
  }
  free(north);
  free(south);
  op_free(&op);
  return ORC_OK;
}

/* Assembled CSR of L for small grids (row order = unknown order; columns
 * sorted within a row).  Arrays sized by the caller: rowptr[n+1],
 * col[7n], val[7n].  Returns nnz, or -1 on a bad argument. */
long orc_csr(int nr, int nt, int np, const double *rf, const double *tf, long *rowptr, long *col,
             double *val) {
  orc_op op;
  if (op_build(&op, nr, nt, np, rf, tf)) return -1;
  const long plane = (long)nt * np;
  long nnz = 0;
  rowptr[0] = 0;
  for (int i = 0; i < nr; i++) {
    for (int j = 0; j < nt; j++) {
      for (int k = 0; k < np; k++) {
        long c = ((long)i * nt + j) * np + k;
        /* gather (column, value) pairs for this row, then sort by column */
        long cols[8];
        double vals[8];
        int m = 0;
        cols[m] = c; vals[m] = op.diag[i * nt + j]; m++;
        if (i < nr - 1) { cols[m] = c + plane; vals[m] = -op.cr[i * nt + j]; m++; }
        if (i > 0) { cols[m] = c - plane; vals[m] = -op.cr[(i - 1) * nt + j]; m++; }
        if (j < nt - 1) { cols[m] = c + np; vals[m] = -op.ct[i * (nt - 1) + j]; m++; }
        if (j > 0) { cols[m] = c - np; vals[m] = -op.ct[i * (nt - 1) + j - 1]; m++; }
        long base = ((long)i * nt + j) * np;
        long kp = base + (k + 1) % np, km = base + (k + np - 1) % np;
        /* with np == 2 both phi faces couple to the same neighbour */
        if (kp == km) {
          cols[m] = kp; vals[m] = -2.0 * op.cp[i * nt + j]; m++;
        } else {
          cols[m] = kp; vals[m] = -op.cp[i * nt + j]; m++;
          cols[m] = km; vals[m] = -op.cp[i * nt + j]; m++;
        }
        /* insertion sort by column */
        for (int a = 1; a < m; a++) {
          long cc = cols[a]; double vv = vals[a]; int b = a - 1;
          while (b >= 0 && cols[b] > cc) { cols[b + 1] = cols[b]; vals[b + 1] = vals[b]; b--; }
          cols[b + 1] = cc; vals[b + 1] = vv;
        }
        for (int a = 0; a < m; a++) { col[nnz] = cols[a]; val[nnz] = vals[a]; nnz++; }
        rowptr[c + 1] = nnz;
      }
    }
  }
  op_free(&op);
  return nnz;
}
