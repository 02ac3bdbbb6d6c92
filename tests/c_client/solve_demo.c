/* Plain-C client of libpot3d (include/pot3d.h only; no Python, no torch):
 * builds a plan, solves with host arrays, evaluates the field and the FP64
 * residual, and exits 0 when the solve converged within tol.
 * Usage: solve_demo [nr nt np] */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "pot3d.h"

int main(int argc, char **argv) {
  int nr = 12, nt = 17, np = 37;
  if (argc == 4) {
    nr = atoi(argv[1]);
    nt = atoi(argv[2]);
    np = atoi(argv[3]);
  }
  const double tol = 1e-10;
  pot3d_grid_t grid = {nr, nt, np, 1.0, 2.5, 1.05, NULL, NULL, POT3D_PREC_FP64};
  pot3d_bc_t bc = {POT3D_OUTER_SOURCE_SURFACE, POT3D_POLE_AVERAGE};
  pot3d_plan_t *plan = pot3d_plan(&grid, &bc);
  if (!plan) {
    fprintf(stderr, "pot3d_plan: %s\n", pot3d_strerror(pot3d_last_error()));
    return 2;
  }
  /* a tilted dipole on cell centres: Br = cos(theta) + 0.3 sin(theta) cos(phi) */
  const double pi = 3.14159265358979323846;
  double *br = malloc(sizeof(double) * nt * np);
  double *phi = calloc((size_t)nr * nt * np, sizeof(double));
  for (int j = 0; j < nt; j++)
    for (int k = 0; k < np; k++) {
      const double t = (j + 0.5) * pi / nt, p = (k + 0.5) * 2.0 * pi / np;
      br[j * np + k] = cos(t) + 0.3 * sin(t) * cos(p);
    }
  int iters = 0;
  int rc = pot3d_solve(plan, br, tol, phi, &iters);
  double relres = -1.0;
  if (rc == POT3D_OK) rc = pot3d_residual(plan, br, phi, &relres);
  pot3d_info_t info;
  pot3d_get_info(plan, &info);
  size_t nb = (size_t)(nr + 1) * nt * np + (size_t)nr * (nt + 1) * np + (size_t)nr * nt * np;
  double *B = malloc(sizeof(double) * nb);
  if (rc == POT3D_OK) rc = pot3d_field(plan, phi, br, B);
  printf("status %d (%s) iters %d relres %.3e n %lld B[0] %.6f\n", rc, pot3d_strerror(rc), iters,
         relres, info.n, rc == POT3D_OK ? B[0] : 0.0);
  /* the inner-face field is the input Br itself */
  const int inner_ok = rc == POT3D_OK && fabs(B[0] - br[0]) <= 1e-12 * fabs(br[0]);
  pot3d_destroy(plan);
  free(br);
  free(phi);
  free(B);
  return (rc == POT3D_OK && relres >= 0.0 && relres <= 1.001 * tol && inner_ok) ? 0 : 1;
}
