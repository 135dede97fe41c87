/*
 * Plain-C use of the C ABI in include/pittpack_gb.h (no CUDA headers or runtime calls needed:
 * the host-buffer entry point copies to and from the device itself).
 *
 * Solves a problem whose discrete solution is known exactly: on the cell-centred grid the
 * products cos(pi a x) (Neumann faces), sin(pi b y) (Dirichlet faces), cos(pi c z) (Neumann) are
 * eigenvectors of the 7-point operator with eigenvalue sum_axis (2 cos(pi k / n) - 2) / h^2, so
 * the source f = lambda u* must give back u* to rounding.
 *
 * Exit status: 0 solved and checked; 3 no usable GPU (plan creation could not reach a device);
 * 1 a check failed.  The argument-validation calls at the start need no GPU.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "pittpack_gb.h"

static int fail(const char* what) {
  printf("FAILED: %s (%s)\n", what, pp_last_error_string());
  return 1;
}

int main(void) {
  const double PI = 3.14159265358979323846;
  printf("%s\n", pp_version());

  /* validation: no device work */
  pp_plan* plan = NULL;
  const pp_bc unpaired[6] = {PP_BC_PERIODIC, PP_BC_NEUMANN, PP_BC_NEUMANN, PP_BC_NEUMANN,
                             PP_BC_DIRICHLET, PP_BC_DIRICHLET};
  if (pp_plan_create(&plan, 8, 8, 8, unpaired, 1.0, 1.0, 1.0, PP_F64, NULL) != PP_ERR_BC_PAIRING || plan)
    return fail("periodic face paired with a Neumann face must be rejected");
  const pp_bc bc[6] = {PP_BC_NEUMANN, PP_BC_NEUMANN, PP_BC_DIRICHLET, PP_BC_DIRICHLET,
                       PP_BC_NEUMANN, PP_BC_NEUMANN};
  if (pp_plan_create(&plan, 22, 8, 8, bc, 1.0, 1.0, 1.0, PP_F64, NULL) != PP_ERR_UNSUPPORTED_SIZE || plan)
    return fail("nx = 22 (prime factor 11) must be rejected");
  if (pp_solve(NULL, NULL, NULL, NULL) != PP_ERR_INVALID_ARG) return fail("NULL plan must be rejected");

  const int nx = 24, ny = 16, nz = 12;
  const double dx = 1.0 / nx, dy = 1.0 / ny, dz = 1.0 / nz;
  pp_status s = pp_plan_create(&plan, nx, ny, nz, bc, dx, dy, dz, PP_F64, NULL);
  if (s == PP_ERR_CUDA || s == PP_ERR_OUT_OF_MEMORY) {
    printf("no usable GPU: %s\n", pp_last_error_string());
    return 3;
  }
  if (s != PP_OK || !plan) return fail("plan creation");

  const int a = 3, b = 2, c = 1; /* mode numbers per axis */
  const double lam = (2.0 * cos(PI * a / nx) - 2.0) / (dx * dx) + (2.0 * cos(PI * b / ny) - 2.0) / (dy * dy) +
                     (2.0 * cos(PI * c / nz) - 2.0) / (dz * dz);
  const size_t n = (size_t)nx * ny * nz;
  double* f = (double*)malloc(n * sizeof(double));
  double* u = (double*)malloc(n * sizeof(double));
  double* us = (double*)malloc(n * sizeof(double));
  if (!f || !u || !us) return fail("host allocation");
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        const size_t p = ((size_t)k * ny + j) * nx + i;
        us[p] = cos(PI * a * (i + 0.5) * dx) * sin(PI * b * (j + 0.5) * dy) * cos(PI * c * (k + 0.5) * dz);
        f[p] = lam * us[p];
      }
  if (pp_solve_host(plan, f, u, NULL) != PP_OK) return fail("pp_solve_host");
  if (pp_plan_status(plan) != PP_OK) return fail("device status");
  double err = 0.0, mag = 0.0;
  for (size_t p = 0; p < n; p++) {
    err = fmax(err, fabs(u[p] - us[p]));
    mag = fmax(mag, fabs(us[p]));
  }
  printf("max |u - u*| / max |u*| = %.3e\n", err / mag);
  if (!(err <= 1e-12 * mag)) return fail("solution does not match the exact discrete eigenfunction");
  if (pp_plan_destroy(plan) != PP_OK) return fail("destroy");
  free(f);
  free(u);
  free(us);
  printf("ok\n");
  return 0;
}
