/* Plain C99 user of include/lbm.h on a GPU: creates a domain (library-owned
 * workspace, legacy default stream), sets the parameters, places one droplet,
 * runs 50 steps in FP32 and in FP64 on the same lattice and reads the
 * diagnostics and the phi field back to host memory.  Checks: the status of
 * every call, the time level, phi mass conserved (1e-12 in FP64, 1e-4 in
 * FP32 shifted storage: its rounding, not a parity bound), FP32 centroid within
 * 1e-3 lu of FP64, the host phi field summing to
 * the diagnostics' mass.  Prints "ok" and exits 0. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lbm.h"

static int fails = 0;
#define CHECK(c)                                                           \
  do {                                                                     \
    if (!(c)) {                                                            \
      fprintf(stderr, "check failed: %s (line %d): %s\n", #c, __LINE__,     \
              lbm_last_error());                                           \
      ++fails;                                                             \
    }                                                                      \
  } while (0)

static int run(lbm_precision prec, double centroid[3], double* mass_drift) {
  const int nx = 80, ny = 24, nz = 16, steps = 50;
  lbm_domain* dom = NULL;
  lbm_params p;
  lbm_droplet d;
  lbm_diag g0, g1;
  double* phi;
  double sum = 0.0;
  long i;
  if (lbm_create_domain(nx, ny, nz, prec, LBM_TH_D3Q7, 15, NULL, NULL, 0, &dom) != LBM_OK) {
    fprintf(stderr, "create failed: %s\n", lbm_last_error());
    return 1;
  }
  lbm_default_params(&p);
  p.sigma_ref = 5e-3;
  p.sigma_T = -5e-4;
  p.grad_T[0] = 1e-3;
  p.grad_T_origin[0] = 40.0;
  p.grad_T_origin[1] = 12.0;
  p.grad_T_origin[2] = 8.0;
  CHECK(lbm_set_params(dom, &p) == LBM_OK);
  d.cx = 40.3; d.cy = 12.2; d.cz = 8.1; d.R = 5.0; d.ux = 1e-3; d.uy = 0.0; d.uz = 0.0;
  CHECK(lbm_init_droplets(dom, 1, &d) == LBM_OK);
  CHECK(lbm_get_diagnostics(dom, &g0) == LBM_OK);
  CHECK(lbm_step(dom, steps) == LBM_OK);
  CHECK(lbm_get_diagnostics(dom, &g1) == LBM_OK);
  CHECK(g1.level == steps && !g1.nonfinite);
  phi = (double*)malloc(sizeof(double) * (size_t)nx * ny * nz);
  CHECK(phi != NULL);
  if (phi) {
    CHECK(lbm_get_fields(dom, LBM_FIELD_PHI, phi, 0, 0) == LBM_OK);
    for (i = 0; i < (long)nx * ny * nz; ++i) sum += phi[i];
    CHECK(fabs(sum - g1.mass) <= 1e-9 * g1.mass);
    free(phi);
  }
  centroid[0] = g1.mx / g1.mass;
  centroid[1] = g1.my / g1.mass;
  centroid[2] = g1.mz / g1.mass;
  *mass_drift = fabs(g1.mass - g0.mass) / g0.mass;
  CHECK(lbm_destroy_domain(dom) == LBM_OK);
  return 0;
}

int main(void) {
  double c64[3], c32[3], m64, m32;
  int k;
  if (run(LBM_FP64, c64, &m64) || run(LBM_FP32, c32, &m32)) return 1;
  CHECK(m64 <= 1e-12);
  CHECK(m32 <= 1e-4);
  for (k = 0; k < 3; ++k) CHECK(fabs(c64[k] - c32[k]) <= 1e-3);
  CHECK(c64[0] > 40.3);   /* the droplet moved along +x */
  if (fails) return 1;
  printf("ok\n");
  return 0;
}
