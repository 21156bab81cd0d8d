/* Plain C99 user of include/lbm.h: compiles with -Wall -Wextra -Werror
 * -pedantic against the header alone and, linked against liblbm.so, runs
 * the entry points that need no GPU (version, defaults, workspace sizing,
 * stencil export, argument validation).  Prints "ok" and exits 0. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "lbm.h"

static int fails = 0;
#define CHECK(c)                                                   \
  do {                                                             \
    if (!(c)) {                                                    \
      fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
      ++fails;                                                     \
    }                                                              \
  } while (0)

int main(void) {
  lbm_params p;
  int32_t c[3 * 27];
  double w[27], sum = 0.0;
  lbm_domain* dom = NULL;
  size_t a, b;
  int i;

  CHECK(strstr(lbm_version(), "sm_103a") != NULL);
  lbm_default_params(&p);
  CHECK(p.nu_L > 0.0 && p.omega_high == 1.0 && p.T_bottom_waves == 0 && p.T_bottom_amp == 0.0);

  a = lbm_workspace_bytes(64, 64, 64, LBM_FP32, LBM_TH_D3Q7, 15);
  b = lbm_workspace_bytes(64, 64, 64, LBM_FP64, LBM_TH_D3Q7, 15);
  CHECK(a > 0 && b > a);
  CHECK(lbm_workspace_bytes(0, 64, 64, LBM_FP32, LBM_TH_D3Q7, 15) == 0);
  CHECK(lbm_workspace_bytes(64, 64, 64, LBM_FP32, LBM_TH_D3Q7, 19) == 0);

  CHECK(lbm_stencil(27, c, w) == LBM_OK);
  for (i = 0; i < 27; ++i) sum += w[i];
  CHECK(fabs(sum - 1.0) < 1e-15);
  CHECK(c[0] == 0 && c[1] == 0 && c[2] == 0);
  CHECK(lbm_stencil(9, c, w) == LBM_ERR_ARG);

  /* rejected before any CUDA call */
  CHECK(lbm_create_domain(0, 8, 8, LBM_FP32, LBM_TH_D3Q7, 15, NULL, NULL, 0, &dom) == LBM_ERR_ARG);
  CHECK(dom == NULL);
  CHECK(lbm_create_domain(8, 8, 8, LBM_FP32, LBM_TH_D3Q7, 21, NULL, NULL, 0, &dom) == LBM_ERR_ARG);
  CHECK(lbm_step(NULL, 1) == LBM_ERR_ARG);
  CHECK(lbm_set_heater_field(NULL, NULL, 0) == LBM_ERR_ARG);
  CHECK(strlen(lbm_last_error()) > 0);

  if (fails) return 1;
  printf("ok\n");
  return 0;
}
