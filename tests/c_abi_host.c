/* Plain C99 client of the C ABI (include/gcamb.h), built and run by
 * tests/test_abi_cpu.py: the header compiles as C with -pedantic, and the
 * host-side entry points (no GPU needed) behave as documented.  Prints one
 * "ok" line and exits 0, or names the failed check and exits 1. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "gcamb.h"

#define CHECK(c)                                              \
  do {                                                        \
    if (!(c)) {                                               \
      printf("FAILED: %s (line %d)\n", #c, __LINE__);         \
      return 1;                                               \
    }                                                         \
  } while (0)

int main(void) {
  double k[6], tau[9], wt[9], wk[6];
  gcamb_grid *g = NULL;
  int64_t info[GCAMB_INFO_N];
  int32_t ext[6 * 1];
  double sum = 0.0;
  int i, comp = -1;
  for (i = 0; i < 6; ++i) k[i] = 0.01 * (i + 1);
  for (i = 0; i < 9; ++i) tau[i] = 200.0 + 100.0 * i;

  CHECK(strstr(gcamb_version(), "sm_103a") != NULL);
  /* decreasing k is refused, with its reason */
  {
    double kd[2] = {0.2, 0.1};
    CHECK(gcamb_grid_create(kd, 2, tau, 9, 1400.0, 2, 10, 1e-30, &g) == GCAMB_EINVAL);
    CHECK(strstr(gcamb_last_error(), "increasing") != NULL);
  }
  CHECK(gcamb_grid_create(k, 6, tau, 9, 1400.0, 2, 40, 1e-30, &g) == GCAMB_OK && g != NULL);
  CHECK(gcamb_grid_info(g, info) == GCAMB_OK);
  CHECK(info[0] == 6 && info[1] == 9 && info[2] == 39 && info[3] == 1 && info[6] == 2 && info[7] == 40);
  CHECK(gcamb_grid_extents(g, ext) == GCAMB_OK);
  for (i = 0; i < 6; ++i) CHECK(ext[i] >= 0 && ext[i] <= 9);
  /* trapezoid weights in tau sum to the tau range */
  CHECK(gcamb_grid_weights(g, wt, wk) == GCAMB_OK);
  for (i = 0; i < 9; ++i) sum += wt[i];
  CHECK(fabs(sum - 800.0) < 1e-12);
  /* a table that was never built */
  CHECK(gcamb_table_compressed(g, GCAMB_F16X3, &comp) == GCAMB_ESTATE);
  CHECK(gcamb_grid_destroy(g) == GCAMB_OK);
  CHECK(gcamb_grid_destroy(NULL) == GCAMB_OK);
  printf("ok\n");
  return 0;
}
