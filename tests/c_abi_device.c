/* Plain C99 client of the whole path through the C ABI, with CUDA runtime
 * allocations and no Python: Eqs. (1)-(2) on a small grid, once by the plain
 * FP64 kernels (gcamb_los_transfer + gcamb_cl) and once by the batched
 * tensor-core path in F16X3 (gcamb_los_cl), which must agree within 1e-5 on
 * every C_l.  Built and run by tests/test_gpu_c_client.py.  Prints
 * "ok <max rel diff>" and exits 0, or names the failed check and exits 1. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "gcamb.h"

#define NK 64
#define NTAU 152
#define LMIN 2
#define LMAX 300
#define NL (LMAX - LMIN + 1)
#define M 8

#define CHECK(c)                                                                     \
  do {                                                                               \
    if (!(c)) {                                                                      \
      printf("FAILED: %s (line %d): %s\n", #c, __LINE__, gcamb_last_error());        \
      return 1;                                                                      \
    }                                                                                \
  } while (0)

int main(void) {
  static double k[NK], tau[NTAU], S64[M * NK * NTAU], P[M * NK], C64[M * NL], C16[M * NL];
  static float S32[M * NK * NTAU];
  const double tau0 = 14000.0;
  gcamb_grid *g = NULL;
  double *dS64 = NULL, *dP = NULL, *dD = NULL, *dC = NULL;
  float *dS32 = NULL;
  void *ws = NULL;
  size_t wsb = 0;
  double worst = 0.0;
  int m, q, i;
  for (q = 0; q < NK; ++q) k[q] = 1e-4 * pow(0.3 / 1e-4, q / (double)(NK - 1));
  for (i = 0; i < NTAU; ++i) tau[i] = 200.0 + (tau0 - 200.0) * i / (NTAU - 1);
  /* a visibility-like peak times an oscillation in k, plus a late smooth term */
  for (m = 0; m < M; ++m)
    for (q = 0; q < NK; ++q) {
      P[m * NK + q] = 2.1e-9 * pow(k[q] / 0.05, -0.035 + 0.005 * m);
      for (i = 0; i < NTAU; ++i) {
        const double a = (tau[i] - 285.0 - 2.0 * m) / 20.0, b = (tau[i] - 11000.0) / 2000.0;
        const double s = exp(-0.5 * a * a) / (20.0 * sqrt(2.0 * M_PI)) * cos(k[q] * 145.0 + 0.3 * m) *
                             exp(-pow(k[q] / 0.15, 2.0)) +
                         0.01 * m * exp(-0.5 * b * b) * exp(-k[q] / 0.01);
        S32[(m * NK + q) * NTAU + i] = (float)s;
        S64[(m * NK + q) * NTAU + i] = (double)(float)s; /* both paths read the same values */
      }
    }
  CHECK(gcamb_grid_create(k, NK, tau, NTAU, tau0, LMIN, LMAX, 1e-30, &g) == GCAMB_OK);
  CHECK(cudaMalloc((void **)&dS64, sizeof S64) == cudaSuccess);
  CHECK(cudaMalloc((void **)&dS32, sizeof S32) == cudaSuccess);
  CHECK(cudaMalloc((void **)&dP, sizeof P) == cudaSuccess);
  CHECK(cudaMalloc((void **)&dD, sizeof(double) * M * NK * NL) == cudaSuccess);
  CHECK(cudaMalloc((void **)&dC, sizeof C64) == cudaSuccess);
  CHECK(cudaMemcpy(dS64, S64, sizeof S64, cudaMemcpyHostToDevice) == cudaSuccess);
  CHECK(cudaMemcpy(dS32, S32, sizeof S32, cudaMemcpyHostToDevice) == cudaSuccess);
  CHECK(cudaMemcpy(dP, P, sizeof P, cudaMemcpyHostToDevice) == cudaSuccess);
  /* plain FP64 */
  CHECK(gcamb_bessel_table(g, GCAMB_PLAIN64, NULL) == GCAMB_OK);
  CHECK(gcamb_los_transfer(g, dS64, M, GCAMB_PLAIN64, dD, NULL) == GCAMB_OK);
  CHECK(gcamb_cl(g, dD, GCAMB_F64, dP, M, dC, NULL) == GCAMB_OK);
  CHECK(gcamb_sync(NULL) == GCAMB_OK);
  CHECK(cudaMemcpy(C64, dC, sizeof C64, cudaMemcpyDeviceToHost) == cudaSuccess);
  /* batched F16X3 on the tensor cores */
  CHECK(gcamb_bessel_table(g, GCAMB_F16X3, NULL) == GCAMB_OK);
  CHECK(gcamb_los_cl_workspace(g, M, GCAMB_F16X3, &wsb) == GCAMB_OK && wsb > 0);
  CHECK(cudaMalloc(&ws, wsb) == cudaSuccess);
  CHECK(gcamb_los_cl(g, dS32, dP, M, GCAMB_F16X3, dC, ws, wsb, NULL) == GCAMB_OK);
  CHECK(gcamb_sync(NULL) == GCAMB_OK);
  CHECK(cudaMemcpy(C16, dC, sizeof C16, cudaMemcpyDeviceToHost) == cudaSuccess);
  for (i = 0; i < M * NL; ++i) {
    CHECK(C64[i] > 0.0);
    const double r = fabs(C16[i] / C64[i] - 1.0);
    if (r > worst) worst = r;
  }
  CHECK(worst <= 1e-5);
  cudaFree(ws);
  cudaFree(dC);
  cudaFree(dD);
  cudaFree(dP);
  cudaFree(dS32);
  cudaFree(dS64);
  CHECK(gcamb_grid_destroy(g) == GCAMB_OK);
  printf("ok %.3e\n", worst);
  return 0;
}
