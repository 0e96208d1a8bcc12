// Throughput probes for the plain arithmetic pipes (the roofline of the FP64
// and FP32 CUDA-core kernels).  Eight independent FMA chains per thread keep
// the pipe busy; the grid covers every SM several times over.
#include "internal.h"
#include "mbar.cuh"

namespace gcamb {

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T a, T b, int iters, T *out) {
  T c[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) c[u] = (T)(threadIdx.x + u);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] = fma(c[u], a, b);
  }
  T s = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += c[u];
  if (s == (T)-12345.678) out[0] = s;  // keeps the chains live; never true for these inputs
}

template <typename T>
static int probe_t(double *flops) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  T *out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "probe: cudaMalloc");
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 2048 : 65536;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_probe_kernel<T><<<blocks, threads>>>((T)0.999999, (T)1e-7, iters / 8, out);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    fma_probe_kernel<T><<<blocks, threads>>>((T)0.999999, (T)1e-7, iters, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "probe: kernel");
  *flops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3);
  return GCAMB_OK;
}

int run_probe_flops(int what, double *flops) {
  return what == 0 ? probe_t<double>(flops) : probe_t<float>(flops);
}

// One thread waits, with the kernels' bounded wait, on an mbarrier that no
// one arrives on: after the wait limit it writes GCAMB_ETIMEOUT to *err and
// the kernel ends.
__global__ void wait_selftest_kernel(int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(smem_u32(&bar), 0, nullptr, err);
  }
}

int run_wait_selftest(int *status, cudaStream_t st) {
  int *err = status ? status : device_error_flag();
  if (!err) return fail(GCAMB_ECUDA, "selftest_wait: error flag allocation");
  wait_selftest_kernel<<<1, 32, 0, st>>>(err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "selftest_wait: launch");
  return GCAMB_OK;
}

}  // namespace gcamb
