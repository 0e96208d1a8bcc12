// gcamb_los_cl_noalloc: the batched tensor-core C_l with every scratch byte in
// one fixed, statically allocated device buffer.
//
// Some callers may not allocate device memory at all: a likelihood callback
// that runs inside a sampler or host framework that owns the device's memory
// budget, a process that pre-reserves its memory and forbids later
// allocations, or code that cannot afford cudaMalloc's implicit device-wide
// synchronisation.  gcamb_los_cl needs a workspace they would have to
// allocate; this entry point uses the buffer below instead.
//
// The buffer is a file-scope __device__ array of kFixedScratchBytes (64 MiB).
// Every device that loads this module holds it until the process exits.  In
// host code the array's name is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress, on the current device, at
// every call (a lookup costs no device work, and a cached address would go
// stale if the context were torn down and the module loaded again).
#include <string>

#include "internal.h"

namespace gcamb {
namespace {

constexpr size_t kFixedScratchBytes = size_t(64) << 20;

__device__ __align__(256) unsigned char g_fixed_scratch[kFixedScratchBytes];

int fixed_scratch(char **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_fixed_scratch);
  if (e != cudaSuccess || !p) return cuda_fail(e, "los_cl_noalloc: cudaGetSymbolAddress");
  *out = static_cast<char *>(p);
  return GCAMB_OK;
}

}  // namespace
}  // namespace gcamb

using namespace gcamb;

extern "C" int gcamb_los_cl_noalloc(const gcamb_grid *g, const float *S, const double *Pk, int M, int mode,
                                    double *Cl, int *status, void *stream) {
  if (!g) return fail(GCAMB_EINVAL, "los_cl_noalloc: NULL grid");
  if (mode != GCAMB_BF16X3 && mode != GCAMB_TF32X3 && mode != GCAMB_F16X3)
    return fail(GCAMB_EINVAL, "los_cl_noalloc: mode must be GCAMB_BF16X3, GCAMB_F16X3 or GCAMB_TF32X3");
  if (M < 0) return fail(GCAMB_EINVAL, "los_cl_noalloc: M < 0");
  if (M == 0) return GCAMB_OK;
  if (!S || !Pk || !Cl) return fail(GCAMB_EINVAL, "los_cl_noalloc: NULL pointer");
  if (!g->tab[mode].built || !g->d_wk)
    return fail(GCAMB_ESTATE, "los_cl_noalloc: build the table for this mode first (gcamb_bessel_table)");
  int dev = 0, maj = 0, mnr = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev);
  if (maj != 10 || mnr != 3) return fail(GCAMB_EUNSUPPORTED, "los_cl_noalloc: needs an sm_103 device");
  // The work list is uploaded from host memory that lives only for this
  // call, which a captured copy would read again at every replay: refuse
  // to run inside a stream capture.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing((cudaStream_t)stream, &cs);
  if (ce != cudaSuccess) return cuda_fail(ce, "los_cl_noalloc: cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone)
    return fail(GCAMB_EUNSUPPORTED, "los_cl_noalloc: not available inside a stream capture");
  char *scratch = nullptr;
  int rc = fixed_scratch(&scratch);
  if (rc) return rc;
  return launch_los_cl_fixed(g, S, Pk, M, mode, Cl, scratch, kFixedScratchBytes, status, (cudaStream_t)stream);
}
