// Source interpolation onto the transfer k grid (the step that prepares the
// sources before the projection, Sec. 3.3): the natural cubic spline in k of
// every (source, tau) column.  On nodes k_0 < ... < k_(n-1), h_j = k_(j+1) - k_j,
// the second derivatives solve the tridiagonal system
//   h_(j-1) M_(j-1) + 2 (h_(j-1) + h_j) M_j + h_j M_(j+1)
//       = 6 [(y_(j+1) - y_j)/h_j - (y_j - y_(j-1))/h_(j-1)],   0 < j < n-1,
// with M_0 = M_(n-1) = 0; on [k_j, k_(j+1)], t = (k - k_j)/h_j,
//   y = (1-t) y_j + t y_(j+1) + h_j^2/6 [((1-t)^3 - (1-t)) M_j + (t^3 - t) M_(j+1)].
// The elimination coefficients depend on the k nodes only and are formed on
// the host; one thread per (source, tau) column runs the forward sweep and
// the back substitution in FP64 (reads along k are coalesced across tau),
// then one thread per output element evaluates the spline.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace gcamb {

namespace {

// Per column: d'_j = (r_j - a_j d'_(j-1)) * inv_j, M_j = d'_j - c'_j M_(j+1).
template <typename T>
__global__ void __launch_bounds__(256) spline_solve_kernel(const T *__restrict__ y, const double *__restrict__ h,
                                                           const double *__restrict__ cp,
                                                           const double *__restrict__ inv, int n, int ntau, int M,
                                                           double *__restrict__ Md) {
  const size_t col = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // m * ntau + tau
  if (col >= (size_t)M * ntau) return;
  const size_t m = col / ntau, t = col - m * ntau;
  const T *yc = y + m * (size_t)n * ntau + t;
  double *mc = Md + m * (size_t)n * ntau + t;
  mc[0] = 0.0;
  mc[(size_t)(n - 1) * ntau] = 0.0;
  if (n < 3) return;
  double y0 = (double)yc[0], y1 = (double)yc[ntau];
  double dprev = 0.0;
  for (int j = 1; j < n - 1; ++j) {
    const double y2 = (double)yc[(size_t)(j + 1) * ntau];
    const double r = 6.0 * ((y2 - y1) / h[j] - (y1 - y0) / h[j - 1]);
    const double d = (r - (j > 1 ? h[j - 1] * dprev : 0.0)) * inv[j];
    mc[(size_t)j * ntau] = d;
    dprev = d;
    y0 = y1;
    y1 = y2;
  }
  double next = 0.0;  // M_(n-1)
  for (int j = n - 2; j >= 1; --j) {
    const double v = mc[(size_t)j * ntau] - cp[j] * next;
    mc[(size_t)j * ntau] = v;
    next = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) spline_eval_kernel(const T *__restrict__ y, const double *__restrict__ Md,
                                                          const int *__restrict__ jq, const double *__restrict__ tq,
                                                          const double *__restrict__ hq, int n, int nq, int ntau,
                                                          int M, T *__restrict__ out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (m * nq + q) * ntau + tau
  if (e >= (size_t)M * nq * ntau) return;
  const size_t t = e % ntau, mq = e / ntau;
  const size_t q = mq % nq, m = mq / nq;
  const int j = jq[q];
  const double s = tq[q], h = hq[q], u = 1.0 - s;
  const size_t i0 = (m * (size_t)n + j) * ntau + t, i1 = i0 + ntau;
  const double v = u * (double)y[i0] + s * (double)y[i1] +
                   h * h / 6.0 * ((u * u * u - u) * Md[i0] + (s * s * s - s) * Md[i1]);
  out[e] = (T)v;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Workspace: [h, c', 1/den] (3 nk_in doubles) | [t, h] of each output node
// (2 nk_out doubles) | interval of each output node (nk_out ints) |
// second derivatives [M][nk_in][ntau] (doubles), each region 256-byte aligned.
size_t interp_workspace_bytes(int M, int nk_in, int ntau, int nk_out) {
  return a256((size_t)nk_in * 3 * sizeof(double)) + a256((size_t)nk_out * 2 * sizeof(double)) +
         a256((size_t)nk_out * sizeof(int)) + a256((size_t)M * nk_in * ntau * sizeof(double));
}

int launch_interp_sources(const double *k_in, int nk_in, const void *S_in, int M, int ntau, int dtype,
                          const gcamb_grid *g, void *S_out, void *ws, size_t ws_bytes, cudaStream_t st) {
  const int n = nk_in, nq = g->nk;
  if (ws_bytes < interp_workspace_bytes(M, n, ntau, nq)) return fail(GCAMB_EINVAL, "interp_sources: workspace too small");
  // elimination coefficients (nodes only) and each output node's interval
  std::vector<double> host(3 * (size_t)n, 0.0), qd(2 * (size_t)nq);
  std::vector<int> qj(nq);
  double *h = host.data(), *cp = h + n, *inv = cp + n;
  for (int j = 0; j + 1 < n; ++j) h[j] = k_in[j + 1] - k_in[j];
  for (int j = 1; j < n - 1; ++j) {
    const double b = 2.0 * (h[j - 1] + h[j]);
    const double den = b - (j > 1 ? h[j - 1] * cp[j - 1] : 0.0);
    inv[j] = 1.0 / den;
    cp[j] = (j < n - 2 ? h[j] : 0.0) * inv[j];
  }
  for (int q = 0; q < nq; ++q) {
    const double k = g->k[q];
    int j = (int)(std::upper_bound(k_in, k_in + n, k) - k_in) - 1;
    j = j < 0 ? 0 : (j > n - 2 ? n - 2 : j);
    qj[q] = j;
    qd[q] = (k - k_in[j]) / h[j];
    qd[nq + q] = h[j];
  }
  char *w = static_cast<char *>(ws);
  const size_t o1 = a256((size_t)n * 3 * sizeof(double));
  const size_t o2 = o1 + a256((size_t)nq * 2 * sizeof(double));
  const size_t o3 = o2 + a256((size_t)nq * sizeof(int));
  double *d_h = reinterpret_cast<double *>(w);
  double *d_t = reinterpret_cast<double *>(w + o1);
  double *d_hq = d_t + nq;
  int *d_j = reinterpret_cast<int *>(w + o2);
  double *d_M = reinterpret_cast<double *>(w + o3);
  // pageable copies return once the host data is staged
  cudaError_t e = cudaMemcpyAsync(d_h, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_j, qj.data(), qj.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_t, qd.data(), qd.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "interp_sources: coefficient upload");
  const size_t cols = (size_t)M * ntau, outs = (size_t)M * nq * ntau;
  ProfScope prof(GCAMB_K_INTERP, st);
  if (dtype == GCAMB_F64) {
    spline_solve_kernel<double><<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(
        static_cast<const double *>(S_in), d_h, d_h + n, d_h + 2 * n, n, ntau, M, d_M);
    spline_eval_kernel<double><<<(unsigned)((outs + 255) / 256), 256, 0, st>>>(
        static_cast<const double *>(S_in), d_M, d_j, d_t, d_hq, n, nq, ntau, M, static_cast<double *>(S_out));
  } else {
    spline_solve_kernel<float><<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(
        static_cast<const float *>(S_in), d_h, d_h + n, d_h + 2 * n, n, ntau, M, d_M);
    spline_eval_kernel<float><<<(unsigned)((outs + 255) / 256), 256, 0, st>>>(
        static_cast<const float *>(S_in), d_M, d_j, d_t, d_hq, n, nq, ntau, M, static_cast<float *>(S_out));
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "interp_sources: launch");
  return GCAMB_OK;
}

}  // namespace gcamb

using namespace gcamb;

extern "C" {

int gcamb_interp_sources_workspace(const gcamb_grid *g, int M, int nk_in, size_t *bytes) {
  if (!g || !bytes) return fail(GCAMB_EINVAL, "interp_sources_workspace: NULL argument");
  if (M < 0 || nk_in < 2) return fail(GCAMB_EINVAL, "interp_sources_workspace: need M >= 0 and nk_in >= 2");
  *bytes = interp_workspace_bytes(M, nk_in, g->ntau, g->nk);
  return GCAMB_OK;
}

int gcamb_interp_sources(const gcamb_grid *g, const double *k_in, int nk_in, const void *S_in, int M, int dtype,
                         void *S_out, void *ws, size_t ws_bytes, void *stream) {
  if (!g) return fail(GCAMB_EINVAL, "interp_sources: NULL grid");
  if (dtype != GCAMB_F64 && dtype != GCAMB_F32) return fail(GCAMB_EINVAL, "interp_sources: dtype must be F64 or F32");
  if (M < 0 || nk_in < 2) return fail(GCAMB_EINVAL, "interp_sources: need M >= 0 and nk_in >= 2");
  if (!k_in) return fail(GCAMB_EINVAL, "interp_sources: NULL k_in");
  for (int j = 0; j < nk_in; ++j) {
    if (!std::isfinite(k_in[j])) return fail(GCAMB_EINVAL, "interp_sources: k_in not finite");
    if (j && !(k_in[j] > k_in[j - 1])) return fail(GCAMB_EINVAL, "interp_sources: k_in must be strictly increasing");
  }
  if (g->k.front() < k_in[0] || g->k.back() > k_in[nk_in - 1])
    return fail(GCAMB_EINVAL, "interp_sources: the grid's k range must lie inside [k_in[0], k_in[nk_in-1]]");
  if (M == 0) return GCAMB_OK;
  if (!S_in || !S_out || !ws) return fail(GCAMB_EINVAL, "interp_sources: NULL pointer");
  return launch_interp_sources(k_in, nk_in, S_in, M, g->ntau, dtype, g, S_out, ws, ws_bytes, (cudaStream_t)stream);
}

}  // extern "C"
