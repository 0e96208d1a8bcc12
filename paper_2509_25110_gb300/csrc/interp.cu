// Source interpolation onto the transfer k grid (the step that prepares the
// sources before the projection, Sec. 3.3): the natural cubic spline in k of
// every (source, tau) column.  On nodes k_0 < ... < k_(n-1), h_j = k_(j+1) - k_j,
// the second derivatives solve the tridiagonal system
//   h_(j-1) M_(j-1) + 2 (h_(j-1) + h_j) M_j + h_j M_(j+1)
//       = 6 [(y_(j+1) - y_j)/h_j - (y_j - y_(j-1))/h_(j-1)],   0 < j < n-1,
// with M_0 = M_(n-1) = 0; on [k_j, k_(j+1)], t = (k - k_j)/h_j,
//   y = (1-t) y_j + t y_(j+1) + h_j^2/6 [((1-t)^3 - (1-t)) M_j + (t^3 - t) M_(j+1)]
// (the cubic factors are evaluated in their factored forms, which do not
// cancel next to a node).
// The elimination coefficients and 1/h depend on the k nodes only and are
// formed on the host; one thread per (source, tau) column runs the forward
// sweep and the back substitution (reads along k are coalesced across tau),
// then one thread per output element evaluates the spline.  The arithmetic
// is that of the sources: FP64 for FP64 sources, FP32 for FP32 sources (the
// GPU's FP64 rate would make the FP32 case ALU-bound).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace gcamb {

namespace {

// Node coefficients of one precision: h, 1/h, c', 1/den (each [n]).
template <typename A>
struct NodeCoef {
  const A *h, *ih, *cp, *inv;
};

// Per column: d'_j = (r_j - h_(j-1) d'_(j-1)) / den_j, M_j = d'_j - c'_j M_(j+1).
template <typename T, typename A>
__global__ void __launch_bounds__(256) spline_solve_kernel(const T *__restrict__ y, NodeCoef<A> c, int n, int ntau,
                                                           int M, A *__restrict__ Md) {
  const size_t col = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // m * ntau + tau
  if (col >= (size_t)M * ntau) return;
  const size_t m = col / ntau, t = col - m * ntau;
  const T *yc = y + m * (size_t)n * ntau + t;
  A *mc = Md + m * (size_t)n * ntau + t;
  mc[0] = A(0);
  mc[(size_t)(n - 1) * ntau] = A(0);
  if (n < 3) return;
  A y0 = (A)yc[0], y1 = (A)yc[ntau];
  A s0 = (y1 - y0) * c.ih[0];  // slope of the previous interval
  A dprev = A(0);
#pragma unroll 8
  for (int j = 1; j < n - 1; ++j) {
    const A y2 = (A)yc[(size_t)(j + 1) * ntau];
    const A s1 = (y2 - y1) * c.ih[j];
    const A r = A(6) * (s1 - s0);
    const A d = (r - (j > 1 ? c.h[j - 1] * dprev : A(0))) * c.inv[j];
    mc[(size_t)j * ntau] = d;
    dprev = d;
    y1 = y2;
    s0 = s1;
  }
  A next = A(0);  // M_(n-1)
#pragma unroll 8
  for (int j = n - 2; j >= 1; --j) {
    const A v = mc[(size_t)j * ntau] - c.cp[j] * next;
    mc[(size_t)j * ntau] = v;
    next = v;
  }
}

// Blocks: x = (block of kQB output nodes) * ntc + (tau chunk of 256),
// y = source; tau is the fastest index, so loads and stores are coalesced.
// Each thread walks kQB consecutive output nodes of its column and reloads
// the interval's y and M only when the interval changes.
constexpr int kQB = 64;

template <typename T, typename A>
__global__ void __launch_bounds__(256) spline_eval_kernel(const T *__restrict__ y, const A *__restrict__ Md,
                                                          const int *__restrict__ jq, const A *__restrict__ tq,
                                                          const A *__restrict__ hq, int n, int nq, int ntau, int ntc,
                                                          T *__restrict__ out) {
  const int qb = (int)(blockIdx.x / (unsigned)ntc);
  const int t = (int)(blockIdx.x - (unsigned)qb * ntc) * 256 + threadIdx.x;
  if (t >= ntau) return;
  const size_t m = blockIdx.y;
  const int q0 = qb * kQB, q1 = min(nq, q0 + kQB);
  int jc = -1;
  A y0 = A(0), y1 = A(0), m0 = A(0), m1 = A(0);
  for (int q = q0; q < q1; ++q) {
    const int j = jq[q];
    if (j != jc) {
      const size_t i0 = (m * (size_t)n + j) * ntau + t, i1 = i0 + ntau;
      y0 = (A)y[i0];
      y1 = (A)y[i1];
      m0 = Md[i0];
      m1 = Md[i1];
      jc = j;
    }
    const A s = tq[q], h = hq[q], u = A(1) - s;
    // u^3 - u = -s u (1 + u) and s^3 - s = -s u (1 + s): no cancellation near the nodes
    const A su = s * u;
    const A v = u * y0 + s * y1 - h * h / A(6) * su * ((A(1) + u) * m0 + (A(1) + s) * m1);
    out[(m * nq + q) * (size_t)ntau + t] = (T)v;
  }
}

// FP32 sources with ntau % 4 == 0 and 16-byte aligned arrays: the same
// arithmetic per element, four adjacent tau columns a thread (16-byte loads
// and stores; the output is written in 512-byte runs per warp).
__global__ void __launch_bounds__(256) spline_eval4_kernel(const float4 *__restrict__ y, const float4 *__restrict__ Md,
                                                           const int *__restrict__ jq, const float *__restrict__ tq,
                                                           const float *__restrict__ hq, int n, int nq, int nt4,
                                                           int ntc, float4 *__restrict__ out) {
  const int qb = (int)(blockIdx.x / (unsigned)ntc);
  const int t = (int)(blockIdx.x - (unsigned)qb * ntc) * 256 + threadIdx.x;
  if (t >= nt4) return;
  const size_t m = blockIdx.y;
  const int q0 = qb * kQB, q1 = min(nq, q0 + kQB);
  int jc = -1;
  float4 y0{}, y1{}, m0{}, m1{};
  for (int q = q0; q < q1; ++q) {
    const int j = jq[q];
    if (j != jc) {
      const size_t i0 = (m * (size_t)n + j) * nt4 + t, i1 = i0 + nt4;
      y0 = y[i0];
      y1 = y[i1];
      m0 = Md[i0];
      m1 = Md[i1];
      jc = j;
    }
    const float s = tq[q], h = hq[q], u = 1.f - s;
    const float su = s * u, c = h * h / 6.f * su, a = 1.f + u, b = 1.f + s;
    float4 v;
    v.x = u * y0.x + s * y1.x - c * (a * m0.x + b * m1.x);
    v.y = u * y0.y + s * y1.y - c * (a * m0.y + b * m1.y);
    v.z = u * y0.z + s * y1.z - c * (a * m0.z + b * m1.z);
    v.w = u * y0.w + s * y1.w - c * (a * m0.w + b * m1.w);
    out[(m * nq + q) * (size_t)nt4 + t] = v;
  }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace regions (each 256-byte aligned): node coefficients in FP64
// [4][n] and FP32 [4][n]; each output node's t and h in FP64 [2][nq] and FP32
// [2][nq]; its interval [nq] (int); the second derivatives [M][n][ntau] in the
// arithmetic's precision (sized for FP64).
struct InterpLayout {
  size_t c64, c32, q64, q32, qj, md, total;
  InterpLayout(int M, int n, int ntau, int nq) {
    c64 = 0;
    c32 = c64 + a256((size_t)n * 4 * sizeof(double));
    q64 = c32 + a256((size_t)n * 4 * sizeof(float));
    q32 = q64 + a256((size_t)nq * 2 * sizeof(double));
    qj = q32 + a256((size_t)nq * 2 * sizeof(float));
    md = qj + a256((size_t)nq * sizeof(int));
    total = md + a256((size_t)M * n * ntau * sizeof(double));
  }
};

template <typename T, typename A>
int launch_interp_t(const InterpLayout &L, char *w, int n, int nq, int ntau, int M, const T *S_in, T *S_out,
                    cudaStream_t st) {
  const A *c = reinterpret_cast<const A *>(w + (sizeof(A) == 8 ? L.c64 : L.c32));
  const A *qd = reinterpret_cast<const A *>(w + (sizeof(A) == 8 ? L.q64 : L.q32));
  NodeCoef<A> nc{c, c + n, c + 2 * n, c + 3 * n};
  A *Md = reinterpret_cast<A *>(w + L.md);
  const size_t cols = (size_t)M * ntau;
  const int ntc = (ntau + 255) / 256, nqb = (nq + kQB - 1) / kQB;
  spline_solve_kernel<T, A><<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(S_in, nc, n, ntau, M, Md);
  if constexpr (sizeof(T) == 4 && sizeof(A) == 4) {
    if (ntau % 4 == 0 && reinterpret_cast<uintptr_t>(S_in) % 16 == 0 && reinterpret_cast<uintptr_t>(S_out) % 16 == 0 &&
        reinterpret_cast<uintptr_t>(Md) % 16 == 0) {
      const int nt4 = ntau / 4, ntc4 = (nt4 + 255) / 256;
      spline_eval4_kernel<<<dim3((unsigned)((size_t)nqb * ntc4), (unsigned)M), 256, 0, st>>>(
          reinterpret_cast<const float4 *>(S_in), reinterpret_cast<const float4 *>(Md),
          reinterpret_cast<const int *>(w + L.qj), qd, qd + nq, n, nq, nt4, ntc4, reinterpret_cast<float4 *>(S_out));
      return GCAMB_OK;
    }
  }
  spline_eval_kernel<T, A><<<dim3((unsigned)((size_t)nqb * ntc), (unsigned)M), 256, 0, st>>>(
      S_in, Md, reinterpret_cast<const int *>(w + L.qj), qd, qd + nq, n, nq, ntau, ntc, S_out);
  return GCAMB_OK;
}

}  // namespace

size_t interp_workspace_bytes(int M, int nk_in, int ntau, int nk_out) {
  return InterpLayout(M, nk_in, ntau, nk_out).total;
}

int launch_interp_sources(const double *k_in, int nk_in, const void *S_in, int M, int ntau, int dtype,
                          const gcamb_grid *g, void *S_out, void *ws, size_t ws_bytes, cudaStream_t st) {
  const int n = nk_in, nq = g->nk;
  const InterpLayout L(M, n, ntau, nq);
  if (ws_bytes < L.total) return fail(GCAMB_EINVAL, "interp_sources: workspace too small");
  if ((size_t)nq * ((ntau + 255) / 256) > 0x7fffffffULL || M > 65535 || (size_t)M * ntau / 256 > 0x7fffffffULL)
    return fail(GCAMB_EINVAL, "interp_sources: too many sources or nodes for one launch");
  // elimination coefficients (nodes only) and each output node's interval
  std::vector<double> c64(4 * (size_t)n, 0.0), q64(2 * (size_t)nq);
  std::vector<int> qj(nq);
  double *h = c64.data(), *ih = h + n, *cp = ih + n, *inv = cp + n;
  for (int j = 0; j + 1 < n; ++j) {
    h[j] = k_in[j + 1] - k_in[j];
    ih[j] = 1.0 / h[j];
  }
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
    q64[q] = (k - k_in[j]) / h[j];
    q64[nq + q] = h[j];
  }
  std::vector<float> c32(c64.begin(), c64.end()), q32(q64.begin(), q64.end());
  char *w = static_cast<char *>(ws);
  // pageable copies return once the host data is staged
  cudaError_t e = cudaMemcpyAsync(w + L.c64, c64.data(), c64.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w + L.c32, c32.data(), c32.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w + L.q64, q64.data(), q64.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w + L.q32, q32.data(), q32.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w + L.qj, qj.data(), qj.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "interp_sources: coefficient upload");
  ProfScope prof(GCAMB_K_INTERP, st);
  if (dtype == GCAMB_F64)
    launch_interp_t<double, double>(L, w, n, nq, ntau, M, static_cast<const double *>(S_in),
                                    static_cast<double *>(S_out), st);
  else
    launch_interp_t<float, float>(L, w, n, nq, ntau, M, static_cast<const float *>(S_in), static_cast<float *>(S_out),
                                  st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "interp_sources: launch");
  return GCAMB_OK;
}

namespace {

// C_l on every multipole from a grid of sampled multipoles: the natural cubic
// spline in l of D_l = l (l+1) C_l through the sampled rows; sampled
// multipoles are copied.  The elimination coefficients depend on the sampled
// multipoles only and come from the host (no divisions on the device); one
// thread per model runs the FP64 sweep over the nl samples ...
__global__ void cl_spline_solve_kernel(const double *__restrict__ Cs, const int *__restrict__ lrow,
                                       const double *__restrict__ h, const double *__restrict__ ih,
                                       const double *__restrict__ cp, const double *__restrict__ inv, int nl, int M,
                                       double *__restrict__ Md) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const double *c = Cs + (size_t)m * nl;
  double *mm = Md + (size_t)m * nl;
  mm[0] = 0.0;
  mm[nl - 1] = 0.0;
  if (nl < 3) return;
  auto D = [&](int j) { const double l = __ldg(lrow + j); return l * (l + 1.0) * __ldg(c + j); };
  double y1 = D(1);
  double s0 = (y1 - D(0)) * ih[0];
  double dprev = 0.0;
#pragma unroll 8
  for (int j = 1; j < nl - 1; ++j) {
    const double y2 = D(j + 1);
    const double s1 = (y2 - y1) * ih[j];
    const double d = (6.0 * (s1 - s0) - (j > 1 ? h[j - 1] * dprev : 0.0)) * inv[j];
    mm[j] = d;
    dprev = d;
    y1 = y2;
    s0 = s1;
  }
  double next = 0.0;
#pragma unroll 8
  for (int j = nl - 2; j >= 1; --j) {
    const double v = mm[j] - cp[j] * next;
    mm[j] = v;
    next = v;
  }
}

// ... and one thread per (model, l) evaluates, with each output multipole's
// bracketing samples (lo, lo+1) and position s from the host.
__global__ void cl_spline_eval_kernel(const double *__restrict__ Cs, const double *__restrict__ Md,
                                      const int *__restrict__ lrow, const int *__restrict__ rowof,
                                      const int *__restrict__ jl, const double *__restrict__ sl, int nl, int lmin,
                                      int nout, int M, double *__restrict__ out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)M * nout) return;
  const int m = (int)(e / nout), i = (int)(e - (size_t)m * nout);
  const int l = lmin + i;
  const double *c = Cs + (size_t)m * nl;
  const int own = rowof[i];
  if (own >= 0) {
    out[e] = c[own];
    return;
  }
  const int lo = jl[i];
  const double l0 = lrow[lo], l1 = lrow[lo + 1], h = l1 - l0;
  const double s = sl[i], u = 1.0 - s, su = s * u;
  const double y0 = l0 * (l0 + 1.0) * c[lo], y1 = l1 * (l1 + 1.0) * c[lo + 1];
  const double *mm = Md + (size_t)m * nl;
  const double d = u * y0 + s * y1 - h * h / 6.0 * su * ((1.0 + u) * mm[lo] + (1.0 + s) * mm[lo + 1]);
  out[e] = d / ((double)l * (l + 1.0));
}

// The same in one block per model for up to kSmemSamples samples: the
// model's D_l and the coefficients are staged in shared memory, thread 0
// sweeps there (no global-memory latency in the chain), then the block
// evaluates the model's multipoles.
constexpr int kSmemSamples = 4000;

__global__ void __launch_bounds__(256) cl_spline_block_kernel(const double *__restrict__ Cs,
                                                              const int *__restrict__ lrow,
                                                              const int *__restrict__ rowof,
                                                              const double *__restrict__ coef,
                                                              const int *__restrict__ jl,
                                                              const double *__restrict__ sl, int nl, int lmin,
                                                              int nout, double *__restrict__ out) {
  extern __shared__ double sh[];
  double *y = sh, *mm = y + nl, *h = mm + nl, *ih = h + nl, *cp = ih + nl, *inv = cp + nl;
  const int m = blockIdx.x;
  const double *c = Cs + (size_t)m * nl;
  for (int j = threadIdx.x; j < nl; j += blockDim.x) {
    const double l = lrow[j];
    y[j] = l * (l + 1.0) * c[j];
    h[j] = coef[j];
    ih[j] = coef[nl + j];
    cp[j] = coef[2 * nl + j];
    inv[j] = coef[3 * nl + j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mm[0] = 0.0;
    mm[nl - 1] = 0.0;
    if (nl >= 3) {
      double s0 = (y[1] - y[0]) * ih[0], dprev = 0.0;
      for (int j = 1; j < nl - 1; ++j) {
        const double s1 = (y[j + 1] - y[j]) * ih[j];
        const double d = (6.0 * (s1 - s0) - (j > 1 ? h[j - 1] * dprev : 0.0)) * inv[j];
        mm[j] = d;
        dprev = d;
        s0 = s1;
      }
      double next = 0.0;
      for (int j = nl - 2; j >= 1; --j) {
        next = mm[j] - cp[j] * next;
        mm[j] = next;
      }
    }
  }
  __syncthreads();
  double *o = out + (size_t)m * nout;
  for (int i = threadIdx.x; i < nout; i += blockDim.x) {
    const int own = rowof[i];
    if (own >= 0) {
      o[i] = c[own];
      continue;
    }
    const int l = lmin + i, lo = jl[i];
    const double hh = h[lo], s = sl[i], u = 1.0 - s, su = s * u;
    const double d = u * y[lo] + s * y[lo + 1] - hh * hh / 6.0 * su * ((1.0 + u) * mm[lo] + (1.0 + s) * mm[lo + 1]);
    o[i] = d / ((double)l * (l + 1.0));
  }
}

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Workspace: [h, 1/h, c', 1/den] (4 nl doubles) | [s] (nout doubles) |
// [lo] (nout ints) | second derivatives [M][nl] (doubles).
size_t cl_interp_workspace_bytes(const gcamb_grid *g, int M) {
  const size_t nout = (size_t)(g->lmax - g->lmin + 1);
  return al(4 * (size_t)g->nl * sizeof(double)) + al(nout * sizeof(double)) + al(nout * sizeof(int)) +
         al((size_t)M * g->nl * sizeof(double));
}

}  // namespace gcamb

using namespace gcamb;

extern "C" {

int gcamb_cl_interp_workspace(const gcamb_grid *g, int M, size_t *bytes) {
  if (!g || !bytes || M < 0) return fail(GCAMB_EINVAL, "cl_interp_workspace: bad argument");
  *bytes = cl_interp_workspace_bytes(g, M);
  return GCAMB_OK;
}

int gcamb_cl_interp(const gcamb_grid *g, const double *Cl_s, int M, double *Cl, void *ws, size_t ws_bytes,
                    void *stream) {
  if (!g) return fail(GCAMB_EINVAL, "cl_interp: NULL grid");
  if (M < 0) return fail(GCAMB_EINVAL, "cl_interp: M < 0");
  if (M == 0) return GCAMB_OK;
  if (!Cl_s || !Cl || !ws) return fail(GCAMB_EINVAL, "cl_interp: NULL pointer");
  if (ws_bytes < cl_interp_workspace_bytes(g, M)) return fail(GCAMB_EINVAL, "cl_interp: workspace too small");
  if (int rc = ensure_device_grid(const_cast<gcamb_grid *>(g))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nl = g->nl, nout = g->lmax - g->lmin + 1;
  std::vector<double> coef(4 * (size_t)nl, 0.0), sv(nout, 0.0);
  std::vector<int> jv(nout, 0);
  double *h = coef.data(), *ih = h + nl, *cp = ih + nl, *inv = cp + nl;
  for (int j = 0; j + 1 < nl; ++j) {
    h[j] = (double)(g->lrow[j + 1] - g->lrow[j]);
    ih[j] = 1.0 / h[j];
  }
  for (int j = 1; j < nl - 1; ++j) {
    const double den = 2.0 * (h[j - 1] + h[j]) - (j > 1 ? h[j - 1] * cp[j - 1] : 0.0);
    inv[j] = 1.0 / den;
    cp[j] = (j < nl - 2 ? h[j] : 0.0) * inv[j];
  }
  for (int i = 0, j = 0; i < nout && nl > 1; ++i) {
    const int l = g->lmin + i;
    while (j + 2 < nl && g->lrow[j + 1] <= l) ++j;
    jv[i] = j;
    sv[i] = (l - g->lrow[j]) * ih[j];
  }
  char *w = static_cast<char *>(ws);
  const size_t o1 = al(4 * (size_t)nl * sizeof(double)), o2 = o1 + al((size_t)nout * sizeof(double));
  const size_t o3 = o2 + al((size_t)nout * sizeof(int));
  double *d_coef = reinterpret_cast<double *>(w);
  double *d_s = reinterpret_cast<double *>(w + o1);
  int *d_j = reinterpret_cast<int *>(w + o2);
  double *Md = reinterpret_cast<double *>(w + o3);
  // pageable copies return once the host data is staged
  cudaError_t e = cudaMemcpyAsync(d_coef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_s, sv.data(), sv.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_j, jv.data(), jv.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "cl_interp: coefficient upload");
  ProfScope prof(GCAMB_K_INTERP, st);
  if (nl <= kSmemSamples) {
    const size_t smem = (size_t)6 * nl * sizeof(double);
    e = cudaFuncSetAttribute(cl_spline_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cl_interp: smem attribute");
    cl_spline_block_kernel<<<M, 256, smem, st>>>(Cl_s, g->d_lrow, g->d_rowof, d_coef, d_j, d_s, nl, g->lmin, nout, Cl);
  } else {
    cl_spline_solve_kernel<<<(M + 127) / 128, 128, 0, st>>>(Cl_s, g->d_lrow, d_coef, d_coef + nl, d_coef + 2 * nl,
                                                            d_coef + 3 * nl, nl, M, Md);
    const size_t n = (size_t)M * nout;
    cl_spline_eval_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Cl_s, Md, g->d_lrow, g->d_rowof, d_j, d_s, nl,
                                                                       g->lmin, nout, M, Cl);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "cl_interp: launch");
  return GCAMB_OK;
}

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
