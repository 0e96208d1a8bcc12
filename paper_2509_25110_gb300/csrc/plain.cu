// Plain FP64 / FP32 path: the tau-window sum of Eq. (2) per (k, l) on the CUDA
// cores (Algorithm 1's gang over k and vector loops over l and tau, here one
// CTA per (l-tile, k, source chunk) and one warp per multipole row), and the
// FP64 k-sum of Eq. (1).
#include "internal.h"

namespace gcamb {

// One CTA: 128 multipoles x MC sources at one k.  The sources' tau-prefix is
// staged in shared memory; each warp walks table rows (tau contiguous, read
// coalesced), the lanes split tau and reduce by shuffles.
template <typename T, int MC>
__global__ void __launch_bounds__(256) los_plain_kernel(const T *__restrict__ table, const int32_t *__restrict__ nkb,
                                                        const int64_t *__restrict__ off, int nk, int nlt, int lmin,
                                                        int lmax, int ntau, const T *__restrict__ S, int M,
                                                        T *__restrict__ Delta) {
  constexpr int KB = 64;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *s = reinterpret_cast<T *>(smem_raw);  // [MC][ext]
  __shared__ T res[MC][kTileL];
  const int lt = blockIdx.x, q = blockIdx.y, m0 = blockIdx.z * MC;
  const int nl = lmax - lmin + 1;
  const int l0 = lmin + lt * kTileL;
  const size_t e_idx = (size_t)q * nlt + lt;
  const int nb = nkb[e_idx];
  const int ext = nb * KB;
  const int mc = min(MC, M - m0);
  for (int idx = threadIdx.x; idx < MC * ext; idx += blockDim.x) {
    const int m = idx / ext, t = idx - m * ext;
    s[idx] = (m < mc && t < ntau) ? S[((size_t)(m0 + m) * nk + q) * ntau + t] : T(0);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T *chunk = table + (size_t)off[e_idx] * (kTileL * KB);
  for (int r = warp; r < kTileL; r += 8) {
    T acc[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) acc[m] = T(0);
    if (l0 + r <= lmax) {
      const T *row = chunk + r * KB + lane;
      for (int b = 0; b < nb; ++b) {
        const T ja = __ldg(row + (size_t)b * kTileL * KB);
        const T jb = __ldg(row + (size_t)b * kTileL * KB + 32);
        const int t = b * KB + lane;
#pragma unroll
        for (int m = 0; m < MC; ++m) {
          acc[m] = fma(ja, s[m * ext + t], acc[m]);
          acc[m] = fma(jb, s[m * ext + t + 32], acc[m]);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < MC; ++m) {
      T v = acc[m];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) res[m][r] = v;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < MC * kTileL; idx += blockDim.x) {
    const int m = idx / kTileL, r = idx - m * kTileL;
    const int l = l0 + r;
    if (m < mc && l <= lmax) Delta[((size_t)(m0 + m) * nk + q) * nl + (l - lmin)] = res[m][r];
  }
}

template <typename T, int MC>
static int launch_plain_t(const gcamb_grid *g, const Table &t, const T *S, int M, T *Delta, cudaStream_t st) {
  int max_ext = 0;
  for (int v : t.nkb) max_ext = max_ext > v ? max_ext : v;
  max_ext *= 64;
  const size_t smem = (size_t)MC * max_ext * sizeof(T);
  if (smem > 200 * 1024) return fail(GCAMB_EINVAL, "los_transfer: tau grid too long for the plain kernel");
  cudaError_t e = cudaFuncSetAttribute(los_plain_kernel<T, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(smem > 0 ? smem : 16));
  if (e != cudaSuccess) return cuda_fail(e, "los_transfer: smem attribute");
  dim3 grid(g->nlt, g->nk, (M + MC - 1) / MC);
  if (grid.z > 65535) return fail(GCAMB_EINVAL, "los_transfer: too many sources for one launch");
  ProfScope prof(GCAMB_K_LOS_PLAIN, st);
  los_plain_kernel<T, MC><<<grid, 256, smem, st>>>(static_cast<const T *>(t.d_data), t.d_nkb, t.d_off, g->nk, g->nlt,
                                                   g->lmin, g->lmax, g->ntau, S, M, Delta);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "los_transfer: launch");
  return GCAMB_OK;
}

int launch_los_plain(const gcamb_grid *g, const void *S, int M, int mode, void *Delta, cudaStream_t st) {
  const Table &t = g->tab[mode];
  if (mode == GCAMB_PLAIN64) {
    auto s = static_cast<const double *>(S);
    auto d = static_cast<double *>(Delta);
    if (M >= 4) return launch_plain_t<double, 4>(g, t, s, M, d, st);
    if (M >= 2) return launch_plain_t<double, 2>(g, t, s, M, d, st);
    return launch_plain_t<double, 1>(g, t, s, M, d, st);
  }
  auto s = static_cast<const float *>(S);
  auto d = static_cast<float *>(Delta);
  if (M >= 8) return launch_plain_t<float, 8>(g, t, s, M, d, st);
  if (M >= 4) return launch_plain_t<float, 4>(g, t, s, M, d, st);
  if (M >= 2) return launch_plain_t<float, 2>(g, t, s, M, d, st);
  return launch_plain_t<float, 1>(g, t, s, M, d, st);
}

// C_l[m][l] = 4 pi sum_k w_k P[m][k] Delta[m][k][l]^2 in FP64, increasing k.
template <typename TD>
__global__ void __launch_bounds__(256) cl_kernel(const TD *__restrict__ Delta, const double *__restrict__ Pk,
                                                 const double *__restrict__ wk, int nk, int nl,
                                                 double *__restrict__ Cl) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (l >= nl) return;
  const TD *d = Delta + (size_t)m * nk * nl + l;
  const double *p = Pk + (size_t)m * nk;
  const double four_pi = 4.0 * 3.14159265358979323846;
  double acc = 0.0;
  for (int q = 0; q < nk; ++q) {
    const double v = (double)d[(size_t)q * nl];
    const double f = four_pi * wk[q] * p[q];
    acc = fma(f, v * v, acc);
  }
  Cl[(size_t)m * nl + l] = acc;
}

int launch_cl(const gcamb_grid *g, const void *Delta, int d_dtype, const double *Pk, int M, double *Cl,
              cudaStream_t st) {
  if (M > 65535) return fail(GCAMB_EINVAL, "cl: too many sources for one launch");
  dim3 grid((g->nl + 255) / 256, M);
  ProfScope prof(GCAMB_K_CL, st);
  if (d_dtype == GCAMB_F64)
    cl_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double *>(Delta), Pk, g->d_wk, g->nk, g->nl, Cl);
  else
    cl_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float *>(Delta), Pk, g->d_wk, g->nk, g->nl, Cl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "cl: launch");
  return GCAMB_OK;
}

}  // namespace gcamb
