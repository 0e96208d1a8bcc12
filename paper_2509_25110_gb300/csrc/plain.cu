// Plain FP64 / FP32 path: the tau-window sum of Eq. (2) per (k, l) on the CUDA
// cores (Algorithm 1's gang over k and vector loops over l and tau, here one
// CTA per (l-tile, k, source chunk) and one warp per multipole row), and the
// FP64 k-sum of Eq. (1).
#include <cmath>

#include "internal.h"

namespace gcamb {

// Sum over the warp of each of the V values v[0..V) (V = 1, 2, 4, 8): every
// step of the first log2(V) halves the values a lane holds (a lane keeps one
// half, sends the other to its partner and adds what it receives), then plain
// shuffle adds finish; lane L returns the total of value L >> (5 - log2 V).
// (V - 1) + (5 - log2 V) adds a lane instead of 5 V.
template <typename T, int N, int V>
__device__ __forceinline__ void halve_lanes(T (&v)[V], int lane, int o) {
  const bool up = (lane & o) != 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const T send = up ? v[j] : v[j + N];
    const T keep = up ? v[j + N] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
}

template <typename T, int V>
__device__ __forceinline__ T reduce_lanes(T (&v)[V], int lane) {
  static_assert(V == 1 || V == 2 || V == 4 || V == 8, "reduce_lanes: V in {1, 2, 4, 8}");
  int o = 16;
  if constexpr (V >= 8) {
    halve_lanes<T, 4>(v, lane, o);
    o >>= 1;
  }
  if constexpr (V >= 4) {
    halve_lanes<T, 2>(v, lane, o);
    o >>= 1;
  }
  if constexpr (V >= 2) {
    halve_lanes<T, 1>(v, lane, o);
    o >>= 1;
  }
  T t = v[0];
  for (; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// One CTA: 128 multipoles x MC sources at one k.  The sources' tau-prefix is
// staged in shared memory; each warp walks table rows (tau contiguous, read
// coalesced), the lanes split tau and reduce by shuffles.
//
// xthr (temperature on flat j_l grids, else null): per row the Watson
// threshold below which |j_l| < eps_cut.  The tile's tau-prefix is that of
// its lowest multipole; a row stops at the first 64-node block whose first
// node has x below its own threshold (x falls along tau, so every later node
// is below it too): the terms left out are below eps_cut |w S| each.
//
// E = true: E-mode polarisation, Eq. (3) with eps_l(x) = c_l j_l(x)/x^2,
// c_l = sqrt((l+2)!/(l-2)!).  The j_l table is shared with temperature: the
// staged source is S_P/x^2, the row sum is multiplied by c_l.  Nodes with
// x < x_lo (x = 0 included) are left out of the table sum: there the table's
// j_2 may be cut to zero (activity threshold, Miller start) although
// j_2(x)/x^2 -> 1/15.  They add, to l = 2 only, the power series
//   j_2(x)/x^2 = 1/15 - x^2/210 + x^4/7560 - x^6/498960 + O(x^8)
// (from j_l(x) = x^l sum_n (-x^2/2)^n / (n! (2l+2n+1)!!)); for l >= 3 their
// eps_l is below c_l x_lo^(l-2)/(2l+1)!!, and x_lo <= 0.2.
//
// XP: the staged source is S x^-XP for x >= x_lo and 0 below (XP >= 0), or
// S itself (XP < 0, temperature); E: the E-mode epilogue above (XP = 2).
// XP = 0, 1, 2 without E give the raw sums D_XP[l] = sum_i w_i j_l S x^-XP of
// the tensor-mode kernels.
template <typename T, int MC, int XP, bool E>
__global__ void __launch_bounds__(256) los_plain_kernel(const T *__restrict__ table, const int32_t *__restrict__ nkb,
                                                        const int64_t *__restrict__ off, int nk, int nlt, int nl,
                                                        const int *__restrict__ lrow, int ntau,
                                                        const T *__restrict__ S, int M,
                                                        T *__restrict__ Delta, const double *__restrict__ kk,
                                                        const double *__restrict__ tau, double tau0,
                                                        const double *__restrict__ wtau, double x_lo,
                                                        const double *__restrict__ xthr) {
  constexpr int KB = 64;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *s = reinterpret_cast<T *>(smem_raw);  // [MC][ext]
  __shared__ T res[MC][kTileL];
  const int lt = blockIdx.x, q = blockIdx.y, m0 = blockIdx.z * MC;
  const int row0 = lt * kTileL;  // first row (output index) of the tile
  const size_t e_idx = (size_t)q * nlt + lt;
  const int nb = nkb[e_idx];
  const int ext = nb * KB;
  const int mc = min(MC, M - m0);
  for (int idx = threadIdx.x; idx < MC * ext; idx += blockDim.x) {
    const int m = idx / ext, t = idx - m * ext;
    T v = (m < mc && t < ntau) ? S[((size_t)(m0 + m) * nk + q) * ntau + t] : T(0);
    if constexpr (XP >= 0) {
      if (m < mc && t < ntau) {
        const double x = kk[q] * (tau0 - tau[t]);
        const double f = XP == 2 ? 1.0 / (x * x) : (XP == 1 ? 1.0 / x : 1.0);
        v = x >= x_lo ? (T)((double)v * f) : T(0);
      }
    }
    s[idx] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T *chunk = table + (size_t)off[e_idx] * (kTileL * KB);
  // A warp takes RV adjacent rows at a time, so that it holds V = MC RV = 8
  // sums a lane and their cross-lane reduction costs 7 + 2 adds a lane for
  // the 8 sums (5 a sum one at a time: on GB300's narrow FP64 pipe that was
  // a third of the plain FP64 path's work for one source).
  constexpr int RV = 8 / MC, V = MC * RV;
  static_assert(kTileL % (8 * RV) == 0, "rows per warp pass");
  for (int rb = warp * RV; rb < kTileL; rb += 8 * RV) {
    T acc[V];  // acc[m * RV + i]: source m, row rb + i
#pragma unroll
    for (int j = 0; j < V; ++j) acc[j] = T(0);
    int nbr[RV];  // blocks each row needs
    int nbmax = 0;
#pragma unroll
    for (int i = 0; i < RV; ++i) {
      nbr[i] = 0;
      if (row0 + rb + i < nl) {
        nbr[i] = nb;
        if (xthr) {
          const double xe = xthr[row0 + rb + i], kq = kk[q];
          nbr[i] = 0;
          for (int b0 = 0; b0 < nb; b0 += 32) {
            const int b = b0 + lane;
            nbr[i] += __popc(__ballot_sync(0xffffffffu, b < nb && kq * (tau0 - tau[b * KB]) >= xe));
          }
        }
      }
      nbmax = max(nbmax, nbr[i]);
    }
    const T *rows = chunk + rb * KB + lane;
    for (int b = 0; b < nbmax; ++b) {
      const int t = b * KB + lane;
      T sa[MC], sb[MC];
#pragma unroll
      for (int m = 0; m < MC; ++m) {
        sa[m] = s[m * ext + t];
        sb[m] = s[m * ext + t + 32];
      }
#pragma unroll
      for (int i = 0; i < RV; ++i) {
        if (b >= nbr[i]) continue;  // the same for every lane
        const T *row = rows + i * KB + (size_t)b * kTileL * KB;
        const T ja = __ldg(row), jb = __ldg(row + 32);
#pragma unroll
        for (int m = 0; m < MC; ++m) {
          acc[m * RV + i] = fma(ja, sa[m], acc[m * RV + i]);
          acc[m * RV + i] = fma(jb, sb[m], acc[m * RV + i]);
        }
      }
    }
    // lane L holds the total of sum L >> 2
    const T v = reduce_lanes<T, V>(acc, lane);
    if ((lane & 3) == 0) {
      const int j = lane >> 2;
      res[j / RV][rb + j % RV] = v;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < MC * kTileL; idx += blockDim.x) {
    const int m = idx / kTileL, r = idx - m * kTileL;
    const int orow = row0 + r;
    if (m < mc && orow < nl) {
      T v = res[m][r];
      if constexpr (E) {
        const int l = lrow[orow];
        const double c = l >= 2 ? sqrt((double)(l + 2) * (l + 1) * l * (l - 1)) : 0.0;
        double d = c * (double)v;
        if (l == 2) {  // the small-x nodes are the tail of the tau grid (x decreases with tau)
          const T *src = S + ((size_t)(m0 + m) * nk + q) * ntau;
          double tail = 0.0;
          for (int i = ntau - 1; i >= 0; --i) {
            const double x = kk[q] * (tau0 - tau[i]);
            if (!(x < x_lo)) break;
            const double x2 = x * x;
            const double e2 = 1.0 / 15.0 - x2 * (1.0 / 210.0 - x2 * (1.0 / 7560.0 - x2 / 498960.0));
            tail += wtau[i] * (double)src[i] * e2;
          }
          d += c * tail;
        }
        v = (T)d;
      }
      Delta[((size_t)(m0 + m) * nk + q) * nl + orow] = v;
    }
  }
}

// E-mode small-x cut: at least 1e-12 and every x at which the l = 2 row of
// the table may hold zero (the activity threshold of the tile holding l = 2,
// the Miller start of j_2); at most 0.2, where the four-term series of
// j_2(x)/x^2 is still exact to 1e-12 (eps_cut <= 1e-3 keeps it near 0.12).
int emode_x_lo(const gcamb_grid *g, double *x_lo) {
  double x = 1e-12;
  if (g->lmin <= 2) {
    if (g->lmin >= 1) x = fmax(x, watson_threshold(g->lmin, std::log(g->eps_cut)));
    if (g->nxs > 2) x = fmax(x, g->xstart[2]);
  }
  *x_lo = x;
  return x <= 0.2 ? 0 : -1;
}

template <typename T, int MC, int XP, bool E>
static int launch_plain_t(const gcamb_grid *g, const Table &t, const T *S, int M, T *Delta, cudaStream_t st) {
  int max_ext = 0;
  for (int v : t.nkb) max_ext = max_ext > v ? max_ext : v;
  max_ext *= 64;
  const size_t smem = (size_t)MC * max_ext * sizeof(T);
  if (smem > 200 * 1024) return fail(GCAMB_EINVAL, "los_transfer: tau grid too long for the plain kernel");
  cudaError_t e = cudaFuncSetAttribute(los_plain_kernel<T, MC, XP, E>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem > 0 ? smem : 16));
  if (e != cudaSuccess) return cuda_fail(e, "los_transfer: smem attribute");
  dim3 grid(g->nlt, g->nk, (M + MC - 1) / MC);
  if (grid.z > 65535) return fail(GCAMB_EINVAL, "los_transfer: too many sources for one launch");
  ProfScope prof(GCAMB_K_LOS_PLAIN, st);
  double x_lo = 1e-12;
  if (XP >= 0 && emode_x_lo(g, &x_lo))
    return fail(GCAMB_EINVAL, "los_transfer: eps_cut too large for the l = 2 limit of the polarisation kernels");
  // rows stop at their own prefix: temperature on flat j_l grids only (the
  // polarisation and tensor sources carry 1/x^2, 1/x factors)
  const double *xthr = (XP < 0 && !E && g->kernel == 0 && !g->curved) ? g->d_xthr : nullptr;
  los_plain_kernel<T, MC, XP, E><<<grid, 256, smem, st>>>(static_cast<const T *>(t.d_data), t.d_nkb, t.d_off,
                                                          g->nk, g->nlt, g->nl, g->d_lrow, g->ntau, S, M, Delta,
                                                          g->d_k, g->d_tau, g->tau0, g->d_wtau, x_lo, xthr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "los_transfer: launch");
  return GCAMB_OK;
}

template <int XP, bool E>
static int launch_los_plain_k(const gcamb_grid *g, const void *S, int M, int mode, void *Delta, cudaStream_t st) {
  const Table &t = g->tab[mode];
  if (mode == GCAMB_PLAIN64) {
    auto s = static_cast<const double *>(S);
    auto d = static_cast<double *>(Delta);
    if (M >= 4) return launch_plain_t<double, 4, XP, E>(g, t, s, M, d, st);
    if (M >= 2) return launch_plain_t<double, 2, XP, E>(g, t, s, M, d, st);
    return launch_plain_t<double, 1, XP, E>(g, t, s, M, d, st);
  }
  auto s = static_cast<const float *>(S);
  auto d = static_cast<float *>(Delta);
  if (M >= 8) return launch_plain_t<float, 8, XP, E>(g, t, s, M, d, st);
  if (M >= 4) return launch_plain_t<float, 4, XP, E>(g, t, s, M, d, st);
  if (M >= 2) return launch_plain_t<float, 2, XP, E>(g, t, s, M, d, st);
  return launch_plain_t<float, 1, XP, E>(g, t, s, M, d, st);
}

int launch_los_plain(const gcamb_grid *g, const void *S, int M, int mode, void *Delta, cudaStream_t st, bool emode) {
  return emode ? launch_los_plain_k<2, true>(g, S, M, mode, Delta, st)
               : launch_los_plain_k<-1, false>(g, S, M, mode, Delta, st);
}

// Tensor modes: power series of the tensor kernels at small x for the nodes
// below the cut, from j_l(x) = x^l s_l(x^2),
// s_l(y) = sum_n (-y/2)^n / (n! (2l+2n+1)!!) (seven terms: exact to rounding
// for x <= 0.2):
//   e_l = x^(l-2) [l (l-1) s_l - 2 x^2 s_l + 2 s_(l-1)],
//   b_l = 2 x^(l-1) [s_(l-1) - (l-1) s_l].
__device__ __forceinline__ double sph_series(int l, double y) {
  double df = 1.0;  // (2l+1)!!
  for (int j = 3; j <= 2 * l + 1; j += 2) df *= j;
  double term = 1.0 / df, sum = term;
  for (int n = 0; n < 6; ++n) {
    term *= (-0.5 * y) / ((n + 1) * (2.0 * l + 2 * n + 3));
    sum += term;
  }
  return sum;
}

// Combines the raw tensor sums, in place: D0 -> Delta_E, D1 -> Delta_B
// (D2 read only), one CTA per (source, k) row walking l in chunks.
//   Delta_E[l] = l (l-1) D2[l] - 2 D0[l] + 2 D1[l-1] + tail_e(l)
//   Delta_B[l] = 2 D0[l-1] - 2 (l-1) D1[l] + tail_b(l)
// Row l-1 of the first multipole (lmin >= 2) comes from the recurrence
// j_(l-1) = (2l+1)/x j_l - j_(l+1):  D1[l-1] = (2l+1) D2[l] - D1[l+1],
// D0[l-1] = (2l+1) D1[l] - D0[l+1] (all three sums leave out the same nodes).
// The tails add, for l = 2..5, the series terms of the nodes below the cut.
template <typename T>
__global__ void __launch_bounds__(256) tensor_combine_kernel(T *__restrict__ DE, T *__restrict__ DB,
                                                             const T *__restrict__ D2, const T *__restrict__ SP,
                                                             const double *__restrict__ kk,
                                                             const double *__restrict__ tau, double tau0,
                                                             const double *__restrict__ wtau, double x_lo, int nk,
                                                             int ntau, int lmin, int lmax) {
  __shared__ double carry[2];
  const int nl = lmax - lmin + 1;
  const size_t row = blockIdx.x;  // m * nk + q
  const int q = (int)(row % nk);
  T *e = DE + row * nl;
  T *b = DB + row * nl;
  const T *d2 = D2 + row * nl;
  const T *src = SP + row * ntau;
  for (int base = 0; base < nl; base += blockDim.x) {
    const int idx = base + threadIdx.x;
    const int l = lmin + idx;
    double d0 = 0, d1 = 0, dd2 = 0, p0 = 0, p1 = 0;
    if (idx < nl) {
      d0 = (double)e[idx];
      d1 = (double)b[idx];
      dd2 = (double)d2[idx];
      if (idx == 0) {
        if (l >= 2 && nl > 1) {
          p1 = (2.0 * l + 1.0) * dd2 - (double)b[1];
          p0 = (2.0 * l + 1.0) * d1 - (double)e[1];
        }
      } else if (threadIdx.x == 0) {
        p0 = carry[0];
        p1 = carry[1];
      } else {
        p0 = (double)e[idx - 1];
        p1 = (double)b[idx - 1];
      }
    }
    __syncthreads();  // every read of this chunk (and of the carry) precedes its writes
    if (threadIdx.x == blockDim.x - 1) {
      carry[0] = d0;
      carry[1] = d1;
    }
    if (idx < nl) {
      double ve = 0.0, vb = 0.0;
      if (l >= 2) {
        ve = (double)l * (l - 1) * dd2 - 2.0 * d0 + 2.0 * p1;
        vb = 2.0 * p0 - 2.0 * (l - 1) * d1;
        if (l <= 5) {
          for (int i = ntau - 1; i >= 0; --i) {
            const double x = kk[q] * (tau0 - tau[i]);
            if (x >= x_lo) break;
            const double y = x * x, sl = sph_series(l, y), sm = sph_series(l - 1, y);
            const double xl2 = l == 2 ? 1.0 : pow(x, l - 2);
            const double ws = wtau[i] * (double)src[i];
            ve += ws * xl2 * ((double)l * (l - 1) * sl - 2.0 * y * sl + 2.0 * sm);
            vb += ws * 2.0 * xl2 * x * (sm - (l - 1) * sl);
          }
        }
      }
      e[idx] = (T)ve;
      b[idx] = (T)vb;
    }
    __syncthreads();  // the carry is read by the next chunk
  }
}

int launch_los_tensor(const gcamb_grid *g, const void *ST, const void *SP, int M, int mode, void *DT, void *DE,
                      void *DB, cudaStream_t st) {
  if (g->lsampled)
    return fail(GCAMB_EUNSUPPORTED, "los_transfer_tensor: the kernels take row l-1: needs a grid of every multipole");
  if (g->lmin >= 2 && g->lmax == g->lmin)
    return fail(GCAMB_EINVAL, "los_transfer_tensor: needs lmax > lmin when lmin >= 2 (the kernels take j_(l-1))");
  double x_lo = 1e-12;
  if (emode_x_lo(g, &x_lo)) return fail(GCAMB_EINVAL, "los_transfer_tensor: eps_cut too large for the l = 2 limit");
  // raw sums of the polarisation source: D0 -> DE, D1 -> DB, D2 -> DT
  int rc = launch_los_plain_k<0, false>(g, SP, M, mode, DE, st);
  if (!rc) rc = launch_los_plain_k<1, false>(g, SP, M, mode, DB, st);
  if (!rc) rc = launch_los_plain_k<2, false>(g, SP, M, mode, DT, st);
  if (rc) return rc;
  const unsigned rows = (unsigned)((size_t)M * g->nk);
  if ((size_t)M * g->nk > 0x7fffffffULL) return fail(GCAMB_EINVAL, "los_transfer_tensor: too many rows");
  {
    ProfScope prof(GCAMB_K_LOS_PLAIN, st);
    if (mode == GCAMB_PLAIN64)
      tensor_combine_kernel<double><<<rows, 256, 0, st>>>(static_cast<double *>(DE), static_cast<double *>(DB),
                                                          static_cast<const double *>(DT),
                                                          static_cast<const double *>(SP), g->d_k, g->d_tau,
                                                          g->tau0, g->d_wtau, x_lo, g->nk, g->ntau, g->lmin, g->lmax);
    else
      tensor_combine_kernel<float><<<rows, 256, 0, st>>>(static_cast<float *>(DE), static_cast<float *>(DB),
                                                         static_cast<const float *>(DT),
                                                         static_cast<const float *>(SP), g->d_k, g->d_tau, g->tau0,
                                                         g->d_wtau, x_lo, g->nk, g->ntau, g->lmin, g->lmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "los_transfer_tensor: launch");
  }
  // temperature: t_l = c_l j_l / x^2, the E-mode kernel of Eq. (3), into DT
  return launch_los_plain_k<2, true>(g, ST, M, mode, DT, st);
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

// C^XY_l[m] = 4 pi sum_k w_k P[m][k] DX[m][k][l] DY[m][k][l] in FP64, increasing k.
template <typename TD>
__global__ void __launch_bounds__(256) cl_cross_kernel(const TD *__restrict__ DX, const TD *__restrict__ DY,
                                                       const double *__restrict__ Pk, const double *__restrict__ wk,
                                                       int nk, int nl, double *__restrict__ Cl) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (l >= nl) return;
  const size_t base = (size_t)m * nk * nl + l;
  const double *p = Pk + (size_t)m * nk;
  const double four_pi = 4.0 * 3.14159265358979323846;
  double acc = 0.0;
  for (int q = 0; q < nk; ++q) {
    const double f = four_pi * wk[q] * p[q];
    acc = fma(f, (double)DX[base + (size_t)q * nl] * (double)DY[base + (size_t)q * nl], acc);
  }
  Cl[(size_t)m * nl + l] = acc;
}

int launch_cl_cross(const gcamb_grid *g, const void *DX, const void *DY, int d_dtype, const double *Pk, int M,
                    double *Cl, cudaStream_t st) {
  if (M > 65535) return fail(GCAMB_EINVAL, "cl_cross: too many sources for one launch");
  dim3 grid((g->nl + 255) / 256, M);
  ProfScope prof(GCAMB_K_CL, st);
  if (d_dtype == GCAMB_F64)
    cl_cross_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double *>(DX), static_cast<const double *>(DY), Pk,
                                                  g->d_wk, g->nk, g->nl, Cl);
  else
    cl_cross_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float *>(DX), static_cast<const float *>(DY), Pk,
                                                 g->d_wk, g->nk, g->nl, Cl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "cl_cross: launch");
  return GCAMB_OK;
}

// Uneven batch in FP32 on the CUDA cores: C_l[m][row] of one chunk of
// sources (m0 .. m0 + mc), each on its own k prefix [0, nk_m) with the
// trapezoid in ln k of that prefix (the last node of a shorter prefix takes
// half its interval) and zero above its own l_max; Delta [mc][nk][nl] FP32 of
// the chunk (rows beyond the chunk's l-tiles and k beyond its longest prefix
// are not read: they belong to no source's sum).  FP64 sum in increasing k.
__global__ void __launch_bounds__(256) cl_prefix_kernel(const float *__restrict__ Delta, const double *__restrict__ Pk,
                                                        const double *__restrict__ wk, const double *__restrict__ kk,
                                                        int nk, int nl, const int *__restrict__ lrow,
                                                        const int *__restrict__ lmax_m, const int *__restrict__ nk_m,
                                                        int m0, double *__restrict__ Cl) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int mi = blockIdx.y, m = m0 + mi;
  if (row >= nl) return;
  double acc = 0.0;
  if (lrow[row] <= lmax_m[m]) {
    const int nkm = nk_m[m];
    const float *d = Delta + (size_t)mi * nk * nl + row;
    const double *p = Pk + (size_t)m * nk;
    const double four_pi = 4.0 * 3.14159265358979323846;
    for (int q = 0; q < nkm; ++q) {
      // trapezoid in ln k on the prefix [0, nkm)
      const double w = (nkm == nk || q + 1 < nkm) ? wk[q] : (q > 0 ? 0.5 * (log(kk[q]) - log(kk[q - 1])) : 0.0);
      const double v = (double)d[(size_t)q * nl];
      acc = fma(four_pi * w * p[q], v * v, acc);
    }
  }
  Cl[(size_t)m * nl + row] = acc;
}

// Sources per launch pair of the FP32 plan (the Delta buffer of a chunk).
constexpr int kPlainChunk = 16;

size_t plain_plan_workspace_bytes(const gcamb_grid *g, int M) {
  const int mc = M < kPlainChunk ? M : kPlainChunk;
  return (size_t)(mc > 0 ? mc : 1) * g->nk * g->nl * sizeof(float);
}

int launch_plain_plan(const gcamb_grid *g, const float *S, const double *Pk, int M, const int *lmax_c,
                      const int *nk_c, const int *d_lmax, const int *d_nk, double *Cl, void *ws, cudaStream_t st) {
  const Table &t = g->tab[GCAMB_PLAIN32];
  float *D = static_cast<float *>(ws);
  for (int m0 = 0; m0 < M; m0 += kPlainChunk) {
    const int mc = M - m0 < kPlainChunk ? M - m0 : kPlainChunk;
    // the chunk's longest k prefix and highest l-tile (host copies of the plan)
    int nkc = 1, ltc = 0;
    for (int j = m0; j < m0 + mc; ++j) {
      nkc = nk_c[j] > nkc ? nk_c[j] : nkc;
      int r = g->rowof[lmax_c[j] - g->lmin];
      for (int l = lmax_c[j]; r < 0 && l > g->lmin; --l) r = g->rowof[l - 1 - g->lmin];
      const int lt = (r < 0 ? 0 : r) / kTileL;
      ltc = lt > ltc ? lt : ltc;
    }
    int max_ext = 0;
    for (int v : t.nkb) max_ext = max_ext > v ? max_ext : v;
    max_ext *= 64;
    constexpr int MC = 8;
    const size_t smem = (size_t)MC * max_ext * sizeof(float);
    if (smem > 200 * 1024) return fail(GCAMB_EINVAL, "plan_launch: tau grid too long for the plain kernel");
    cudaError_t e = cudaFuncSetAttribute(los_plain_kernel<float, MC, -1, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem > 0 ? smem : 16));
    if (e != cudaSuccess) return cuda_fail(e, "plan_launch: smem attribute");
    const double *xthr = (g->kernel == 0 && !g->curved) ? g->d_xthr : nullptr;
    {
      ProfScope prof(GCAMB_K_LOS_PLAIN, st);
      dim3 grid(ltc + 1, nkc, (mc + MC - 1) / MC);
      los_plain_kernel<float, MC, -1, false><<<grid, 256, smem, st>>>(
          static_cast<const float *>(t.d_data), t.d_nkb, t.d_off, g->nk, g->nlt, g->nl, g->d_lrow, g->ntau,
          S + (size_t)m0 * g->nk * g->ntau, mc, D, g->d_k, g->d_tau, g->tau0, g->d_wtau, 1e-12, xthr);
    }
    {
      ProfScope prof(GCAMB_K_CL, st);
      dim3 grid((g->nl + 255) / 256, mc);
      cl_prefix_kernel<<<grid, 256, 0, st>>>(D, Pk, g->d_wk, g->d_k, g->nk, g->nl, g->d_lrow, d_lmax, d_nk, m0, Cl);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "plan_launch: FP32 launch");
  }
  return GCAMB_OK;
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
