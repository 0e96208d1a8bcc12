// Spherical Bessel tables: w_i j_l(k (tau0 - tau_i)) over the active extents,
// generated in FP64 per (k, tau) node by three-term recurrences in l.
//
// For x = k (tau0 - tau) the orders split at ls = min(floor(x), l_top):
//   l <= ls  (x >= 1): forward recurrence from j_0 = sin x / x and
//            j_1 = (sin x / x - cos x) / x; forward is stable while l < x.
//   l >  ls: Miller's backward recurrence from f_{L+1} = 0, f_L = 1, with L
//            the first order at which Watson's bound (A&S 9.1.63) puts
//            |j_L(x)| below delta; the backward values are scaled to match
//            the forward value at ls or ls-1 (the larger of the two), or to
//            j_0 for x < 1.  A first backward pass finds the scale, a second
//            writes the scaled values, so no per-thread order buffer is kept.
// Recurrence: j_{l-1} + j_{l+1} = (2l+1)/x j_l (both directions).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "internal.h"

namespace gcamb {

// First order l >= lfrom whose start threshold exceeds x (|j_l(x)| < delta);
// xs is increasing for l >= 1.
__device__ __forceinline__ int miller_start(const double *__restrict__ xs, int nxs, int lfrom, double x) {
  int lo = lfrom < 1 ? 1 : lfrom, hi = nxs - 1;
  if (lo >= hi) return hi > lo ? hi : lo;
  if (xs[hi] <= x) return hi;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (xs[mid] > x) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Calls put(l, j_l(x)) for the orders l in [lmin, ltop] that are not below
// the Miller start; orders not passed to put are zero to within delta.
template <class Sink>
__device__ __forceinline__ void bessel_orders(double x, int lmin, int ltop, const double *__restrict__ xs, int nxs,
                                              Sink &put) {
  if (ltop < lmin) return;
  if (x == 0.0) {
    if (lmin == 0) put(0, 1.0);
    return;
  }
  if (x < 1e-150) {  // j_1 = x/3, j_l < 1e-300 for l >= 2
    if (lmin == 0) put(0, 1.0);
    if (lmin <= 1 && ltop >= 1) put(1, x / 3.0);
    return;
  }
  const double inv = 1.0 / x;
  int ls = 0;
  double fa = 0.0, fb = 0.0;  // forward j_{ls-1}, j_{ls}
  double j0 = 0.0;
  if (x >= 1.0) {
    ls = x >= (double)ltop ? ltop : (int)floor(x);
    double s, c;
    sincos(x, &s, &c);
    double jm = s / x;
    double j = (jm - c) / x;
    if (lmin == 0) put(0, jm);
    if (ls >= 1 && lmin <= 1) put(1, j);
    double dl = 3.0;  // 2l+1 at l = 1
    for (int l = 1; l < ls; ++l) {
      const double jn = fma(dl * inv, j, -jm);
      jm = j;
      j = jn;
      dl += 2.0;
      if (l + 1 >= lmin) put(l + 1, j);
    }
    if (ls >= ltop) return;
    fa = jm;
    fb = j;
  } else {
    j0 = sin(x) / x;
    if (lmin == 0) put(0, j0);
  }
  const int L = miller_start(xs, nxs, ls + 1, x);
  const int lstop = x >= 1.0 ? ls - 1 : 0;  // pass 1 ends with f at this order
  // pass 1: scale
  double fh = 0.0, f = 1.0, dl = 2.0 * L + 1.0;
  for (int l = L; l > lstop; --l) {
    const double fm = fma(dl * inv, f, -fh);
    fh = f;
    f = fm;
    dl -= 2.0;
  }
  double scale;
  if (x >= 1.0) scale = (fabs(fb) >= fabs(fa)) ? fb / fh : fa / f;  // fh = f_ls, f = f_{ls-1}
  else scale = j0 / f;                                                // f = f_0
  // pass 2: scaled values above ls
  const int lwrite_hi = L < ltop ? L : ltop;
  fh = 0.0;
  f = 1.0;
  dl = 2.0 * L + 1.0;
  for (int l = L; l > ls; --l) {
    if (l <= lwrite_hi && l >= lmin) put(l, scale * f);
    const double fm = fma(dl * inv, f, -fh);
    fh = f;
    f = fm;
    dl -= 2.0;
  }
}

// Calls put(l, Phi^beta_l(chi)) for l in [lmin, ltop]: the hyperspherical
// Bessel functions of open (closed = false: sh = sinh, ct = coth,
// s_l = sqrt(beta^2 + l^2)) or closed space (sh = sin, ct = cot,
// s_l = sqrt(beta^2 - l^2), integer beta, Phi_l = 0 for l >= beta), with
//   Phi_0 = sin(beta chi) / (beta sh),
//   Phi_1 = (sin(beta chi) ct - beta cos(beta chi)) / (beta sh s_1),
//   s_(l+1) Phi_(l+1) = (2l+1) ct Phi_l - s_l Phi_(l-1).
// Forward from Phi_0, Phi_1 below the turning order beta |sh| (where the
// solutions oscillate); above it Miller's downward recurrence, started past
// max(ltop, turning order) + 60 + 8 sqrt(.) and, in open space, past the
// tail that falls by tanh(chi/2) per order (46 / -ln tanh(chi/2) orders);
// in closed space at most at beta - 1 (exact: Phi_beta = 0).  The downward
// pass rescales by 1e-250 on overflow and counts it; the second pass writes
// scale * f for the orders within one rescale of the match and 0 above.
//
// S, IS (optional): s_l and 1/s_l for l = 0..nS-1 (the block's q), staged in
// shared memory; orders beyond nS fall back to the square root and division.
template <class Sink>
__device__ void hyper_orders(double beta, double chi, bool closed, int lmin, int ltop, Sink &put,
                             const double *S = nullptr, const double *IS = nullptr, int nS = 0) {
  if (ltop < lmin) return;
  if (chi == 0.0) {
    if (lmin == 0) put(0, 1.0);
    return;
  }
  double sh, ch;
  if (closed) {
    sincos(chi, &sh, &ch);
  } else {
    sh = sinh(chi);
    ch = cosh(chi);
  }
  const double ct = ch / sh, b2 = beta * beta, sg = closed ? -1.0 : 1.0;
  auto sl = [&](int l) {
    if (l < nS) return S[l];
    const double v = fma(sg * (double)l, (double)l, b2);
    return v > 0.0 ? sqrt(v) : 0.0;
  };
  auto isl = [&](int l) { return l < nS ? IS[l] : 1.0 / sl(l); };
  const int lcap = closed ? (int)llrint(beta) - 1 : 0x3fffffff;
  const int lt = min(ltop, lcap);
  if (lt < lmin) return;
  double sb, cb;
  sincos(beta * chi, &sb, &cb);
  const double p0 = sb / (beta * sh);
  const double p1 = (sb * ct - beta * cb) / (beta * sh * sl(1));
  const double turn = beta * fabs(sh);
  const int ls = (int)fmin(floor(turn), (double)lt);
  double fa = 0.0, fb = 0.0;  // forward Phi_(ls-1), Phi_ls
  if (ls >= 1) {
    double pm = p0, p = p1, sc = sl(1);
    if (lmin == 0) put(0, p0);
    if (lmin <= 1) put(1, p1);
    for (int l = 1; l < ls; ++l) {
      const double sn = sl(l + 1);
      const double pn = ((2.0 * l + 1.0) * ct * p - sc * pm) * isl(l + 1);
      pm = p;
      p = pn;
      sc = sn;
      if (l + 1 >= lmin) put(l + 1, p);
    }
    if (ls >= lt) return;
    fa = pm;
    fb = p;
  }
  const double hi = fmax((double)lt, turn);
  double extra = 0.0;
  if (!closed) {
    const double th = tanh(0.5 * chi);
    extra = th < 1.0 ? fmin(46.0 / -log(th), 1e6) : 1e6;
  }
  const int L = (int)fmin(hi + 60.0 + 8.0 * sqrt(hi) + extra + 10.0, (double)lcap);
  const int lend = ls >= 1 ? ls : 1;
  // pass 1: down to f_(lend-1), counting rescales
  double fh = 0.0, f = 1.0, s_up = sl(L + 1);
  int R = 0;
  for (int l = L; l >= lend; --l) {
    const double s_l = sl(l);
    const double fm = ((2.0 * l + 1.0) * ct * f - s_up * fh) * isl(l);
    fh = f;
    f = fm;
    s_up = s_l;
    if (fabs(f) > 1e250) {
      f *= 1e-250;
      fh *= 1e-250;
      ++R;
    }
  }
  double scale;  // fh = f_lend, f = f_(lend-1)
  if (ls >= 1) scale = fabs(fb) >= fabs(fa) ? fb / fh : fa / f;
  else scale = fabs(p1) > fabs(p0) ? p1 / fh : p0 / f;
  const double scale2 = scale * 1e-250;
  // pass 2: the orders above the match (all of them when ls = 0)
  const int lbot = ls >= 1 ? ls + 1 : 0;
  fh = 0.0;
  f = 1.0;
  s_up = sl(L + 1);
  int r = 0;
  for (int l = L;; --l) {
    if (l <= lt && l >= lmin) {
      const int d = R - r;
      put(l, d == 0 ? scale * f : (d == 1 ? scale2 * f : 0.0));
    }
    if (l <= lbot) break;
    const double s_l = sl(l);
    const double fm = ((2.0 * l + 1.0) * ct * f - s_up * fh) * isl(l);
    fh = f;
    f = fm;
    s_up = s_l;
    if (fabs(f) > 1e250) {
      f *= 1e-250;
      fh *= 1e-250;
      ++r;
    }
  }
}

__device__ __forceinline__ uint32_t tf32_rna(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

// Byte offset of (row r, column c) in a 128-row plane of 128-byte rows, in the
// 128-byte swizzled order: 16-byte chunk index XOR (r % 8).
__device__ __forceinline__ uint32_t sw128_offset(int r, int cbytes) {
  return (uint32_t)r * 128u + ((uint32_t)((cbytes >> 4) ^ (r & 7)) << 4) + (uint32_t)(cbytes & 15);
}

// The same for 64-byte rows in the 64-byte swizzled order: 16-byte chunk
// index XOR ((r / 2) % 4) (address bits 7-8 into bits 4-5).
__device__ __forceinline__ uint32_t sw64_offset(int r, int cbytes) {
  return (uint32_t)r * 64u + ((uint32_t)((cbytes >> 4) ^ ((r >> 1) & 3)) << 4) + (uint32_t)(cbytes & 15);
}

// Writes w_i j_l into row (l - lmin), or, on a grid of sampled multipoles,
// into row rowof[l - lmin] (orders that are not sampled are skipped).
template <int MODE>
struct TableSink {
  char *table;
  const int64_t *off_q;
  int lmin, kbi, c;
  double w;  // tau weight (times 2^scale for F16X3)
  int cur_lt;
  char *base;
  const int *rowof;  // null: every order is a row
  __device__ __forceinline__ void operator()(int l, double v) {
    const int t = rowof ? rowof[l - lmin] : l - lmin;
    if (t < 0) return;
    const int lt = t >> 7, r = t & 127;
    if (lt != cur_lt) {
      cur_lt = lt;
      base = table + (size_t)(off_q[lt] + kbi) * TableSink::block_bytes();
    }
    const double wv = w * v;
    if constexpr (MODE == GCAMB_PLAIN64) {
      reinterpret_cast<double *>(base)[r * 64 + c] = wv;
    } else if constexpr (MODE == GCAMB_PLAIN32) {
      reinterpret_cast<float *>(base)[r * 64 + c] = (float)wv;
    } else if constexpr (MODE == GCAMB_BF16X3) {
      const __nv_bfloat16 hi = __double2bfloat16(wv);
      const __nv_bfloat16 lo = __double2bfloat16(wv - (double)__bfloat162float(hi));
      const uint32_t o = sw64_offset(r, c * 2);
      *reinterpret_cast<__nv_bfloat16 *>(base + o) = hi;
      *reinterpret_cast<__nv_bfloat16 *>(base + 8192 + o) = lo;
    } else if constexpr (MODE == GCAMB_F16X3) {
      const __half hi = __double2half(wv);
      const __half lo = __double2half(wv - (double)__half2float(hi));
      const uint32_t o = sw64_offset(r, c * 2);
      *reinterpret_cast<__half *>(base + o) = hi;
      *reinterpret_cast<__half *>(base + 8192 + o) = lo;
    } else {  // TF32X3
      const uint32_t hi = tf32_rna((float)wv);
      const uint32_t lo = tf32_rna((float)(wv - (double)__uint_as_float(hi)));
      const uint32_t o = sw128_offset(r, c * 4);
      *reinterpret_cast<uint32_t *>(base + o) = hi;
      *reinterpret_cast<uint32_t *>(base + 16384 + o) = lo;
    }
  }
  static constexpr size_t block_bytes() {
    return MODE == GCAMB_PLAIN64 ? 65536 : (MODE == GCAMB_BF16X3 || MODE == GCAMB_F16X3 ? 16384 : 32768);
  }
};

// Kernel grids: turns the stream put(l, j_l(x)) into put(l, kernel_l(x)) for
//   1: c_l j_l / x^2                          (scalar E, tensor T)
//   2: (l (l-1) / x^2 - 2) j_l + 2 j_(l-1) / x (tensor E)
//   3: 2 j_(l-1) - 2 (l-1) j_l / x            (tensor B)
// (l >= 2).  bessel_orders passes the orders ascending below the match and
// descending above it; each kernel value is formed when j_l and j_(l-1) are
// both at hand, the last forward value being kept across the jump.
template <class Inner>
struct KernelSink {
  Inner &out;
  int kern, lmin;
  double ix, ix2;
  int pl, fl;
  double pv, fv;
  __device__ __forceinline__ void emit(int l, double jl, double jm) {
    if (l < lmin || l < 2) return;
    const double dl = (double)l;
    double v;
    if (kern == 1) v = sqrt((dl + 2.0) * (dl + 1.0) * dl * (dl - 1.0)) * jl * ix2;
    else if (kern == 2) v = (dl * (dl - 1.0) * ix2 - 2.0) * jl + 2.0 * jm * ix;
    else v = 2.0 * jm - 2.0 * (dl - 1.0) * jl * ix;
    out(l, v);
  }
  __device__ __forceinline__ void operator()(int l, double v) {
    if (l == pl + 1) {
      emit(l, v, pv);
    } else if (l == pl - 1) {
      emit(pl, pv, v);
      if (l - 1 == fl) emit(l, v, fv);
    } else {
      fl = pl;
      fv = pv;
    }
    pl = l;
    pv = v;
  }
};

// The kernels at x below the small-x cut (x <= 0.2), from the power series
// j_l = x^l s_l(x^2), s_l(y) = sum_n (-y/2)^n / (n! (2l+2n+1)!!), for l = 2..5
// (every other kernel value there is below c_l x^(l-2) / (2l+1)!!).
__device__ double small_x_kernel(int kern, int l, double x) {
  auto sser = [](int ll, double y) {
    double df = 1.0;
    for (int j = 3; j <= 2 * ll + 1; j += 2) df *= j;
    double term = 1.0 / df, sum = term;
    for (int n = 0; n < 6; ++n) {
      term *= (-0.5 * y) / ((n + 1) * (2.0 * ll + 2 * n + 3));
      sum += term;
    }
    return sum;
  };
  const double y = x * x, sl = sser(l, y), sm = sser(l - 1, y), dl = (double)l;
  const double xl2 = l == 2 ? 1.0 : pow(x, l - 2);
  if (kern == 1) return sqrt((dl + 2.0) * (dl + 1.0) * dl * (dl - 1.0)) * xl2 * sl;
  if (kern == 2) return xl2 * (dl * (dl - 1.0) * sl - 2.0 * y * sl + 2.0 * sm);
  return 2.0 * xl2 * x * (sm - (dl - 1.0) * sl);
}

template <int MODE>
__global__ void __launch_bounds__(128) bessel_table_kernel(const double *__restrict__ k, const double *__restrict__ tau,
                                                           const double *__restrict__ wtau, double tau0, int ntau,
                                                           int lmin, int lmax, int nlt,
                                                           const int32_t *__restrict__ nkb,
                                                           const int64_t *__restrict__ off,
                                                           const double *__restrict__ xs, int nxs, int scale_exp,
                                                           const int *__restrict__ lrow,
                                                           const int *__restrict__ rowof, int nl, int curved,
                                                           double rk, int kern, double x_lo, int ns, void *table) {
  constexpr int KB = (MODE == GCAMB_PLAIN64 || MODE == GCAMB_PLAIN32) ? 64 : 32;
  const int q = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // curved grids: s_l and 1/s_l of this block's q, for l < ns (dynamic shared memory)
  extern __shared__ double s_stage[];
  const double *s_sh = nullptr, *is_sh = nullptr;
  if (curved && ns > 0) {
    const double b2 = (k[q] / rk) * (k[q] / rk), sg = curved == 2 ? -1.0 : 1.0;
    for (int l = threadIdx.x; l < ns; l += blockDim.x) {
      const double v = fma(sg * (double)l, (double)l, b2);
      const double sv = v > 0.0 ? sqrt(v) : 0.0;
      s_stage[l] = sv;
      s_stage[ns + l] = sv > 0.0 ? 1.0 / sv : 0.0;
    }
    __syncthreads();
    s_sh = s_stage;
    is_sh = s_stage + ns;
  }
  if (i >= ntau) return;
  const int32_t *nkb_q = nkb + (size_t)q * nlt;
  const int kbi = i / KB;
  int lt_last = -1;
  while (lt_last + 1 < nlt && nkb_q[lt_last + 1] > kbi) ++lt_last;
  if (lt_last < 0) return;
  // the highest multipole of the last tile this node is active in
  const int ltop = lrow ? lrow[min((lt_last + 1) * kTileL, nl) - 1] : min(lmin + (lt_last + 1) * kTileL - 1, lmax);
  TableSink<MODE> sink{static_cast<char *>(table), off + (size_t)q * nlt, lmin, kbi, i % KB,
                       ldexp(wtau[i], scale_exp), -1, nullptr, rowof};
  if (curved) {  // hyperspherical: beta = q / sqrt|K|, chi = sqrt|K| (tau0 - tau)
    hyper_orders(k[q] / rk, rk * (tau0 - tau[i]), curved == 2, lmin, ltop, sink, s_sh, is_sh, ns);
  } else if (kern) {
    const double x = k[q] * (tau0 - tau[i]);
    if (x < x_lo) {
      for (int l = max(lmin, 2); l <= min(ltop, 5); ++l) sink(l, small_x_kernel(kern, l, x));
    } else {
      KernelSink<TableSink<MODE>> ks{sink, kern, lmin, 1.0 / x, 1.0 / (x * x), -10, -10, 0.0, 0.0};
      bessel_orders(x, lmin > 0 ? lmin - 1 : 0, ltop, xs, nxs, ks);
    }
  } else {
    bessel_orders(k[q] * (tau0 - tau[i]), lmin, ltop, xs, nxs, sink);
  }
}

// Activity of one node on a curved grid: the highest l-tile in which some
// |Phi_l| reaches eps; the node then belongs to the tau-prefix of that tile
// and of every tile below it.
struct ActSink {
  int lmin;
  const int *rowof;
  double eps;
  int ltmax;
  __device__ __forceinline__ void operator()(int l, double v) {
    if (fabs(v) >= eps) {
      const int row = rowof ? rowof[l - lmin] : l - lmin;
      if (row >= 0) ltmax = max(ltmax, row >> 7);
    }
  }
};

__global__ void __launch_bounds__(128) curved_activity_kernel(const double *__restrict__ k,
                                                              const double *__restrict__ tau, double tau0, int ntau,
                                                              int lmin, int lmax, int nlt, double rk, int closed,
                                                              double eps, const int *__restrict__ rowof, int ns,
                                                              int *ext) {
  const int q = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  extern __shared__ double s_stage[];
  if (ns > 0) {
    const double b2 = (k[q] / rk) * (k[q] / rk), sg = closed ? -1.0 : 1.0;
    for (int l = threadIdx.x; l < ns; l += blockDim.x) {
      const double v = fma(sg * (double)l, (double)l, b2);
      const double sv = v > 0.0 ? sqrt(v) : 0.0;
      s_stage[l] = sv;
      s_stage[ns + l] = sv > 0.0 ? 1.0 / sv : 0.0;
    }
    __syncthreads();
  }
  if (i >= ntau) return;
  ActSink a{lmin, rowof, eps, -1};
  hyper_orders(k[q] / rk, rk * (tau0 - tau[i]), closed != 0, lmin, lmax, a, s_stage, s_stage + ns, ns);
  for (int t = 0; t <= a.ltmax && t < nlt; ++t) atomicMax(ext + (size_t)q * nlt + t, i + 1);
}

// Orders of s_l to stage for a curved grid: every order the recurrence can
// reach below l_max (the Miller start is at most l_max + 60 + 8 sqrt(l_max)
// + the open-space tail + 10, and the forward part stops at l_max), if 2 of
// them fit in 160 KB of shared memory; else 0 (computed on the fly).
int curved_stage_orders(const gcamb_grid *g) {
  double chimax = 0.0;
  for (double t : g->tau) chimax = std::max(chimax, g->rk * (g->tau0 - t));
  double extra = 0.0;
  if (g->curved == 1 && chimax > 0.0) {
    const double th = std::tanh(0.5 * chimax);
    extra = th < 1.0 ? std::min(46.0 / -std::log(th), 1e6) : 1e6;
  }
  const double hi = (double)g->lmax;
  const double nsd = hi + 60.0 + 8.0 * std::sqrt(hi) + extra + 16.0;
  if (nsd * 2 * sizeof(double) > 160.0 * 1024) return 0;
  return (int)nsd;
}

// The tau-prefixes of a curved grid, from the activity of every node (run
// once, before the first table is laid out).
int curved_extents(gcamb_grid *g, cudaStream_t st) {
  const size_t n = (size_t)g->nk * g->nlt;
  int *d_ext = nullptr;
  cudaError_t e = cudaMalloc(&d_ext, n * sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "bessel_table: curved extents");
  e = cudaMemsetAsync(d_ext, 0, n * sizeof(int), st);
  if (e == cudaSuccess) {
    dim3 grid((g->ntau + 127) / 128, g->nk);
    const int ns = curved_stage_orders(g);
    const size_t smem = (size_t)2 * ns * sizeof(double);
    if (smem > 48 * 1024)
      e = cudaFuncSetAttribute(curved_activity_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      curved_activity_kernel<<<grid, 128, smem, st>>>(g->d_k, g->d_tau, g->tau0, g->ntau, g->lmin, g->lmax, g->nlt,
                                                      g->rk, g->curved == 2, g->eps_cut,
                                                      g->lsampled ? g->d_rowof : nullptr, ns, d_ext);
      e = cudaGetLastError();
    }
  }
  std::vector<int> h(n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_ext, n * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_ext);
  if (e != cudaSuccess) return cuda_fail(e, "bessel_table: curved extents");
  int64_t act = 0;
  for (int q = 0; q < g->nk; ++q)
    for (int t = 0; t < g->nlt; ++t) {
      const int v = h[(size_t)q * g->nlt + t];
      g->ext[(size_t)q * g->nlt + t] = v;
      act += (int64_t)v * std::min(kTileL, g->nl - t * kTileL);
    }
  g->active = act;  // rows of a tile times its prefix (no per-l cut on curved grids)
  g->ext_ready = true;
  return GCAMB_OK;
}

struct DenseSink {
  double *row;
  __device__ __forceinline__ void operator()(int l, double v) { row[l] = v; }
};

__global__ void sph_bessel_kernel(const double *__restrict__ x, int n, int lmax, const double *__restrict__ xs, int nxs,
                                  double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  DenseSink s{out + (size_t)i * (lmax + 1)};
  bessel_orders(x[i], 0, lmax, xs, nxs, s);
}

// ------------------------------------------------------------------ table memory
//
// Each stored tau-block holds all 128 multipoles of its tile, but a tile's
// upper multipoles have shorter tau-prefixes than its lowest, so the blocks
// beyond them carry rows of zeros (and the 16-bit split formats flush the
// tiny values of the evanescent region, x < l, to zero as well).  Generic
// compression of device memory lets the memory system move such lines
// between DRAM and L2 in compressed form; it is transparent to the kernels.
// The driver's virtual-memory calls are looked up at run time (the library
// links only the CUDA runtime).
namespace {

struct VmmApi {
  CUresult (*dev_get)(CUdevice *, int) = nullptr;
  CUresult (*attr)(int *, CUdevice_attribute, CUdevice) = nullptr;
  CUresult (*gran)(size_t *, const CUmemAllocationProp *, CUmemAllocationGranularity_flags) = nullptr;
  CUresult (*create)(CUmemGenericAllocationHandle *, size_t, const CUmemAllocationProp *, unsigned long long) = nullptr;
  CUresult (*props)(CUmemAllocationProp *, CUmemGenericAllocationHandle) = nullptr;
  CUresult (*reserve)(CUdeviceptr *, size_t, size_t, CUdeviceptr, unsigned long long) = nullptr;
  CUresult (*map)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle, unsigned long long) = nullptr;
  CUresult (*access)(CUdeviceptr, size_t, const CUmemAccessDesc *, size_t) = nullptr;
  CUresult (*unmap)(CUdeviceptr, size_t) = nullptr;
  CUresult (*addr_free)(CUdeviceptr, size_t) = nullptr;
  CUresult (*release)(CUmemGenericAllocationHandle) = nullptr;
  bool ok = false;
};

template <class F>
bool driver_fn(const char *name, F &fn) {
  void *f = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !f) {
    cudaGetLastError();
    return false;
  }
  fn = reinterpret_cast<F>(f);
  return true;
}

const VmmApi &vmm_api() {
  static VmmApi a;
  static std::once_flag once;
  std::call_once(once, [] {
    a.ok = driver_fn("cuDeviceGet", a.dev_get) && driver_fn("cuDeviceGetAttribute", a.attr) &&
           driver_fn("cuMemGetAllocationGranularity", a.gran) &&
           driver_fn("cuMemCreate", a.create) && driver_fn("cuMemGetAllocationPropertiesFromHandle", a.props) &&
           driver_fn("cuMemAddressReserve", a.reserve) && driver_fn("cuMemMap", a.map) &&
           driver_fn("cuMemSetAccess", a.access) && driver_fn("cuMemUnmap", a.unmap) &&
           driver_fn("cuMemAddressFree", a.addr_free) && driver_fn("cuMemRelease", a.release);
  });
  return a;
}

// Compressible memory of `bytes` on the current device, or false (nothing held).
bool vmm_compressed_alloc(Table &t, size_t bytes) {
  const char *env = std::getenv("GCAMB_TABLE_COMPRESS");
  if (env && env[0] == '0') return false;
  const VmmApi &a = vmm_api();
  if (!a.ok) return false;
  int dev = 0, sup = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  CUdevice cudev = 0;
  if (a.dev_get(&cudev, dev) != CUDA_SUCCESS ||
      a.attr(&sup, CU_DEVICE_ATTRIBUTE_GENERIC_COMPRESSION_SUPPORTED, cudev) != CUDA_SUCCESS || !sup)
    return false;
  CUmemAllocationProp prop{};
  prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  prop.location.id = dev;
  prop.allocFlags.compressionType = CU_MEM_ALLOCATION_COMP_GENERIC;
  size_t gran = 0;
  if (a.gran(&gran, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) != CUDA_SUCCESS || gran == 0) return false;
  const size_t sz = (bytes + gran - 1) / gran * gran;
  CUmemGenericAllocationHandle h = 0;
  if (a.create(&h, sz, &prop, 0) != CUDA_SUCCESS) return false;
  CUmemAllocationProp got{};
  bool done = false;
  CUdeviceptr ptr = 0;
  // the driver may grant the memory without compression: then it is not kept
  if (a.props(&got, h) == CUDA_SUCCESS && got.allocFlags.compressionType == CU_MEM_ALLOCATION_COMP_GENERIC &&
      a.reserve(&ptr, sz, 0, 0, 0) == CUDA_SUCCESS) {
    if (a.map(ptr, sz, 0, h, 0) == CUDA_SUCCESS) {
      CUmemAccessDesc acc{};
      acc.location = prop.location;
      acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
      if (a.access(ptr, sz, &acc, 1) == CUDA_SUCCESS) done = true;
      else a.unmap(ptr, sz);
    }
    if (!done) a.addr_free(ptr, sz);
  }
  if (!done) {
    a.release(h);
    return false;
  }
  t.d_data = reinterpret_cast<void *>(ptr);
  t.vmm = (unsigned long long)h;
  t.mapped = sz;
  return true;
}

}  // namespace

int table_alloc(Table &t, size_t bytes) {
  t.vmm = 0;
  t.mapped = 0;
  if (vmm_compressed_alloc(t, bytes)) return GCAMB_OK;
  cudaError_t e = cudaMalloc(&t.d_data, bytes);
  if (e != cudaSuccess) {
    t.d_data = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? fail(GCAMB_ENOMEM, "bessel_table: device allocation")
                                          : cuda_fail(e, "bessel_table: cudaMalloc");
  }
  return GCAMB_OK;
}

void table_free(Table &t) {
  if (t.vmm) {
    const VmmApi &a = vmm_api();
    cudaDeviceSynchronize();  // no kernel may still read the table (cudaFree waits the same way)
    const CUdeviceptr ptr = reinterpret_cast<CUdeviceptr>(t.d_data);
    a.unmap(ptr, t.mapped);
    a.addr_free(ptr, t.mapped);
    a.release((CUmemGenericAllocationHandle)t.vmm);
  } else if (t.d_data) {
    cudaFree(t.d_data);
  }
  t.d_data = nullptr;
  t.vmm = 0;
  t.mapped = 0;
}

int launch_bessel_table(gcamb_grid *g, int mode, cudaStream_t st) {
  Table &t = g->tab[mode];
  const ModeLayout lay = mode_layout(mode);
  if (g->curved && !g->ext_ready) {
    if (int rc = curved_extents(g, st)) return rc;
  }
  if (!t.d_data) {
    t.lay = lay;
    t.nkb.assign((size_t)g->nk * g->nlt, 0);
    t.off.assign((size_t)g->nk * g->nlt, 0);
    int64_t nb = 0;
    for (int q = 0; q < g->nk; ++q)
      for (int lt = 0; lt < g->nlt; ++lt) {
        const size_t e = (size_t)q * g->nlt + lt;
        t.nkb[e] = (g->ext[e] + lay.kb - 1) / lay.kb;
        t.off[e] = nb;
        nb += t.nkb[e];
      }
    t.nblocks = nb;
    if (mode == GCAMB_F16X3) {
      // |j_l| <= 1: scale so that max_i w_i j_l < 2^14, inside fp16's normal range
      double wmax = 0.0;
      for (double w : g->wtau) wmax = w > wmax ? w : wmax;
      int e = 0;
      if (wmax > 0.0) std::frexp(wmax, &e);  // wmax < 2^e
      // kernel grids: |kernel_l| < 4 (t_l <= c_2/15, |e_l|, |b_l| <= 4 max|j|)
      t.scale_exp = wmax > 0.0 ? 14 - e - (g->kernel ? 2 : 0) : 0;
    }
    t.bytes = (size_t)nb * lay.block_bytes();
    if (int rc = table_alloc(t, std::max<size_t>(t.bytes, 256))) return rc;
    cudaError_t e;
    if ((e = cudaMalloc(&t.d_nkb, t.nkb.size() * sizeof(int32_t))) != cudaSuccess) return cuda_fail(e, "bessel_table");
    if ((e = cudaMalloc(&t.d_off, t.off.size() * sizeof(int64_t))) != cudaSuccess) return cuda_fail(e, "bessel_table");
    if ((e = cudaMemcpy(t.d_nkb, t.nkb.data(), t.nkb.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "bessel_table");
    if ((e = cudaMemcpy(t.d_off, t.off.data(), t.off.size() * sizeof(int64_t), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "bessel_table");
  }
  double x_lo = 0.0;
  if (g->kernel && emode_x_lo(g, &x_lo)) return fail(GCAMB_EINVAL, "bessel_table: eps_cut too large for the kernel's limits");
  cudaError_t e = cudaMemsetAsync(t.d_data, 0, t.bytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "bessel_table: memset");
  dim3 grid((g->ntau + 127) / 128, g->nk);
  // curved grids: s_l, 1/s_l staged per block (the block's q)
  const int ns = g->curved ? curved_stage_orders(g) : 0;
  const size_t tsmem = (size_t)2 * ns * sizeof(double);
  if (tsmem > 48 * 1024) {
    switch (mode) {
      case GCAMB_PLAIN64: e = cudaFuncSetAttribute(bessel_table_kernel<GCAMB_PLAIN64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem); break;
      case GCAMB_PLAIN32: e = cudaFuncSetAttribute(bessel_table_kernel<GCAMB_PLAIN32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem); break;
      case GCAMB_BF16X3: e = cudaFuncSetAttribute(bessel_table_kernel<GCAMB_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem); break;
      case GCAMB_F16X3: e = cudaFuncSetAttribute(bessel_table_kernel<GCAMB_F16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem); break;
      default: e = cudaFuncSetAttribute(bessel_table_kernel<GCAMB_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "bessel_table: smem attribute");
  }
  ProfScope prof(GCAMB_K_TABLE, st);
  switch (mode) {
    case GCAMB_PLAIN64:
      bessel_table_kernel<GCAMB_PLAIN64><<<grid, 128, tsmem, st>>>(g->d_k, g->d_tau, g->d_wtau, g->tau0, g->ntau, g->lmin,
                                                               g->lmax, g->nlt, t.d_nkb, t.d_off, g->d_xstart, g->nxs,
                                                               t.scale_exp, g->lsampled ? g->d_lrow : nullptr,
                                                               g->lsampled ? g->d_rowof : nullptr, g->nl, g->curved, g->rk,
                                                               g->kernel, x_lo, ns, t.d_data);
      break;
    case GCAMB_PLAIN32:
      bessel_table_kernel<GCAMB_PLAIN32><<<grid, 128, tsmem, st>>>(g->d_k, g->d_tau, g->d_wtau, g->tau0, g->ntau, g->lmin,
                                                               g->lmax, g->nlt, t.d_nkb, t.d_off, g->d_xstart, g->nxs,
                                                               t.scale_exp, g->lsampled ? g->d_lrow : nullptr,
                                                               g->lsampled ? g->d_rowof : nullptr, g->nl, g->curved, g->rk,
                                                               g->kernel, x_lo, ns, t.d_data);
      break;
    case GCAMB_BF16X3:
      bessel_table_kernel<GCAMB_BF16X3><<<grid, 128, tsmem, st>>>(g->d_k, g->d_tau, g->d_wtau, g->tau0, g->ntau, g->lmin,
                                                              g->lmax, g->nlt, t.d_nkb, t.d_off, g->d_xstart, g->nxs,
                                                              t.scale_exp, g->lsampled ? g->d_lrow : nullptr,
                                                               g->lsampled ? g->d_rowof : nullptr, g->nl, g->curved, g->rk,
                                                               g->kernel, x_lo, ns, t.d_data);
      break;
    case GCAMB_F16X3:
      bessel_table_kernel<GCAMB_F16X3><<<grid, 128, tsmem, st>>>(g->d_k, g->d_tau, g->d_wtau, g->tau0, g->ntau, g->lmin,
                                                             g->lmax, g->nlt, t.d_nkb, t.d_off, g->d_xstart, g->nxs,
                                                             t.scale_exp, g->lsampled ? g->d_lrow : nullptr,
                                                               g->lsampled ? g->d_rowof : nullptr, g->nl, g->curved, g->rk,
                                                               g->kernel, x_lo, ns, t.d_data);
      break;
    case GCAMB_TF32X3:
      bessel_table_kernel<GCAMB_TF32X3><<<grid, 128, tsmem, st>>>(g->d_k, g->d_tau, g->d_wtau, g->tau0, g->ntau, g->lmin,
                                                              g->lmax, g->nlt, t.d_nkb, t.d_off, g->d_xstart, g->nxs,
                                                              t.scale_exp, g->lsampled ? g->d_lrow : nullptr,
                                                               g->lsampled ? g->d_rowof : nullptr, g->nl, g->curved, g->rk,
                                                               g->kernel, x_lo, ns, t.d_data);
      break;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "bessel_table: launch");
  t.built = true;
  return GCAMB_OK;
}

// Start thresholds for the stand-alone entry point: delta = 1e-40, orders up to 24096.
static std::mutex g_xs_mu;
static double *g_xs_dev = nullptr;
static int g_nxs = 0;

int launch_sph_bessel(const double *x, int n, int lmax, double *out, cudaStream_t st) {
  {
    std::lock_guard<std::mutex> lk(g_xs_mu);
    if (!g_xs_dev) {
      const int cap = kMaxL + 4096;
      std::vector<double> xs(cap + 1);
      const double logdelta = std::log(1e-40);
      for (int l = 0; l <= cap; ++l) xs[l] = watson_threshold(l, logdelta);
      double *d = nullptr;
      cudaError_t e = cudaMalloc(&d, xs.size() * sizeof(double));
      if (e != cudaSuccess) return cuda_fail(e, "sph_bessel: cudaMalloc");
      e = cudaMemcpy(d, xs.data(), xs.size() * sizeof(double), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "sph_bessel: upload");
      g_xs_dev = d;
      g_nxs = (int)xs.size();
    }
  }
  cudaError_t e = cudaMemsetAsync(out, 0, (size_t)n * (lmax + 1) * sizeof(double), st);
  if (e != cudaSuccess) return cuda_fail(e, "sph_bessel: memset");
  sph_bessel_kernel<<<(n + 127) / 128, 128, 0, st>>>(x, n, lmax, g_xs_dev, g_nxs, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "sph_bessel: launch");
  return GCAMB_OK;
}

}  // namespace gcamb
