// Batched Eqs. (1)-(2) on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Many sources share one (k, tau) grid, so for each k the tau-sum of Eq. (2)
// for all multipoles and all sources is one dense product
//     D_k[l][m] = sum_i  J_k[l][i] S_k[i][m],   J_k[l][i] = w_i j_l(k (tau0 - tau_i)),
// restricted to the active tau-blocks of each 128-multipole tile (the
// Algorithm 1 window).  Both operands are split into hi + lo parts (bf16 or
// tf32) and D_k accumulates hi*hi + hi*lo + lo*hi in FP32 in tensor memory.
// The epilogue squares D_k, weights it by 4 pi w_k P_m(k) (Eq. 1) and adds it
// to per-thread FP32 sums over a chunk of at most 64 k; the chunk sums are
// added in FP64 in a fixed order by a second kernel.  D_k never leaves the SM.
//
// Work item = (l-tile, source tile, contiguous k-chunk).  One CTA per item:
//   warp 0      bulk-copy producer (table block + split-source block per stage)
//   warp 1      TMEM allocator and single-thread MMA issuer
//   warps 2..9  epilogue: TMEM -> registers, square, weight, accumulate
// Every mbarrier wait is bounded (1 s); a timeout sets the device error flag,
// the CTA drains its own copies and MMAs, frees TMEM and exits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace gcamb {

namespace {

constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kKChunkMax = 64;     // k per work item: bounds the FP32 partial-sum length
constexpr int kABytes = 32768;     // one table block: hi + lo planes of 128 x 128 B
constexpr int kSmemBudget = 196608;

struct TcItem {
  int lt, mt, qb, qe;
};

struct TcParams {
  const char *table;
  const int64_t *off;    // [nk][nlt]
  const int32_t *nkb;    // [nk][nlt]
  const char *sp;        // split sources [nk][n_mt][nkbs] blocks of 256*NT bytes
  const float *wp;       // [nk][mpad] 4 pi w_k P_m(k)
  const TcItem *items;
  float *partial;        // [n_items][NT][128]
  int *err;
  int nlt, n_mt, nkbs, mpad;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait.  abort_flag may be null (teardown drains wait on time only).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err) {
  uint64_t t0 = 0;
  for (uint32_t n = 1;; ++n) {
    if (mbar_try(bar, parity)) return true;
    if (abort_flag && *abort_flag) return false;
    if ((n & 255u) == 0) {
      const uint64_t now = globaltimer();
      if (t0 == 0) t0 = now;
      else if (now - t0 > 1000000000ull) {
        if (abort_flag) *abort_flag = 1;
        if (err) *reinterpret_cast<volatile int *>(err) = kDevErrTimeout;
        return false;
      }
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (SBO), descriptor version 1 (bit 46).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}



// Split modes of the batched path.
enum TcMode { kBF16 = 0, kF16 = 1, kTF32 = 2 };

template <int MODE>
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (MODE == kTF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

template <int W>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[W]) {
  uint32_t r[W];
  if constexpr (W == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  } else {
    static_assert(W == 8, "tmem_ld width");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
  }
#pragma unroll
  for (int j = 0; j < W; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Per k the accumulators are a pair: D_hh (hi*hi) and D_x (hi*lo + lo*hi).
// Keeping the correction products out of D_hh leaves the main chain with a
// third of the accumulate steps (the tensor core's FP32 accumulation error
// grows with their number); D_x is ~2^-8 of D_hh, so its own rounding is
// negligible.  The pairs are double-buffered across k when TMEM allows.
template <int NT>
struct TcCfg {
  static constexpr int kBBytes = 256 * NT;               // hi + lo planes of NT x 128 B
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kStages = (kSmemBudget / kStageBytes) > 4 ? 4 : (kSmemBudget / kStageBytes);
  static constexpr int kNBuf = (4 * NT <= 512) ? 2 : 1;
  static constexpr int kTmemCols = kNBuf * 2 * NT < 32 ? 32 : kNBuf * 2 * NT;
  static constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int kColsPerThread = NT / 2;
  static constexpr int kChunk = NT >= 256 ? 8 : 16;      // TMEM load width (register budget)
};

template <int NT, int MODE>
__global__ void __launch_bounds__(kThreads, 1) los_cl_tc_kernel(TcParams p) {
  using C = TcCfg<NT>;
  constexpr int S = C::kStages;
  constexpr int NB = C::kNBuf;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S * C::kStageBytes);
  // bars: full[S], empty[S], tfull[2], tempty[2], drain
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 5);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * S + 6);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S);
  const uint32_t tfull0 = smem_u32(bars + 2 * S), tempty0 = smem_u32(bars + 2 * S + 2);
  const uint32_t drain = smem_u32(bars + 2 * S + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TcItem it = p.items[blockIdx.x];

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(tfull0, 1);
    mbar_init(tfull0 + 8, 1);
    mbar_init(tempty0, kEpiWarps);
    mbar_init(tempty0 + 8, kEpiWarps);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)C::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int32_t *nkb_row = p.nkb + it.lt;
  const int64_t *off_row = p.off + it.lt;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer
      int stage = 0;
      uint32_t phase = 0;
      int armed_phase[4] = {-1, -1, -1, -1};
      bool ok = true;
      for (int q = it.qb; q < it.qe && ok; ++q) {
        const int nb = nkb_row[(size_t)q * p.nlt];
        const char *a = p.table + (size_t)off_row[(size_t)q * p.nlt] * kABytes;
        const char *b = p.sp + ((size_t)q * p.n_mt + it.mt) * (size_t)p.nkbs * C::kBBytes;
        for (int kb = 0; kb < nb; ++kb) {
          if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort_flag, p.err)) {
            ok = false;
            break;
          }
          const uint32_t sa = smem_u32(smem + stage * C::kStageBytes);
          mbar_expect_tx(full0 + 8 * stage, C::kStageBytes);
          armed_phase[stage] = (int)phase;
          bulk_g2s(sa, a + (size_t)kb * kABytes, kABytes, full0 + 8 * stage);
          bulk_g2s(sa + kABytes, b + (size_t)kb * C::kBBytes, C::kBBytes, full0 + 8 * stage);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // no copy may still be landing when the CTA exits
      for (int s = 0; s < S; ++s)
        if (armed_phase[s] >= 0) mbar_wait(full0 + 8 * s, (uint32_t)armed_phase[s], nullptr, p.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t fmt = MODE == kTF32 ? 2u : (MODE == kBF16 ? 1u : 0u);
      constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NT >> 3) << 17) |
                                 ((uint32_t)(128 >> 4) << 24);
      int stage = 0;
      uint32_t phase = 0;
      int n = 0;
      bool ok = true;
      for (int q = it.qb; q < it.qe && ok; ++q) {
        const int nb = nkb_row[(size_t)q * p.nlt];
        if (nb == 0) continue;
        const int buf = n % NB;
        const uint32_t use = (uint32_t)(n / NB);
        if (!mbar_wait(tempty0 + 8 * buf, (use & 1u) ^ 1u, abort_flag, p.err)) break;
        tc_fence_after();
        const uint32_t dhh = tmem + (uint32_t)(buf * 2 * NT);
        const uint32_t dx = dhh + (uint32_t)NT;
        for (int kb = 0; kb < nb; ++kb) {
          if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, p.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * C::kStageBytes);
          const uint32_t sb = sa + kABytes;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ah = sw128_desc(sa + kk * 32), al = sw128_desc(sa + 16384 + kk * 32);
            const uint64_t bh = sw128_desc(sb + kk * 32), bl = sw128_desc(sb + NT * 128 + kk * 32);
            const uint32_t accum = (kb | kk) ? 1u : 0u;
            mma<MODE>(dhh, ah, bh, idesc, accum);
            mma<MODE>(dx, ah, bl, idesc, accum);
            mma<MODE>(dx, al, bh, idesc, 1u);
          }
          mma_commit(empty0 + 8 * stage);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(tfull0 + 8 * buf);
        ++n;
      }
      // every MMA this thread issued has completed before TMEM is freed
      mma_commit(drain);
      mbar_wait(drain, 0, nullptr, p.err);
    }
  } else {
    // ---------------- epilogue: acc += (sqrt(4 pi w_k P) (D_hh + D_x))^2
    constexpr int CW = C::kChunk;
    const int sp = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = sp * 32 + lane;
    const int col0 = half * C::kColsPerThread;
    float acc[C::kColsPerThread];
#pragma unroll
    for (int j = 0; j < C::kColsPerThread; ++j) acc[j] = 0.f;
    int n = 0;
    for (int q = it.qb; q < it.qe; ++q) {
      const int nb = nkb_row[(size_t)q * p.nlt];
      if (nb == 0) continue;
      const int buf = n % NB;
      const uint32_t use = (uint32_t)(n / NB);
      if (!mbar_wait(tfull0 + 8 * buf, use & 1u, abort_flag, p.err)) break;
      tc_fence_after();
      const float4 *w4 = reinterpret_cast<const float4 *>(p.wp + (size_t)q * p.mpad + it.mt * NT + col0);
      const uint32_t taddr = tmem + ((uint32_t)(sp * 32) << 16) + (uint32_t)(buf * 2 * NT + col0);
#pragma unroll
      for (int c = 0; c < C::kColsPerThread / CW; ++c) {
        float vh[CW], vx[CW];
        tmem_ld<CW>(taddr + c * CW, vh);
        tmem_ld<CW>(taddr + NT + c * CW, vx);
        tmem_wait_ld();
#pragma unroll
        for (int j4 = 0; j4 < CW / 4; ++j4) {
          const float4 w = __ldg(w4 + c * (CW / 4) + j4);
          const float t0 = w.x * (vh[4 * j4 + 0] + vx[4 * j4 + 0]);
          const float t1 = w.y * (vh[4 * j4 + 1] + vx[4 * j4 + 1]);
          const float t2 = w.z * (vh[4 * j4 + 2] + vx[4 * j4 + 2]);
          const float t3 = w.w * (vh[4 * j4 + 3] + vx[4 * j4 + 3]);
          acc[c * CW + 4 * j4 + 0] = fmaf(t0, t0, acc[c * CW + 4 * j4 + 0]);
          acc[c * CW + 4 * j4 + 1] = fmaf(t1, t1, acc[c * CW + 4 * j4 + 1]);
          acc[c * CW + 4 * j4 + 2] = fmaf(t2, t2, acc[c * CW + 4 * j4 + 2]);
          acc[c * CW + 4 * j4 + 3] = fmaf(t3, t3, acc[c * CW + 4 * j4 + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
      ++n;
    }
    float *part = p.partial + (size_t)blockIdx.x * NT * 128;
#pragma unroll
    for (int j = 0; j < C::kColsPerThread; ++j) part[(size_t)(col0 + j) * 128 + row] = acc[j];
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)C::kTmemCols)
                 : "memory");
  }
}

// ------------------------------------------------------------------ prep

__device__ __forceinline__ uint32_t tf32_rna_u(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ uint32_t sw_off(int n, int cbytes) {
  return (uint32_t)n * 128u + ((uint32_t)((cbytes >> 4) ^ (n & 7)) << 4) + (uint32_t)(cbytes & 15);
}

// bf16 / tf32: S[M][nk][ntau] fp32 -> split blocks [q][mt][kb]{hi plane, lo
// plane}; rows = sources (NT per tile), 128-byte swizzled rows of KB tau, zero
// padded.  One thread per element.
template <int MODE>
__global__ void __launch_bounds__(256) split_sources_kernel(const float *__restrict__ S, int M, int nk, int ntau, int NT,
                                                            int n_mt, int nkbs, char *__restrict__ sp) {
  constexpr int KB = MODE == kTF32 ? 32 : 64;
  constexpr int ES = MODE == kTF32 ? 4 : 2;
  constexpr int ROWS = 256 / KB;  // rows per CTA
  const int qm = blockIdx.y;      // q * n_mt + mt
  const int q = qm / n_mt, mt = qm - q * n_mt;
  const int groups = NT / ROWS;
  const int kb = blockIdx.x / groups, rg = blockIdx.x - kb * groups;
  const int c = threadIdx.x % KB;
  const int n = rg * ROWS + threadIdx.x / KB;
  const int m = mt * NT + n;
  const int t = kb * KB + c;
  float v = 0.f;
  if (m < M && t < ntau) v = __ldg(S + ((size_t)m * nk + q) * ntau + t);
  char *blk = sp + (((size_t)qm * nkbs) + kb) * (size_t)(256 * NT);
  const uint32_t o = sw_off(n, c * ES);
  if constexpr (MODE == kTF32) {
    const uint32_t hi = tf32_rna_u(v);
    const uint32_t lo = tf32_rna_u(v - __uint_as_float(hi));
    *reinterpret_cast<uint32_t *>(blk + o) = hi;
    *reinterpret_cast<uint32_t *>(blk + NT * 128 + o) = lo;
  } else {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    *reinterpret_cast<__nv_bfloat16 *>(blk + o) = hi;
    *reinterpret_cast<__nv_bfloat16 *>(blk + NT * 128 + o) = lo;
  }
}

// wq[q][m] = sqrt(4 pi w_k P[m][q]) (zero for padded sources).
__global__ void weights_kernel(const double *__restrict__ Pk, const double *__restrict__ wk, int M, int nk, int mpad,
                               float *__restrict__ wq) {
  const int q = blockIdx.x;
  for (int m = threadIdx.x; m < mpad; m += blockDim.x)
    wq[(size_t)q * mpad + m] =
        m < M ? (float)sqrt(4.0 * 3.14159265358979323846 * wk[q] * Pk[(size_t)m * nk + q]) : 0.f;
}

// fp16: one warp per (k, source) row.  The row is scaled by 2^s so that its
// largest |S| lies in [2^13, 2^14) (fp16 keeps 11 significant bits only in
// its normal range), split into fp16 hi/lo, and written like the bf16 path.
// The weight absorbs the scales: wq = sqrt(4 pi w_k P) 2^-(sJ + s), where
// 2^sJ is the table's scale, so (wq D')^2 is the unscaled contribution.
__global__ void __launch_bounds__(256) split_sources_f16_kernel(const float *__restrict__ S,
                                                                const double *__restrict__ Pk,
                                                                const double *__restrict__ wk, int M, int nk,
                                                                int ntau, int NT, int n_mt, int nkbs, int mpad,
                                                                int sJ, char *__restrict__ sp,
                                                                float *__restrict__ wq) {
  const int lane = threadIdx.x & 31;
  const size_t row = (size_t)blockIdx.x * 8 + (threadIdx.x >> 5);  // q * mpad + m
  if (row >= (size_t)nk * mpad) return;
  const int q = (int)(row / mpad), mfull = (int)(row - (size_t)q * mpad);
  const int mt = mfull / NT, n = mfull - mt * NT;
  const bool live = mfull < M;
  const float *src = S + ((size_t)(live ? mfull : 0) * nk + q) * ntau;
  float mx = 0.f;
  if (live)
    for (int t = lane; t < ntau; t += 32) mx = fmaxf(mx, fabsf(__ldg(src + t)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int s = 0;
  if (mx > 0.f) {
    int e;
    frexpf(mx, &e);  // mx < 2^e
    s = 14 - e;
    s = s < -40 ? -40 : (s > 80 ? 80 : s);
  }
  char *base = sp + ((size_t)(q * n_mt + mt) * nkbs) * (size_t)(256 * NT);
  for (int t = lane; t < nkbs * 64; t += 32) {
    const float v = (live && t < ntau) ? ldexpf(__ldg(src + t), s) : 0.f;
    const __half hi = __float2half_rn(v);
    const __half lo = __float2half_rn(v - __half2float(hi));
    char *blk = base + (size_t)(t >> 6) * (256 * NT);
    const uint32_t o = sw_off(n, (t & 63) * 2);
    *reinterpret_cast<__half *>(blk + o) = hi;
    *reinterpret_cast<__half *>(blk + NT * 128 + o) = lo;
  }
  if (lane == 0)
    wq[row] = live ? (float)ldexp(sqrt(4.0 * 3.14159265358979323846 * wk[q] * Pk[(size_t)mfull * nk + q]), -(sJ + s))
                   : 0.f;
}

// C[m][l] = sum over the tile's items (fixed order) of the FP32 chunk sums, in FP64.
__global__ void __launch_bounds__(128) reduce_kernel(const float *__restrict__ partial, const int *__restrict__ tile_ptr,
                                                     const int *__restrict__ tile_items, int NT, int n_mt, int M,
                                                     int lmin, int lmax, double *__restrict__ Cl) {
  const int r = threadIdx.x;
  const int ml = blockIdx.x;       // source within the tile
  const int tile = blockIdx.y;     // lt * n_mt + mt
  const int lt = tile / n_mt, mt = tile - lt * n_mt;
  const int m = mt * NT + ml;
  const int l = lmin + lt * kTileL + r;
  if (m >= M || l > lmax) return;
  double acc = 0.0;
  for (int e = tile_ptr[tile]; e < tile_ptr[tile + 1]; ++e)
    acc += (double)partial[((size_t)tile_items[e] * NT + ml) * 128 + r];
  Cl[(size_t)m * (lmax - lmin + 1) + (l - lmin)] = acc;
}

// ------------------------------------------------------------------ plan

struct TcPlan {
  int mode = -1, M = 0, NT = 0, n_mt = 0, nkbs = 0, mpad = 0;
  std::vector<TcItem> items;
  std::vector<int> tile_ptr, tile_items;
  TcItem *d_items = nullptr;
  int *d_tile_ptr = nullptr, *d_tile_items = nullptr;
  size_t off_sp = 0, off_wp = 0, off_part = 0, ws_bytes = 0;
};

std::mutex g_plan_mu;
std::vector<std::pair<const gcamb_grid *, TcPlan *>> g_plans;

// Source-tile width: 64 for small batches, else 128 (double-buffered
// accumulator pairs); GCAMB_TC_NT=64|128|256 overrides it.
int pick_nt(int M, int *n_mt) {
  int nt = M <= 64 ? 64 : 128;
  if (const char *e = getenv("GCAMB_TC_NT")) {
    const int v = atoi(e);
    if (v == 64 || v == 128 || v == 256) nt = v;
  }
  *n_mt = (M + nt - 1) / nt;
  return nt;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

void plan_layout(const gcamb_grid *g, int M, int mode, TcPlan &pl) {
  const ModeLayout lay = mode_layout(mode);
  pl.mode = mode;
  pl.M = M;
  pl.NT = pick_nt(M, &pl.n_mt);
  pl.nkbs = (g->ntau + lay.kb - 1) / lay.kb;
  pl.mpad = pl.n_mt * pl.NT;
  const Table &t = g->tab[mode];
  // cost per (q, lt): table blocks + a fixed epilogue share
  double total = 0.0;
  for (size_t e = 0; e < t.nkb.size(); ++e)
    if (t.nkb[e] > 0) total += t.nkb[e] + 0.5;
  total *= pl.n_mt;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const double target = std::max(4.0, total / (sms * 4.0));
  pl.items.clear();
  for (int lt = 0; lt < g->nlt; ++lt)
    for (int mt = 0; mt < pl.n_mt; ++mt) {
      int qb = -1;
      double c = 0.0;
      for (int q = 0; q < g->nk; ++q) {
        const int nb = t.nkb[(size_t)q * g->nlt + lt];
        if (nb == 0) continue;
        if (qb < 0) { qb = q; c = 0.0; }
        c += nb + 0.5;
        if (c >= target || q - qb + 1 >= kKChunkMax) {
          pl.items.push_back({lt, mt, qb, q + 1});
          qb = -1;
        }
      }
      if (qb >= 0) pl.items.push_back({lt, mt, qb, g->nk});
    }
  // launch order: by k position so that tiles sharing source blocks run together
  std::stable_sort(pl.items.begin(), pl.items.end(), [](const TcItem &a, const TcItem &b) {
    return (a.qb + a.qe) > (b.qb + b.qe);
  });
  const int ntile = g->nlt * pl.n_mt;
  pl.tile_ptr.assign(ntile + 1, 0);
  for (const auto &x : pl.items) pl.tile_ptr[x.lt * pl.n_mt + x.mt + 1]++;
  for (int i = 0; i < ntile; ++i) pl.tile_ptr[i + 1] += pl.tile_ptr[i];
  pl.tile_items.assign(pl.items.size(), 0);
  {
    std::vector<int> fill(pl.tile_ptr.begin(), pl.tile_ptr.end() - 1);
    // fixed order inside a tile: increasing k
    std::vector<int> idx(pl.items.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return pl.items[a].qb < pl.items[b].qb; });
    for (int i : idx) {
      const auto &x = pl.items[i];
      pl.tile_items[fill[x.lt * pl.n_mt + x.mt]++] = i;
    }
  }
  const size_t sp_bytes = (size_t)g->nk * pl.n_mt * pl.nkbs * 256 * pl.NT;
  const size_t wp_bytes = (size_t)g->nk * pl.mpad * sizeof(float);
  const size_t part_bytes = std::max<size_t>(1, pl.items.size()) * pl.NT * 128 * sizeof(float);
  pl.off_sp = 0;
  pl.off_wp = align256(sp_bytes);
  pl.off_part = pl.off_wp + align256(wp_bytes);
  pl.ws_bytes = pl.off_part + align256(part_bytes);
}

TcPlan *get_plan(const gcamb_grid *g, int M, int mode, int *rc) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  int nmt = 0;
  const int nt = pick_nt(M, &nmt);
  for (auto &e : g_plans)
    if (e.first == g && e.second->M == M && e.second->mode == mode && e.second->NT == nt) return e.second;
  TcPlan *pl = new TcPlan();
  plan_layout(g, M, mode, *pl);
  cudaError_t e1 = cudaMalloc(&pl->d_items, std::max<size_t>(1, pl->items.size()) * sizeof(TcItem));
  cudaError_t e2 = cudaMalloc(&pl->d_tile_ptr, pl->tile_ptr.size() * sizeof(int));
  cudaError_t e3 = cudaMalloc(&pl->d_tile_items, std::max<size_t>(1, pl->tile_items.size()) * sizeof(int));
  if (e1 || e2 || e3) {
    *rc = cuda_fail(e1 ? e1 : (e2 ? e2 : e3), "los_cl: plan allocation");
    delete pl;
    return nullptr;
  }
  cudaMemcpy(pl->d_items, pl->items.data(), pl->items.size() * sizeof(TcItem), cudaMemcpyHostToDevice);
  cudaMemcpy(pl->d_tile_ptr, pl->tile_ptr.data(), pl->tile_ptr.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaError_t e4 = cudaMemcpy(pl->d_tile_items, pl->tile_items.data(), pl->tile_items.size() * sizeof(int),
                              cudaMemcpyHostToDevice);
  if (e4) {
    *rc = cuda_fail(e4, "los_cl: plan upload");
    return nullptr;
  }
  g_plans.push_back({g, pl});
  return pl;
}

template <int NT, int MODE>
int launch_tc(const gcamb_grid *g, const TcPlan &pl, const float *S, const double *Pk, double *Cl, char *ws,
              cudaStream_t st, int *err_word = nullptr, bool use_err_word = false) {
  using Cfg = TcCfg<NT>;
  const Table &t = g->tab[pl.mode];
  char *sp = ws + pl.off_sp;
  float *wp = reinterpret_cast<float *>(ws + pl.off_wp);
  float *part = reinterpret_cast<float *>(ws + pl.off_part);
  if constexpr (MODE == kF16) {
    const size_t rows = (size_t)g->nk * pl.mpad;
    ProfScope prof(GCAMB_K_SPLIT, st);
    split_sources_f16_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
        S, Pk, g->d_wk, pl.M, g->nk, g->ntau, NT, pl.n_mt, pl.nkbs, pl.mpad, t.scale_exp, sp, wp);
  } else {
    {
      constexpr int KB = MODE == kTF32 ? 32 : 64;
      dim3 grid(pl.nkbs * (NT / (256 / KB)), g->nk * pl.n_mt);
      ProfScope prof(GCAMB_K_SPLIT, st);
      split_sources_kernel<MODE><<<grid, 256, 0, st>>>(S, pl.M, g->nk, g->ntau, NT, pl.n_mt, pl.nkbs, sp);
    }
    ProfScope prof(GCAMB_K_WEIGHTS, st);
    weights_kernel<<<g->nk, 256, 0, st>>>(Pk, g->d_wk, pl.M, g->nk, pl.mpad, wp);
  }
  if (!pl.items.empty()) {
    cudaError_t e = cudaFuncSetAttribute(los_cl_tc_kernel<NT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg::kSmemBytes);
    if (e != cudaSuccess) return cuda_fail(e, "los_cl: smem attribute");
    TcParams prm{static_cast<const char *>(t.d_data), t.d_off, t.d_nkb, sp, wp, pl.d_items, part,
                 use_err_word ? err_word : device_error_flag(), g->nlt, pl.n_mt, pl.nkbs, pl.mpad};
    if (!prm.err && !use_err_word) return fail(GCAMB_ECUDA, "los_cl: error flag allocation");
    ProfScope prof(GCAMB_K_TC, st);
    los_cl_tc_kernel<NT, MODE><<<(unsigned)pl.items.size(), kThreads, Cfg::kSmemBytes, st>>>(prm);
  }
  dim3 rgrid(NT, g->nlt * pl.n_mt);
  ProfScope prof(GCAMB_K_REDUCE, st);
  reduce_kernel<<<rgrid, 128, 0, st>>>(part, pl.d_tile_ptr, pl.d_tile_items, NT, pl.n_mt, pl.M, g->lmin, g->lmax, Cl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "los_cl: launch");
  return GCAMB_OK;
}

template <int MODE>
int launch_mode(const gcamb_grid *g, const TcPlan &pl, const float *S, const double *Pk, double *Cl, char *w,
                cudaStream_t st, int *err_word = nullptr, bool use_err_word = false) {
  switch (pl.NT) {
    case 64: return launch_tc<64, MODE>(g, pl, S, Pk, Cl, w, st, err_word, use_err_word);
    case 128: return launch_tc<128, MODE>(g, pl, S, Pk, Cl, w, st, err_word, use_err_word);
    default: return launch_tc<256, MODE>(g, pl, S, Pk, Cl, w, st, err_word, use_err_word);
  }
}

}  // namespace

size_t los_cl_workspace_bytes(const gcamb_grid *g, int M, int mode) {
  if (!g->tab[mode].built) {
    // without the table: an upper bound from the extents
    TcPlan tmp;
    tmp.NT = pick_nt(M, &tmp.n_mt);
    const ModeLayout lay = mode_layout(mode);
    tmp.nkbs = (g->ntau + lay.kb - 1) / lay.kb;
    tmp.mpad = tmp.n_mt * tmp.NT;
    size_t sp_bytes = (size_t)g->nk * tmp.n_mt * tmp.nkbs * 256 * tmp.NT;
    size_t wp_bytes = (size_t)g->nk * tmp.mpad * sizeof(float);
    size_t max_items = (size_t)g->nk * g->nlt * tmp.n_mt;
    return align256(sp_bytes) + align256(wp_bytes) + align256(max_items * tmp.NT * 128 * sizeof(float));
  }
  int rc = 0;
  TcPlan *p = get_plan(g, M, mode, &rc);
  return p ? p->ws_bytes : 0;
}

int launch_los_cl(const gcamb_grid *g, const float *S, const double *Pk, int M, int mode, double *Cl, void *ws,
                  size_t ws_bytes, cudaStream_t st) {
  int rc = 0;
  TcPlan *pl = get_plan(g, M, mode, &rc);
  if (!pl) return rc ? rc : fail(GCAMB_ECUDA, "los_cl: plan");
  if (ws_bytes < pl->ws_bytes) return fail(GCAMB_EINVAL, "los_cl: workspace too small");
  char *w = static_cast<char *>(ws);
  switch (mode) {
    case GCAMB_TF32X3: return launch_mode<kTF32>(g, *pl, S, Pk, Cl, w, st);
    case GCAMB_F16X3: return launch_mode<kF16>(g, *pl, S, Pk, Cl, w, st);
    default: return launch_mode<kBF16>(g, *pl, S, Pk, Cl, w, st);
  }
}

// Fixed-buffer variant for gcamb_los_cl_noalloc: the plan is computed on the
// host and its arrays, the split sources, the weights and the chunk partials
// all live in the caller's buffer `scratch` (no device allocation).
size_t los_cl_fixed_bytes(const gcamb_grid *g, int M, int mode) {
  TcPlan pl;
  plan_layout(g, M, mode, pl);
  return align256(pl.items.size() * sizeof(TcItem)) + align256(pl.tile_ptr.size() * sizeof(int)) +
         align256(pl.tile_items.size() * sizeof(int)) + pl.ws_bytes;
}

int launch_los_cl_fixed(const gcamb_grid *g, const float *S, const double *Pk, int M, int mode, double *Cl,
                        char *scratch, size_t cap, int *status, cudaStream_t st) {
  TcPlan pl;
  plan_layout(g, M, mode, pl);
  const size_t b_items = align256(pl.items.size() * sizeof(TcItem));
  const size_t b_ptr = align256(pl.tile_ptr.size() * sizeof(int));
  const size_t b_ti = align256(pl.tile_items.size() * sizeof(int));
  const size_t need = b_items + b_ptr + b_ti + pl.ws_bytes;
  if (need > cap)
    return fail(GCAMB_EINVAL, "los_cl_noalloc: needs " + std::to_string(need) + " bytes of scratch, the fixed buffer holds " +
                                  std::to_string(cap) + "; use gcamb_los_cl with a caller workspace");
  pl.d_items = reinterpret_cast<TcItem *>(scratch);
  pl.d_tile_ptr = reinterpret_cast<int *>(scratch + b_items);
  pl.d_tile_items = reinterpret_cast<int *>(scratch + b_items + b_ptr);
  char *ws = scratch + b_items + b_ptr + b_ti;
  cudaError_t e = cudaSuccess;
  if (!pl.items.empty())
    e = cudaMemcpyAsync(pl.d_items, pl.items.data(), pl.items.size() * sizeof(TcItem), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pl.d_tile_ptr, pl.tile_ptr.data(), pl.tile_ptr.size() * sizeof(int), cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess && !pl.tile_items.empty())
    e = cudaMemcpyAsync(pl.d_tile_items, pl.tile_items.data(), pl.tile_items.size() * sizeof(int),
                        cudaMemcpyHostToDevice, st);
  // copies from pageable memory return once the host data is staged, so the
  // vectors may go out of scope when this function returns
  if (e != cudaSuccess) return cuda_fail(e, "los_cl_noalloc: plan upload");
  int rc;
  switch (mode) {
    case GCAMB_TF32X3: rc = launch_mode<kTF32>(g, pl, S, Pk, Cl, ws, st, status, true); break;
    case GCAMB_F16X3: rc = launch_mode<kF16>(g, pl, S, Pk, Cl, ws, st, status, true); break;
    default: rc = launch_mode<kBF16>(g, pl, S, Pk, Cl, ws, st, status, true); break;
  }
  return rc;
}

void drop_plans(const gcamb_grid *g) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  for (auto it = g_plans.begin(); it != g_plans.end();) {
    if (it->first == g) {
      cudaFree(it->second->d_items);
      cudaFree(it->second->d_tile_ptr);
      cudaFree(it->second->d_tile_items);
      delete it->second;
      it = g_plans.erase(it);
    } else {
      ++it;
    }
  }
}

}  // namespace gcamb
