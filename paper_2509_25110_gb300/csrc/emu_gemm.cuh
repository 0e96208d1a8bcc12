// Small tcgen05 GEMM for the emulator network.
//
//   C[M][N] = op(A)[M][K] . op(B)[N][K]^T   (+ fused epilogue)
//
// Both operands are fp32 tensors in global memory read through a strided
// view (element (i, k) at p[row(i) * rs + k * cs], row(i) = rows ? rows[i] :
// i) and rounded to bf16 by the loaders, which write them straight into the
// 128-byte swizzled K-major layout the tensor cores read.  One CTA (4 warps)
// per 128 x 128 tile of C, K in chunks of 64, two shared-memory buffers: the
// threads fill one while the single issuing thread's MMAs (M = 128, N = 128,
// K = 16, bf16 x bf16 -> FP32 in TMEM) drain the other.  Every wait is
// bounded; a timeout sets the device error flag and the CTA frees its TMEM.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "mbar.cuh"

namespace gcamb {
namespace emu {

struct View {
  const float *p;
  long long rs, cs;  // element strides of rows (i) and of the contraction index (k)
  const int *rows;   // optional row gather
  int R, K;          // valid extents (rows, contraction); zero beyond
};

enum Epi { kStore = 0, kBias = 1, kBiasGelu = 2, kDGelu = 3 };

struct GemmArgs {
  View A, B;
  int M, N, K;
  float *C;        // [M][ldc]
  long long ldc;
  float *CT;       // optional transposed copy: CT[n * ldct + i] (kBiasGelu: of H)
  long long ldct;
  int kchunks;     // K-chunks (of 64) per CTA along grid z; the z-th CTA writes C + z * M * ldc
  const float *bias;   // kBias, kBiasGelu: [N]
  float *H;            // kBiasGelu: GELU(C) also written here, [M][ldc]
  const float *Zprev;  // kDGelu: C *= GELU'(Zprev), [M][ldc]
  int *err;
};

__device__ __forceinline__ uint64_t e_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Fills a 128 x 64 bf16 tile (rows i0.., contraction k0..) of a view.
__device__ __forceinline__ void load_tile(const View &v, int i0, int k0, unsigned char *tile) {
  const int tid = threadIdx.x;
  if (v.cs == 1 && v.rs != 1) {
    // contraction index contiguous: one row per thread, eight 8-element chunks,
    // 16-byte loads where the row and the chunk allow
    const int i = i0 + tid;
    const bool ok_row = i < v.R;
    const float *src = ok_row ? v.p + (long long)(v.rows ? v.rows[i] : i) * v.rs : v.p;
    const bool vec = ok_row && (v.rs % 4 == 0) && ((reinterpret_cast<uintptr_t>(v.p) & 15) == 0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int kc = k0 + c * 8;
      float f[8];
      if (vec && kc + 8 <= v.K) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(src + kc));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(src + kc + 4));
        f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
        f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) f[u] = (ok_row && kc + u < v.K) ? __ldg(src + kc + u) : 0.f;
      }
      uint32_t w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * u], f[2 * u + 1]);
        w[u] = *reinterpret_cast<const uint32_t *>(&h);
      }
      const uint32_t o = (uint32_t)tid * 128u + ((uint32_t)(c ^ (tid & 7)) << 4);
      *reinterpret_cast<uint4 *>(tile + o) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    // rows contiguous (or general): consecutive threads take consecutive rows
    for (int e = tid; e < 128 * 64; e += 128) {
      const int r = e & 127, kk = e >> 7;
      const int i = i0 + r, k = k0 + kk;
      float a = 0.f;
      if (i < v.R && k < v.K) a = __ldg(v.p + (long long)(v.rows ? v.rows[i] : i) * v.rs + (long long)k * v.cs);
      const uint32_t o = (uint32_t)r * 128u + ((uint32_t)(((kk * 2) >> 4) ^ (r & 7)) << 4) + (uint32_t)((kk * 2) & 15);
      *reinterpret_cast<__nv_bfloat16 *>(tile + o) = __float2bfloat16_rn(a);
    }
  }
}

template <int EPI>
__global__ void __launch_bounds__(128, 1) gemm_kernel(GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // [buf0: A 16 KB | B 16 KB][buf1: A | B][barriers]
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 65536);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3);
  const uint32_t done0 = smem_u32(bars), fin = smem_u32(bars + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * 128, n0 = blockIdx.y * 128;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done0 + 8) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fin) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
  const int nkc_all = (a.K + 63) / 64;
  const int kc0 = a.kchunks > 0 ? blockIdx.z * a.kchunks : 0;
  const int kc1 = a.kchunks > 0 ? min(nkc_all, kc0 + a.kchunks) : nkc_all;
  const int nkc = kc1 > kc0 ? kc1 - kc0 : 0;
  float *Cout = a.C + (a.kchunks > 0 ? (long long)blockIdx.z * a.M * a.ldc : 0);
  bool ok = true;
  for (int kc = 0; kc < nkc && ok; ++kc) {
    const int buf = kc & 1;
    bool w = true;
    if (kc >= 2) w = mbar_wait(done0 + 8 * buf, (uint32_t)((kc - 2) >> 1) & 1u, nullptr, a.err);
    // every thread takes the same branch (no thread may be left at a barrier)
    if (!__syncthreads_and(w)) {
      ok = false;
      break;
    }
    unsigned char *ta = smem + buf * 32768, *tb = ta + 16384;
    load_tile(a.A, i0, (kc0 + kc) * 64, ta);
    load_tile(a.B, n0, (kc0 + kc) * 64, tb);
    // generic-proxy stores -> visible to the tensor cores (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(ta), sb = smem_u32(tb);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t da = e_desc(sa + kk * 32), db = e_desc(sb + kk * 32);
        const uint32_t acc = (kc | kk) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done0 + 8 * buf)
                   : "memory");
    }
  }
  // all MMAs done (also on the error path, before TMEM is freed)
  if (threadIdx.x == 0)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(fin) : "memory");
  const bool fin_ok = mbar_wait(fin, 0, nullptr, a.err);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && fin_ok) {
    const int i = i0 + warp * 32 + lane;
    const bool zero = nkc == 0;  // an empty K range contributes zero
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (i < a.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c * 16 + j;
          if (n >= a.N) break;
          float v = zero ? 0.f : __uint_as_float(r[j]);
          const long long o = (long long)i * a.ldc + n;
          if constexpr (EPI == kBias || EPI == kBiasGelu) v += a.bias[n];
          if constexpr (EPI == kDGelu) v *= gelu_grad_f(a.Zprev[o]);
          Cout[o] = v;
          if constexpr (EPI == kBiasGelu) {
            const float hv = gelu_f(v);
            a.H[o] = hv;
            if (a.CT) a.CT[(long long)n * a.ldct + i] = hv;
          } else {
            if (a.CT) a.CT[(long long)n * a.ldct + i] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
  }
}

constexpr int kGemmSmem = 65536 + 1024 + 256;

}  // namespace emu
}  // namespace gcamb
