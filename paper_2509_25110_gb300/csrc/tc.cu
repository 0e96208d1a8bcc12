// Batched Eqs. (1)-(2) on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Many sources share one (k, tau) grid, so for each k the tau-sum of Eq. (2)
// for all multipoles and all sources is one dense product
//     D_k[l][m] = sum_i  J_k[l][i] S_k[i][m],   J_k[l][i] = w_i j_l(k (tau0 - tau_i)),
// restricted to the active tau-blocks of each 128-multipole tile (the
// Algorithm 1 window).  Both operands are split into hi + lo parts (bf16 or
// tf32) and D_k accumulates hi*hi + hi*lo + lo*hi in FP32 in tensor memory.
// The epilogue squares D_k, weights it by 4 pi w_k P_m(k) (Eq. 1) and adds it
// to per-thread FP32 sums over a chunk of at most 16 k (each chunk sum of
// n <= 16 positive terms is within (n - 1) 2^-24 of their exact sum); a second
// kernel adds the chunk sums in a fixed order (TwoSum pairs, read out in
// FP64).  D_k never leaves the SM.
//
// Work item = (l-tile, source tile, contiguous k-chunk); with LP = 2 (fused
// uniform batches) two adjacent l-tiles that share each source block.  One
// persistent CTA per SM takes items from a counter:
//   warp 0      producer: bulk copy of the table block(s) and of the source
//               block per stage (split sources, or FP32 sources by TMA when fused)
//   warp 1      TMEM allocator and single-thread MMA issuer
//   (LP = 2: warps 2, 3 idle, so that every role is whole warpgroups)
//   4 warps     (fused only) converters: FP32 source tile -> hi/lo planes in
//               place, in the swizzled operand layout
//   the rest    8 epilogue warps per tile: TMEM -> registers, square, weight,
//               accumulate
// Every mbarrier wait is bounded (1 s); a timeout sets the device error flag,
// the CTA drains its own copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "mbar.cuh"

namespace gcamb {

namespace {

constexpr int kEpiWarps = 8;
constexpr int kConvWarps = 4;
constexpr int kKChunkMax = 64;     // k per work item
constexpr int kKSub = 16;          // records (k) per FP32 chunk sum: each item's sums are flushed to
                                   // their own partial every kKSub records (GCAMB_TC_KSUB overrides it)
constexpr int kSmemBudget = 196608;

// Work item: first l-tile, source tile, k range [qb, qe), and its number of
// l-tiles (LP = 2 plans: 2, or 1 where the source tile's l_max stops before
// the second tile or no tile follows); pbase: its first partial slot (one
// slot per chunk of ksub non-empty k, each holding LP tiles' sums); chain:
// (LP = 2 plans) an item of l-tile 0 alone whose hi*hi sum is spread over
// three accumulators (see the MMA warp).
struct TcItem {
  int lt, mt, qb, qe, ntl, pbase, chain, pad;
};

struct TcParams {
  const char *table;
  const char *table2;    // pair: the second field's table (same layout)
  const int64_t *off;    // [nk][nlt]
  const int32_t *nkb;    // [nk][nlt]
  const char *sp;        // split sources [nk][n_mt][nkbs] blocks of 256*NT bytes
  const float *wp;       // [nk][mpad] sqrt(4 pi w_k P_m(k))
  const float *sc;       // fused F16X3: [nk][mpad] power-of-two row scales of the sources;
                         // TE: [nk][mpad] small-x tail of Delta_E at l = 2
  const float *ix2;      // TE: [nk][nkbs * 32] 1/x^2 of each node (0 below the small-x cut and beyond ntau)
  int r2;                // TE: row of l = 2 in the first l-tile, or -1
  const TcItem *items;
  int *counter;          // next item to hand out (zeroed before each launch)
  int nitems;
  int ksub;              // non-empty k per FP32 chunk sum (partial slot)
  int chain_free;        // LP = 2: a k at which the item's second tile has no blocks is a chain record
  float *partial;        // [n_slots * LP][NT][128] (TE: [n_slots][3 NT/2][128])
  int *err;
  int nlt, n_mt, nkbs, mpad;
};

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Named barrier 1 over the converter warps; returns the AND of every
// converter thread's `ok`, so that all of them leave their loops together.
__device__ __forceinline__ bool conv_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)ok), "n"(kConvWarps * 32)
      : "memory");
  return r != 0;
}

// 3-D tiled TMA load (x innermost) into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 8-row groups `sbo` bytes
// apart, swizzle `layout` (2: 128-byte, 4: 64-byte), descriptor version 1
// (bit 46).
__device__ __forceinline__ uint64_t op_desc(uint32_t saddr, uint32_t sbo, uint64_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(sbo >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;
  d |= layout << 61;
  return d;
}



// Split modes of the batched path.
enum TcMode { kBF16 = 0, kF16 = 1, kTF32 = 2 };

// Operand geometry of a split mode: a tau-block is 32 nodes; its operand rows
// are 64 bytes (bf16, fp16; 64-byte swizzle) or 128 bytes (tf32; 128-byte
// swizzle); one K step of the MMA covers 32 bytes of a row.
template <int MODE>
struct TcGeom {
  static constexpr int kRowB = MODE == kTF32 ? 128 : 64;
  static constexpr int kKSteps = kRowB / 32;
  static constexpr int kPlaneA = 128 * kRowB;          // one plane of a table block
  static constexpr int kABytes = 2 * kPlaneA;          // table block: hi + lo planes
  static constexpr uint32_t kSbo = 8 * kRowB;
  static constexpr uint64_t kLayout = MODE == kTF32 ? 2 : 4;
  __device__ static __forceinline__ uint64_t desc(uint32_t saddr) { return op_desc(saddr, kSbo, kLayout); }
};

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
  } else if constexpr (W == 2) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
  } else if constexpr (W == 4) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
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
//
// LP = 2: an item covers two adjacent l-tiles; a stage holds the table block
// of each and one source block, which both multiply (the sources are loaded
// and split once for the two tiles).  Each tile has its own accumulator pair
// and barriers; 16 epilogue warps, 8 per tile.
template <int NT, int MODE, int NA = 1, int LP = 1>
struct TcCfg {
  static constexpr int kABytes = TcGeom<MODE>::kABytes;
  static constexpr int kBBytes = 2 * NT * TcGeom<MODE>::kRowB;  // hi + lo planes of NT rows
  static constexpr int kStageBytes = NA * kABytes + kBBytes;     // NA table blocks (pair, LP = 2: 2)
  static constexpr int kStages = (kSmemBudget / kStageBytes) > 8 ? 8 : (kSmemBudget / kStageBytes);
  static constexpr int kNBuf = (LP * 4 * NT <= 512) ? 2 : 1;
  static constexpr int kTB = kNBuf * LP;                 // accumulator pairs (TMEM) and their barrier pairs
  static constexpr int kTmemCols = kTB * 2 * NT < 32 ? 32 : kTB * 2 * NT;
  static constexpr int kKSlots = 4;                      // per-k records in flight
  static constexpr int kSlotBytes = 16 + 8 * NT;         // header, weights, row scales
  static constexpr int kQBytes = kKChunkMax * 12 * LP;   // the item's block counts and offsets
  static constexpr int kFBytes = kStages * 128;          // TE: 1/x^2 of each stage's 32 nodes
  static constexpr int kSmemBytes =
      kStages * kStageBytes + kFBytes + kKSlots * kSlotBytes + kQBytes + 1024 /*align*/ + 512 /*barriers*/;
  static constexpr int kColsPerThread = NT / 2;
  // TMEM load width (register budget: 22 warps leave 88 registers a thread)
  static constexpr int kChunk = NT >= 128 ? (LP == 2 ? 4 : 8) : 16;
};

// Warp roles.  LP = 2 keeps each role in whole warpgroups (warps 2, 3 idle)
// so that the warpgroups can trade registers: launched at 80 a thread (24
// warps), the producer/MMA warpgroup drops to 40, the converter warpgroup to
// 56, and the four epilogue warpgroups take 96 (4 x 40 + 4 x 56 + 16 x 96 =
// 24 x 80).
template <bool FUSED, int TE = 0, int LP = 1>
struct TcRoles {
  static constexpr int kConv = FUSED ? kConvWarps : 0;
  static constexpr int kConv0 = (LP == 2 && FUSED) ? 4 : 2;  // first converter warp (or epilogue warp)
  static constexpr int kEpi0 = kConv0 + kConv;    // first epilogue warp
  static constexpr int kEpi = kEpiWarps * LP;
  static constexpr int kThreadsT = 32 * (kEpi0 + kEpi);
  // LP = 2 split (launched at 80 a thread): producer/MMA warpgroup, converter
  // warpgroup, four epilogue warpgroups: 4 x 40 + 4 x 56 + 16 x 96 = 24 x 80
  static constexpr int kRegCtl = 40, kRegConv = 56, kRegHigh = 96;
};

// Per-k record, written by the producer into a ring in shared memory:
// header {q, nb, item, mt | flags}, then the epilogue weights of the k for
// the item's source tile (bulk copy) and, fused fp16 only, the sources' row
// scales; TE: the NT/2 models' weights and small-x tails.  nb < 0 ends the
// work.  kL2: the item's l-tile is the first (it may hold l = 2).
constexpr int kFirst = 1 << 16, kLast = 1 << 17, kL2 = 1 << 18;
// LP = 2, chain record (the item's first l-tile only at this k): its hi*hi
// products go round-robin by tau-block into three accumulators (the tile's
// own D_hh and the other tile's pair), its corrections into the tile's D_x
// (see the MMA warp).
constexpr int kChain = 1 << 19;

// TE = 2 (pair): two fields X, Y of kernel grids with the same layout (for
// instance the tensor T and E kernels): each stage holds a block of both
// tables; the X rows are multiplied by the first, the Y rows by the second
// (six MMAs of N = NT/2 per K step), into the TMEM layout of TE = 1, and the
// sources are split without scaling.  The epilogue is that of TE = 1.
//
// TE = 1 (temperature and E-mode together, fused bf16 only): a source tile holds
// NT/2 models, their FP32 temperature sources in operand rows 0 .. NT/2-1 and
// their polarisation sources in rows NT/2 .. NT-1 (one TMA box from each).
// The converters scale the E rows by 1/x^2 (0 below the small-x cut), so
// that the shared table of w_i j_l gives D_E' = sum_i w_i j_l S_P / x^2; the
// epilogue adds the l = 2 small-x tail and accumulates, per model,
// (w D_T)^2, (w D_E')^2 and w^2 D_T D_E'; the reduce applies c_l^2 and c_l.
template <int NT, int MODE, bool FUSED, int TE = 0, int LP = 1>
__global__ void __launch_bounds__(TcRoles<FUSED, TE, LP>::kThreadsT, 1)
    los_cl_tc_kernel(const __grid_constant__ CUtensorMap tm_src, const __grid_constant__ CUtensorMap tm_src2,
                     TcParams p) {
  static_assert(!TE || (FUSED && MODE == kBF16 && NT <= 128), "TE: fused bf16, NT <= 128");
  static_assert(LP == 1 || (LP == 2 && !TE && MODE != kTF32 && NT <= 128), "LP = 2: bf16/fp16 without TE, NT <= 128");
  using C = TcCfg<NT, MODE, (TE == 2 || LP == 2) ? 2 : 1, LP>;
  using G = TcGeom<MODE>;
  using R = TcRoles<FUSED, TE, LP>;
  constexpr int S = C::kStages;
  constexpr int NB = C::kNBuf;
  constexpr int TB = C::kTB;
  constexpr int KS = C::kKSlots;
  constexpr bool kScale = FUSED && MODE == kF16;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *fbuf = smem + S * C::kStageBytes;  // TE: [S][32] floats
  unsigned char *kslots = fbuf + C::kFBytes;
  int64_t *q_off = reinterpret_cast<int64_t *>(kslots + KS * C::kSlotBytes);  // [LP][kKChunkMax]
  int32_t *q_nb = reinterpret_cast<int32_t *>(q_off + LP * kKChunkMax);      // [LP][kKChunkMax]
  uint64_t *bars = reinterpret_cast<uint64_t *>(kslots + KS * C::kSlotBytes + C::kQBytes);
  // bars: full[S], empty[S], conv[S], kfull[KS], kempty[KS], tfull[TB],
  //       tempty[TB], drain, (tmem slot), (abort), src[S]; accumulator pair
  //       buf * LP + tile sits at TMEM column (buf * LP + tile) * 2 NT.
  // Fused kernels: a stage's source box (and TE's 1/x^2) completes on src,
  // its table blocks on full, so that the converters split the sources while
  // the table blocks are still landing; the MMA waits for conv and full.
  uint64_t *b1 = bars + 3 * S + 2 * KS;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(b1 + 2 * TB + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(b1 + 2 * TB + 2);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S), conv0 = smem_u32(bars + 2 * S);
  const uint32_t kfull0 = smem_u32(bars + 3 * S), kempty0 = smem_u32(bars + 3 * S + KS);
  const uint32_t tfull0 = smem_u32(b1), tempty0 = smem_u32(b1 + TB);
  const uint32_t drain = smem_u32(b1 + 2 * TB);
  const uint32_t src0 = smem_u32(b1 + 2 * TB + 3);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
      mbar_init(conv0 + 8 * s, R::kConv > 0 ? R::kConv : 1);
      if (FUSED) mbar_init(src0 + 8 * s, 1);
    }
    for (int s = 0; s < KS; ++s) {
      mbar_init(kfull0 + 8 * s, 1);
      mbar_init(kempty0 + 8 * s, 1 + R::kEpi + R::kConv);
    }
    for (int b = 0; b < TB; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      // the 8 epilogue warps of the accumulator pair's tile (LP = 2: two
      // arrivals each, or one from each of the 16 warps on a chain item)
      mbar_init(tempty0 + 8 * b, LP == 2 ? 2 * kEpiWarps : kEpiWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (FUSED && threadIdx.x == 32)
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_src)) : "memory");
  if (TE && threadIdx.x == 33)
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_src2)) : "memory");
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

  // Roles.  Each register change sits in its warpgroups' own branch, so that
  // the code it covers is compiled to its budget.
  // producer (warp 0) and MMA issuer (warp 1)
  auto control_role = [&]() {
    if (warp == 0) {
      // ---------------- producer: items from the counter; the whole warp loads
      // the item's block counts and table offsets into shared memory (one
      // round trip per item), then lane 0 writes per non-empty k a record and
      // issues the k's table and source blocks into the stage ring
      int stage = 0;
      uint32_t phase = 0;
      int armed_phase[S];
#pragma unroll
      for (int s = 0; s < S; ++s) armed_phase[s] = -1;
      int ks = 0;
      uint32_t kph = 0;
      int karmed[C::kKSlots];
#pragma unroll
      for (int s = 0; s < KS; ++s) karmed[s] = -1;
      bool ok = true;
      while (ok) {
        int item = 0;
        if (lane == 0) item = atomicAdd(p.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= p.nitems) break;
        const TcItem it = p.items[item];
        const int cnt = min(it.qe - it.qb, kKChunkMax);  // the plan keeps items within kKChunkMax k
        for (int j = lane; j < cnt; j += 32) {
          const size_t e = (size_t)(it.qb + j) * p.nlt + it.lt;
          q_nb[j] = p.nkb[e];
          q_off[j] = p.off[e];
          if constexpr (LP == 2) {  // the pair's second tile (none past the last)
            const bool has2 = it.ntl == 2;
            q_nb[kKChunkMax + j] = has2 ? p.nkb[e + 1] : 0;
            q_off[kKChunkMax + j] = has2 ? p.off[e + 1] : 0;
          }
        }
        __syncwarp();
        if (lane == 0) {
          int rc = 0;  // records of this item so far: chunk rc / ksub, slot pbase + rc / ksub
          for (int j = 0; j < cnt && ok; ++j) {
            const int q = it.qb + j;
            const int nb0 = q_nb[j];
            const int nb1 = LP == 2 ? q_nb[kKChunkMax + j] : 0;
            const int nb = max(nb0, nb1);
            if (nb == 0) continue;
            // the k's record
            if (!mbar_wait(kempty0 + 8 * ks, kph ^ 1u, abort_flag, p.err)) {
              ok = false;
              break;
            }
            unsigned char *rec = kslots + ks * C::kSlotBytes;
            volatile int *hdr = reinterpret_cast<volatile int *>(rec);
            hdr[0] = q;
            hdr[1] = LP == 2 ? (nb0 | (nb1 << 16)) : nb;  // LP = 2: both tiles' block counts (< 2^15 each)
            hdr[2] = it.pbase + rc / p.ksub;                // the chunk's partial slot
            const int rs = rc % p.ksub;
            hdr[3] = it.mt | (rs == 0 ? kFirst : 0) | ((rs == p.ksub - 1 || q == it.qe - 1) ? kLast : 0) |
                     (TE && it.lt == 0 ? kL2 : 0) |
                     (LP == 2 && (it.chain || (p.chain_free && nb1 == 0)) ? kChain : 0);
            ++rc;
            const uint32_t kb_bar = kfull0 + 8 * ks;
            karmed[ks] = (int)kph;
            if constexpr (TE) {
              // NT/2 models: weights, then the l = 2 tails
              mbar_expect_tx(kb_bar, NT * 4);
              const size_t wrow = (size_t)q * p.mpad + (size_t)it.mt * (NT / 2);
              bulk_g2s(smem_u32(rec + 16), p.wp + wrow, NT * 2, kb_bar);
              bulk_g2s(smem_u32(rec + 16 + NT * 2), p.sc + wrow, NT * 2, kb_bar);
            } else {
              mbar_expect_tx(kb_bar, (kScale ? 2 : 1) * NT * 4);
              const size_t wrow = (size_t)q * p.mpad + (size_t)it.mt * NT;
              bulk_g2s(smem_u32(rec + 16), p.wp + wrow, NT * 4, kb_bar);
              if constexpr (kScale) bulk_g2s(smem_u32(rec + 16 + NT * 4), p.sc + wrow, NT * 4, kb_bar);
            }
            if (++ks == KS) {
              ks = 0;
              kph ^= 1u;
            }
            const char *a = p.table + (size_t)q_off[j] * C::kABytes;
            const char *b = FUSED ? nullptr : p.sp + ((size_t)q * p.n_mt + it.mt) * (size_t)p.nkbs * C::kBBytes;
            for (int kb = 0; kb < nb; ++kb) {
              if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort_flag, p.err)) {
                ok = false;
                break;
              }
              const uint32_t sa = smem_u32(smem + stage * C::kStageBytes);
              armed_phase[stage] = (int)phase;
              if constexpr (LP == 2) {
                // the tiles' blocks while each has some, and the source block (fused: the
                // source box first, on its own barrier, which the converters wait for alone)
                const bool u0 = kb < nb0, u1 = kb < nb1;
                const uint32_t tb = (u0 ? C::kABytes : 0) + (u1 ? C::kABytes : 0);
                if constexpr (FUSED) {
                  mbar_expect_tx(src0 + 8 * stage, C::kBBytes);
                  tma_load_3d(sa + 2 * C::kABytes, &tm_src, kb * 32, q, it.mt * NT, src0 + 8 * stage);
                  mbar_expect_tx(full0 + 8 * stage, tb);
                } else {
                  mbar_expect_tx(full0 + 8 * stage, tb + C::kBBytes);
                }
                if (u0) bulk_g2s(sa, a + (size_t)kb * C::kABytes, C::kABytes, full0 + 8 * stage);
                if (u1)
                  bulk_g2s(sa + C::kABytes, p.table + ((size_t)q_off[kKChunkMax + j] + kb) * C::kABytes, C::kABytes,
                           full0 + 8 * stage);
                if constexpr (!FUSED)  // split sources: evict first, so that L2 keeps the table blocks the other
                                       // source tiles' items read next (uneven 1000-source batch: 16.56 -> 16.35 ms
                                       // per step)
                  bulk_g2s_hint(sa + 2 * C::kABytes, b + (size_t)kb * C::kBBytes, C::kBBytes, full0 + 8 * stage,
                                l2_policy_evict_first());
                if (++stage == S) {
                  stage = 0;
                  phase ^= 1u;
                }
                continue;
              }
              constexpr uint32_t kTabBytes = (TE == 2 ? 2 : 1) * C::kABytes;
              // fused: the source box (and TE's 1/x^2) on src, the table blocks on full
              const uint32_t sbar = FUSED ? src0 + 8 * stage : full0 + 8 * stage;
              if constexpr (FUSED) {
                mbar_expect_tx(sbar, C::kBBytes + (TE == 1 ? 128 : 0));
                mbar_expect_tx(full0 + 8 * stage, kTabBytes);
              } else {
                mbar_expect_tx(full0 + 8 * stage, C::kStageBytes);
              }
              bulk_g2s(sa, a + (size_t)kb * C::kABytes, C::kABytes, full0 + 8 * stage);
              if constexpr (TE == 2)  // the second field's table block
                bulk_g2s(sa + C::kABytes, p.table2 + (size_t)q_off[j] * C::kABytes + (size_t)kb * C::kABytes,
                         C::kABytes, full0 + 8 * stage);
              if constexpr (TE == 1)  // the block's 32 values of 1/x^2
                bulk_g2s(smem_u32(fbuf + stage * 128), p.ix2 + ((size_t)q * p.nkbs + kb) * 32, 128, sbar);
              constexpr int kBOff = (TE == 2 ? 2 : 1) * C::kABytes;  // the source region of the stage
              if constexpr (TE) {  // FP32 boxes [NT/2 models][1 k][32 tau] of the two fields
                tma_load_3d(sa + kBOff, &tm_src, kb * 32, q, it.mt * (NT / 2), sbar);
                tma_load_3d(sa + kBOff + (NT / 2) * 128, &tm_src2, kb * 32, q, it.mt * (NT / 2), sbar);
              } else if constexpr (FUSED)  // FP32 box [NT sources][1 k][32 tau]; zero beyond ntau and M
                tma_load_3d(sa + kBOff, &tm_src, kb * 32, q, it.mt * NT, sbar);
              else
                bulk_g2s(sa + kBOff, b + (size_t)kb * C::kBBytes, C::kBBytes, full0 + 8 * stage);
              if (++stage == S) {
                stage = 0;
                phase ^= 1u;
              }
            }
          }
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;  // also orders lane 0's reads before the next item's writes
      }
      if (lane == 0) {
        // end-of-work record (no copies)
        if (ok && mbar_wait(kempty0 + 8 * ks, kph ^ 1u, abort_flag, p.err)) {
          reinterpret_cast<volatile int *>(kslots + ks * C::kSlotBytes)[1] = -1;
          mbar_arrive(kfull0 + 8 * ks);
          karmed[ks] = (int)kph;  // this phase completes now; the drain below must not wait for a later one
        }
        // no copy may still be landing when the CTA exits
        for (int s = 0; s < S; ++s)
          if (armed_phase[s] >= 0) {
            mbar_wait(full0 + 8 * s, (uint32_t)armed_phase[s], nullptr, p.err);
            if (FUSED) mbar_wait(src0 + 8 * s, (uint32_t)armed_phase[s], nullptr, p.err);
          }
        for (int s = 0; s < KS; ++s)
          if (karmed[s] >= 0) mbar_wait(kfull0 + 8 * s, (uint32_t)karmed[s], nullptr, p.err);
      }
    } else if (warp == 1) {
      if (lane == 0) {
        // ---------------- MMA issuer
        constexpr uint32_t fmt = MODE == kTF32 ? 2u : (MODE == kBF16 ? 1u : 0u);
        constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NT >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);
        // With NT <= 128 the hi and lo source planes are one operand of 2 NT
        // rows and D_hh, D_x adjacent TMEM columns, so hi*hi and hi*lo are one
        // MMA of N = 2 NT: each K step reads A_hi once (shared-memory bandwidth
        // bounds these MMAs).
        constexpr bool kPair = 2 * NT <= 256;
        constexpr uint32_t idesc2 = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)((2 * NT) >> 3) << 17) |
                                    ((uint32_t)(128 >> 4) << 24);
        int stage = 0;
        uint32_t phase = 0;
        int n = 0;
        int ks = 0;
        uint32_t kph = 0;
        int nt2[2] = {0, 0};  // LP = 2: k's accumulated so far per tile
        while (true) {
          if (!mbar_wait(kfull0 + 8 * ks, kph, abort_flag, p.err)) break;
          const int hv = reinterpret_cast<volatile int *>(kslots + ks * C::kSlotBytes)[1];
          if (hv < 0) break;
          const int hfl = reinterpret_cast<volatile int *>(kslots + ks * C::kSlotBytes)[3];
          mbar_arrive(kempty0 + 8 * ks);
          if (++ks == KS) {
            ks = 0;
            kph ^= 1u;
          }
          if constexpr (LP == 2) {
            // per tile: its block count, its accumulator pair (waited for just
            // before the tile's first MMA of this k)
            const int nbt[2] = {hv & 0xFFFF, hv >> 16};
            const int nb = max(nbt[0], nbt[1]);
            uint32_t dt[2];
            int bt[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              bt[t] = (nt2[t] % NB) * LP + t;
              dt[t] = tmem + (uint32_t)(bt[t] * 2 * NT);
            }
            bool ok = true;
            if (hfl & kChain) {
              // Chain record (the item's first tile only: the second has no
              // blocks at this k, or the item is l-tile 0 alone).  The tensor cores add each MMA's
              // products to the FP32 accumulator after dropping their bits
              // below a quarter ulp of the largest term and truncate the sum,
              // so every accumulate step loses a little relative to the running
              // sum.  Three accumulators that each take every third tau-block
              // hold about a third of the sum each, which cuts the loss to
              // about a third.  D_hh of block kb: kb % 3 == 0 -> this tile's
              // D_hh (with its D_x, one N = 2 NT MMA), 1 -> the other pair's
              // D_hh, 2 -> the other pair's D_x; every correction goes to this
              // tile's D_x.  Both pairs are waited for (empty) and committed
              // (full); the epilogue reads the chains that received a block.
#pragma unroll
              for (int t = 0; t < 2; ++t)
                if (ok && !mbar_wait(tempty0 + 8 * bt[t], ((uint32_t)(nt2[t] / NB) & 1u) ^ 1u, abort_flag, p.err))
                  ok = false;
              if (!ok) break;
              tc_fence_after();
              const uint32_t dx0 = dt[0] + (uint32_t)NT;
              for (int kb = 0; kb < nbt[0] && ok; ++kb) {
                if ((FUSED && !mbar_wait(conv0 + 8 * stage, phase, abort_flag, p.err)) ||
                    !mbar_wait(full0 + 8 * stage, phase, abort_flag, p.err)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + stage * C::kStageBytes);
                const uint32_t sb = sa + 2 * C::kABytes;
                const int c = kb % 3;
                const uint32_t dhh = c == 0 ? dt[0] : (c == 1 ? dt[1] : dt[1] + (uint32_t)NT);
#pragma unroll
                for (int kk = 0; kk < G::kKSteps; ++kk) {
                  const uint64_t ah = G::desc(sa + kk * 32), al = G::desc(sa + G::kPlaneA + kk * 32);
                  const uint64_t bh = G::desc(sb + kk * 32), bl = G::desc(sb + NT * G::kRowB + kk * 32);
                  if (c == 0) {
                    mma<MODE>(dhh, ah, bh, idesc2, (kb | kk) ? 1u : 0u);  // [D_hh | D_x] (+)= A_hi [B_hi | B_lo]
                  } else {
                    mma<MODE>(dhh, ah, bh, idesc, (kb > c || kk) ? 1u : 0u);  // first written at kb == c
                    mma<MODE>(dx0, ah, bl, idesc, 1u);
                  }
                  mma<MODE>(dx0, al, bh, idesc, 1u);
                }
                mma_commit(empty0 + 8 * stage);
                if (++stage == S) {
                  stage = 0;
                  phase ^= 1u;
                }
              }
              if (!ok) break;
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                mma_commit(tfull0 + 8 * bt[t]);
                ++nt2[t];
              }
              continue;
            }
            for (int kb = 0; kb < nb && ok; ++kb) {
              if ((FUSED && !mbar_wait(conv0 + 8 * stage, phase, abort_flag, p.err)) ||
                  !mbar_wait(full0 + 8 * stage, phase, abort_flag, p.err)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + stage * C::kStageBytes);
              const uint32_t sb = sa + 2 * C::kABytes;
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                if (kb >= nbt[t]) continue;
                if (kb == 0) {
                  if (!mbar_wait(tempty0 + 8 * bt[t], ((uint32_t)(nt2[t] / NB) & 1u) ^ 1u, abort_flag, p.err)) {
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                }
                const uint32_t at = sa + t * C::kABytes;
#pragma unroll
                for (int kk = 0; kk < G::kKSteps; ++kk) {
                  const uint64_t ah = G::desc(at + kk * 32), al = G::desc(at + G::kPlaneA + kk * 32);
                  const uint64_t bh = G::desc(sb + kk * 32);
                  const uint32_t accum = (kb | kk) ? 1u : 0u;
                  mma<MODE>(dt[t], ah, bh, idesc2, accum);  // [D_hh | D_x] (+)= A_hi [B_hi | B_lo]
                  mma<MODE>(dt[t] + NT, al, bh, idesc, 1u);
                }
              }
              if (!ok) break;
              mma_commit(empty0 + 8 * stage);
              if (++stage == S) {
                stage = 0;
                phase ^= 1u;
              }
            }
            if (!ok) break;
#pragma unroll
            for (int t = 0; t < 2; ++t)
              if (nbt[t] > 0) {
                mma_commit(tfull0 + 8 * bt[t]);
                ++nt2[t];
              }
            continue;
          }
          const int nb = hv;
          const int buf = n % NB;
          const uint32_t use = (uint32_t)(n / NB);
          if (!mbar_wait(tempty0 + 8 * buf, (use & 1u) ^ 1u, abort_flag, p.err)) break;
          tc_fence_after();
          const uint32_t dhh = tmem + (uint32_t)(buf * 2 * NT);
          const uint32_t dx = dhh + (uint32_t)NT;
          bool ok = true;
          for (int kb = 0; kb < nb; ++kb) {
            if ((FUSED && !mbar_wait(conv0 + 8 * stage, phase, abort_flag, p.err)) ||
                !mbar_wait(full0 + 8 * stage, phase, abort_flag, p.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + stage * C::kStageBytes);
            const uint32_t sb = sa + (TE == 2 ? 2 : 1) * C::kABytes;
#pragma unroll
            for (int kk = 0; kk < G::kKSteps; ++kk) {
              const uint64_t ah = G::desc(sa + kk * 32), al = G::desc(sa + G::kPlaneA + kk * 32);
              const uint64_t bh = G::desc(sb + kk * 32), bl = G::desc(sb + NT * G::kRowB + kk * 32);
              const uint32_t accum = (kb | kk) ? 1u : 0u;
              if constexpr (TE == 2) {
                // X rows [0, NT/2) times table 1, Y rows [NT/2, NT) times table 2;
                // row NT/2 starts on a whole 8-row swizzle atom
                constexpr int H = NT / 2;
                constexpr uint32_t idescH = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(H >> 3) << 17) |
                                            ((uint32_t)(128 >> 4) << 24);
                const uint32_t sa2 = sa + C::kABytes;
                const uint64_t ah2 = G::desc(sa2 + kk * 32), al2 = G::desc(sa2 + G::kPlaneA + kk * 32);
                const uint64_t bhY = G::desc(sb + H * G::kRowB + kk * 32);
                const uint64_t blY = G::desc(sb + NT * G::kRowB + H * G::kRowB + kk * 32);
                mma<MODE>(dhh, ah, bh, idescH, accum);       // D_X hh
                mma<MODE>(dhh + H, ah2, bhY, idescH, accum);  // D_Y hh
                mma<MODE>(dx, ah, bl, idescH, accum);        // D_X x
                mma<MODE>(dx, al, bh, idescH, 1u);
                mma<MODE>(dx + H, ah2, blY, idescH, accum);  // D_Y x
                mma<MODE>(dx + H, al2, bhY, idescH, 1u);
                continue;
              }
              if constexpr (kPair) {
                mma<MODE>(dhh, ah, bh, idesc2, accum);  // [D_hh | D_x] (+)= A_hi [B_hi | B_lo]
              } else {
                mma<MODE>(dhh, ah, bh, idesc, accum);
                mma<MODE>(dx, ah, bl, idesc, accum);
              }
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
    }
  };
  // converters (fused only)
  auto convert_role = [&]() {
      // ---------------- converters: the stage's FP32 tile [NT][32] becomes the
      // hi and lo planes [NT][64 B] (64-byte swizzle) in the same bytes.  Thread
      // ct owns float4 column c4 of rows r0 + 16 j; every row it writes has the
      // same (row / 2) mod 4, hence one swizzle offset.  All reads precede all
      // writes (conv_all is the barrier between them).
      if constexpr (FUSED) {
        constexpr int RJ = NT / 16;
        const int ct = threadIdx.x - 32 * R::kConv0;
        const int c4 = ct & 7, r0 = ct >> 3;
        const uint32_t swz = ((uint32_t)(((c4 >> 1) ^ ((r0 >> 1) & 3)) << 4)) | ((uint32_t)(c4 & 1) << 3);
        int stage = 0;
        uint32_t phase = 0;
        int ks = 0;
        uint32_t kph = 0;
        while (true) {
          const bool w = mbar_wait(kfull0 + 8 * ks, kph, abort_flag, p.err);
          const unsigned char *rec = kslots + ks * C::kSlotBytes;
          int nb = w ? reinterpret_cast<const volatile int *>(rec)[1] : -1;
          if (!conv_all(w) || nb < 0) break;
          if constexpr (LP == 2) nb = max(nb & 0xFFFF, nb >> 16);  // stages of the k: the longer tile's
          float scl[RJ];
          if constexpr (MODE == kF16) {
            const float *sr = reinterpret_cast<const float *>(rec + 16 + NT * 4) + r0;
#pragma unroll
            for (int j = 0; j < RJ; ++j) scl[j] = sr[16 * j];
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(kempty0 + 8 * ks);
          if (++ks == KS) {
            ks = 0;
            kph ^= 1u;
          }
          bool ok = true;
          for (int kb = 0; kb < nb; ++kb) {
            const bool w2 = mbar_wait(src0 + 8 * stage, phase, abort_flag, p.err);  // the source box alone
            unsigned char *sb = smem + stage * C::kStageBytes + ((TE == 2 || LP == 2) ? 2 : 1) * C::kABytes;
            const float4 *raw = reinterpret_cast<const float4 *>(sb);
            float4 v[RJ];
#pragma unroll
            for (int j = 0; j < RJ; ++j) v[j] = raw[ct + 128 * j];
            // TE: 1/x^2 of this thread's four tau nodes (copied with the stage)
            float4 f = make_float4(1.f, 1.f, 1.f, 1.f);
            if constexpr (TE == 1) f = reinterpret_cast<const float4 *>(fbuf + stage * 128)[c4];
            if (!conv_all(w2)) {
              ok = false;
              break;
            }
#pragma unroll
            for (int j = 0; j < RJ; ++j) {
              float x0 = v[j].x, x1 = v[j].y, x2 = v[j].z, x3 = v[j].w;
              if constexpr (TE == 1) {
                if (j >= RJ / 2) {  // rows NT/2 .. NT-1: polarisation sources
                  x0 *= f.x;
                  x1 *= f.y;
                  x2 *= f.z;
                  x3 *= f.w;
                }
              }
              uint2 hi, lo;
              if constexpr (MODE == kF16) {
                x0 *= scl[j];
                x1 *= scl[j];
                x2 *= scl[j];
                x3 *= scl[j];
                const __half2 h01 = __floats2half2_rn(x0, x1), h23 = __floats2half2_rn(x2, x3);
                const __half2 l01 = __floats2half2_rn(x0 - __low2float(h01), x1 - __high2float(h01));
                const __half2 l23 = __floats2half2_rn(x2 - __low2float(h23), x3 - __high2float(h23));
                hi = make_uint2(*reinterpret_cast<const uint32_t *>(&h01), *reinterpret_cast<const uint32_t *>(&h23));
                lo = make_uint2(*reinterpret_cast<const uint32_t *>(&l01), *reinterpret_cast<const uint32_t *>(&l23));
              } else {
                const __nv_bfloat162 h01 = __floats2bfloat162_rn(x0, x1), h23 = __floats2bfloat162_rn(x2, x3);
                const __nv_bfloat162 l01 = __floats2bfloat162_rn(x0 - __low2float(h01), x1 - __high2float(h01));
                const __nv_bfloat162 l23 = __floats2bfloat162_rn(x2 - __low2float(h23), x3 - __high2float(h23));
                hi = make_uint2(*reinterpret_cast<const uint32_t *>(&h01), *reinterpret_cast<const uint32_t *>(&h23));
                lo = make_uint2(*reinterpret_cast<const uint32_t *>(&l01), *reinterpret_cast<const uint32_t *>(&l23));
              }
              const uint32_t o = (uint32_t)(r0 + 16 * j) * 64u + swz;
              *reinterpret_cast<uint2 *>(sb + o) = hi;
              *reinterpret_cast<uint2 *>(sb + NT * 64 + o) = lo;
            }
            // generic-proxy stores, read next by the tensor cores
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(conv0 + 8 * stage);
            if (++stage == S) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
        }
      }
  };
  if (warp < R::kEpi0) {
    if constexpr (LP == 2 && FUSED) {
      // LP = 2: warps 2, 3 have no role; the producer/MMA warpgroup and the
      // converter warpgroup each drop to their own budget
      static_assert(R::kThreadsT == 768 && R::kEpi0 == 8 && R::kConv0 == 4, "LP = 2 register split: 6 warpgroups");
      if (warp >= R::kConv0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(R::kRegConv));
        convert_role();
      } else {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(R::kRegCtl));
        control_role();
      }
    } else {
      if (warp < R::kConv0) control_role();
      else if (FUSED) convert_role();
    }
  } else {
    if constexpr (LP == 2 && FUSED) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(R::kRegHigh));
    if constexpr (TE) {
      // ---------------- epilogue (TE): per model j of the thread's quarter,
      // t = w (D_T), e = w (D_E' + tail at l = 2); tt += t^2, ee += e^2, te += t e
      constexpr int H = NT / 2, MPT = H / 2;
      constexpr int CWE = NT >= 128 ? 4 : 8;  // TMEM load width (register budget)
      const int sp = warp & 3;
      const int half = (warp - R::kEpi0) >> 2;
      const int row = sp * 32 + lane;
      const int j0 = half * MPT;
      float att[MPT], aee[MPT], ate[MPT];
#pragma unroll
      for (int j = 0; j < MPT; ++j) att[j] = aee[j] = ate[j] = 0.f;
      int n = 0;
      int ks = 0;
      uint32_t kph = 0;
      while (true) {
        if (!mbar_wait(kfull0 + 8 * ks, kph, abort_flag, p.err)) break;
        const unsigned char *rec = kslots + ks * C::kSlotBytes;
        const volatile int *hdr = reinterpret_cast<const volatile int *>(rec);
        const int nb = hdr[1];
        if (nb < 0) break;
        const int item = hdr[2], flags = hdr[3];  // item: the chunk's partial slot
        const int buf = n % NB;
        const uint32_t use = (uint32_t)(n / NB);
        if (!mbar_wait(tfull0 + 8 * buf, use & 1u, abort_flag, p.err)) break;
        tc_fence_after();
        if (flags & kFirst) {
#pragma unroll
          for (int j = 0; j < MPT; ++j) att[j] = aee[j] = ate[j] = 0.f;
        }
        const float *wr = reinterpret_cast<const float *>(rec + 16);
        const float *cr = wr + H;
        // the small-x tail at l = 2: lane r2 of the first l-tile only
        const float cm = ((flags & kL2) && row == p.r2) ? 1.f : 0.f;
        const uint32_t taddr = tmem + ((uint32_t)(sp * 32) << 16) + (uint32_t)(buf * 2 * NT);
#pragma unroll
        for (int c = 0; c < MPT / CWE; ++c) {
          const int jc = j0 + c * CWE;
          float th[CWE], tx[CWE], eh[CWE], ex[CWE];
          tmem_ld<CWE>(taddr + jc, th);
          tmem_ld<CWE>(taddr + NT + jc, tx);
          tmem_ld<CWE>(taddr + H + jc, eh);
          tmem_ld<CWE>(taddr + NT + H + jc, ex);
          tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < CWE; ++u) {
            const float w = wr[jc + u];
            const float t = w * (th[u] + tx[u]);
            const float e = w * fmaf(cm, cr[jc + u], eh[u] + ex[u]);
            att[c * CWE + u] = fmaf(t, t, att[c * CWE + u]);
            aee[c * CWE + u] = fmaf(e, e, aee[c * CWE + u]);
            ate[c * CWE + u] = fmaf(t, e, ate[c * CWE + u]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(tempty0 + 8 * buf);
          mbar_arrive(kempty0 + 8 * ks);
        }
        if (++ks == KS) {
          ks = 0;
          kph ^= 1u;
        }
        ++n;
        if (flags & kLast) {
          float *part = p.partial + (size_t)item * 3 * H * 128;
#pragma unroll
          for (int j = 0; j < MPT; ++j) {
            part[(size_t)(j0 + j) * 128 + row] = att[j];
            part[(size_t)(H + j0 + j) * 128 + row] = aee[j];
            part[(size_t)(2 * H + j0 + j) * 128 + row] = ate[j];
          }
        }
      }
    } else {
      // ---------------- epilogue: acc += (sqrt(4 pi w_k P) (D_hh + D_x))^2
      // (LP = 2: warps 8 t .. 8 t + 7 of the epilogue serve tile t; on a
      // chain record tile 0's D_hh is the sum of three accumulators)
      constexpr int CW = C::kChunk;
      constexpr int CWC = 2;  // chain records: TMEM load width (four accumulators per column)
      const int sp = warp & 3;  // a warp reads the TMEM lanes 32 (warp mod 4) .. + 31
      const int grp = (warp - R::kEpi0) >> 2;
      const int half = grp & 1, tile = grp >> 1;
      const int row = sp * 32 + lane;
      const int col0 = half * C::kColsPerThread;
      float acc[C::kColsPerThread];
#pragma unroll
      for (int j = 0; j < C::kColsPerThread; ++j) acc[j] = 0.f;
      int nu[2] = {0, 0};  // uses so far of each tile's accumulator pair (LP = 1: tile 0 only)
      int ks = 0;
      uint32_t kph = 0;
      while (true) {
        if (!mbar_wait(kfull0 + 8 * ks, kph, abort_flag, p.err)) break;
        const unsigned char *rec = kslots + ks * C::kSlotBytes;
        const volatile int *hdr = reinterpret_cast<const volatile int *>(rec);
        const int hv = hdr[1];
        if (hv < 0) break;
        const int item = hdr[2], flags = hdr[3];  // item: the chunk's partial slot
        if (flags & kFirst) {
#pragma unroll
          for (int j = 0; j < C::kColsPerThread; ++j) acc[j] = 0.f;
        }
        const bool chain = LP == 2 && (flags & kChain);
        if (chain) {
          // chain record: tile 0's warps read both pairs (tile 0's D_hh and
          // D_x, and the chains 1, 2 in the other pair) for their usual
          // columns; a chain that took no block (fewer than three blocks) is
          // read but not added (its columns hold whatever they held).  Tile
          // 1's warps follow the other pair's phase and release it with them.
          const int nb0 = hv & 0xFFFF;
          int btc[2];
#pragma unroll
          for (int t = 0; t < 2; ++t) btc[t] = (nu[t] % NB) * LP + t;
          if (!mbar_wait(tfull0 + 8 * btc[tile], (uint32_t)(nu[tile] / NB) & 1u, abort_flag, p.err)) break;
          if (tile == 0) {
            tc_fence_after();
            const float *wr = reinterpret_cast<const float *>(rec + 16) + col0;
            const uint32_t ta0 = tmem + ((uint32_t)(sp * 32) << 16) + (uint32_t)(btc[0] * 2 * NT + col0);
            const uint32_t d1 = (uint32_t)((btc[1] - btc[0]) * 2 * NT);
            const bool u1 = nb0 > 1, u2 = nb0 > 2;
            // D_hh = (h0 + h1) + h2, in three load rounds of CWC columns (loading all four
            // accumulators before one wait measured 1% slower over the launch)
#pragma unroll
            for (int c = 0; c < C::kColsPerThread / CWC; ++c) {
              const uint32_t ta = ta0 + c * CWC;
              float x[CWC], y[CWC];
              tmem_ld<CWC>(ta, x);
              tmem_ld<CWC>(ta + d1, y);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < CWC; ++j) x[j] = u1 ? x[j] + y[j] : x[j];
              tmem_ld<CWC>(ta + NT + d1, y);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < CWC; ++j) x[j] = u2 ? x[j] + y[j] : x[j];
              tmem_ld<CWC>(ta + NT, y);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < CWC; ++j) {
                const float t = wr[c * CWC + j] * (x[j] + y[j]);
                acc[c * CWC + j] = fmaf(t, t, acc[c * CWC + j]);
              }
            }
            tc_fence_before();
          }
          __syncwarp();
          // 16 arrivals each: tile 0's pair two from each tile-0 warp, the
          // other pair one from each of the 16 warps
          if (lane == 0) {
            if (tile == 0) mbar_arrive_n(tempty0 + 8 * btc[0], 2u);
            mbar_arrive(tempty0 + 8 * btc[1]);
          }
          ++nu[0];
          ++nu[1];
        }
        // this tile's blocks at this k (LP = 2: none when only the other tile has some)
        const int nbt = chain ? 0 : (LP == 2 ? ((hv >> (16 * tile)) & 0xFFFF) : hv);
        if constexpr (LP == 2) {  // the other tile's pair (its use count; its warps consume it)
          if (!chain && ((hv >> (16 * (tile ^ 1))) & 0xFFFF) > 0) ++nu[tile ^ 1];
        }
        if (nbt > 0) {
          const int bt = (nu[tile] % NB) * LP + tile;
          const uint32_t use = (uint32_t)(nu[tile] / NB);
          if (!mbar_wait(tfull0 + 8 * bt, use & 1u, abort_flag, p.err)) break;
          tc_fence_after();
          const float4 *w4 = reinterpret_cast<const float4 *>(rec + 16) + col0 / 4;
          const uint32_t taddr = tmem + ((uint32_t)(sp * 32) << 16) + (uint32_t)(bt * 2 * NT + col0);
#pragma unroll
          for (int c = 0; c < C::kColsPerThread / CW; ++c) {
            float vh[CW], vx[CW];
            tmem_ld<CW>(taddr + c * CW, vh);
            tmem_ld<CW>(taddr + NT + c * CW, vx);
            tmem_wait_ld();
#pragma unroll
            for (int j4 = 0; j4 < CW / 4; ++j4) {
              const float4 w = w4[c * (CW / 4) + j4];
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
          // LP = 2: the barrier counts 16 arrivals (all 16 warps on a chain item)
          if (lane == 0) mbar_arrive_n(tempty0 + 8 * bt, LP == 2 ? 2u : 1u);
          ++nu[tile];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(kempty0 + 8 * ks);
        if (++ks == KS) {
          ks = 0;
          kph ^= 1u;
        }
        if (flags & kLast) {
          // k-chunk sums of (chunk slot, tile): partial index slot * LP + tile
          float *part = p.partial + ((size_t)item * LP + tile) * NT * 128;
#pragma unroll
          for (int j = 0; j < C::kColsPerThread; ++j) part[(size_t)(col0 + j) * 128 + row] = acc[j];
        }
      }
    }
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

// Byte offset of (row n, byte c) in a plane of the mode's operand rows, in
// its swizzled order (64-byte rows: chunk XOR (n / 2) % 4; 128-byte rows:
// chunk XOR n % 8).
template <int MODE>
__device__ __forceinline__ uint32_t sw_off(int n, int cbytes) {
  if constexpr (TcGeom<MODE>::kRowB == 64)
    return (uint32_t)n * 64u + ((uint32_t)((cbytes >> 4) ^ ((n >> 1) & 3)) << 4) + (uint32_t)(cbytes & 15);
  else
    return (uint32_t)n * 128u + ((uint32_t)((cbytes >> 4) ^ (n & 7)) << 4) + (uint32_t)(cbytes & 15);
}

// Trapezoid weight in ln k of node q on a source's own k prefix [0, nkm):
// the master weight, except at the prefix's last node (half interval) and
// beyond it (zero).
__device__ __forceinline__ double prefix_weight(const double *__restrict__ wk, const double *__restrict__ k, int nk,
                                                int nkm, int q) {
  if (q >= nkm) return 0.0;
  if (nkm == nk || q + 1 < nkm) return wk[q];
  return q > 0 ? 0.5 * (log(k[q]) - log(k[q - 1])) : 0.0;
}

// Split of the sources, all modes: one warp per (k, plan-order source) row.
// S[perm[m]][q][*] (fp32) -> hi/lo planes of the source's row in every
// tau-block [q][mt][kb]{hi, lo}[NT rows][128 B], 128-byte swizzled, zero
// padded beyond ntau and beyond the source's k prefix.  Each lane converts
// one 16-byte output chunk per plane at a time (8 bf16/fp16 or 4 tf32
// elements), so loads are 32-byte (16-byte for tf32) contiguous runs and
// stores whole 16-byte chunks.
// fp16 rows are first scaled by 2^s so that their largest |S| lies in
// [2^13, 2^14) (fp16 keeps 11 significant bits only in its normal range).
// Lane 0 writes the row's epilogue weight wq = sqrt(4 pi w_k P) 2^-(sJ + s),
// with the source's own k weights; (wq D')^2 is then the unscaled term.
// Every epilogue weight forms 4 pi w_k P in FP64 and takes its square root in
// FP32 (wq within 2^-24 relative; the same expression on every path).
// Rows at or beyond their source tile's longest k prefix (tile_nk) are left
// out: no work item of that tile reaches them.
template <int MODE, int CACHE>
__global__ void __launch_bounds__(256) split_rows_kernel(const float *__restrict__ S, const double *__restrict__ Pk,
                                                         const double *__restrict__ wk, const double *__restrict__ kk,
                                                         int M, int nk, int ntau, int NT, int n_mt, int nkbs,
                                                         int mpad, int sJ, const int *__restrict__ perm,
                                                         const int *__restrict__ nk_m,
                                                         const int *__restrict__ tile_nk, int vec,
                                                         char *__restrict__ sp, float *__restrict__ wq) {
  constexpr int EPC = MODE == kTF32 ? 4 : 8;  // elements per 16-byte chunk
  const int lane = threadIdx.x & 31;
  const size_t row = (size_t)blockIdx.x * 8 + (threadIdx.x >> 5);  // q * mpad + m
  if (row >= (size_t)nk * mpad) return;
  const int q = (int)(row / mpad), mfull = (int)(row - (size_t)q * mpad);
  const int mt = mfull / NT, n = mfull - mt * NT;
  if (q >= tile_nk[mt]) return;
  const bool live = mfull < M && q < nk_m[mfull];
  const int mc = live ? perm[mfull] : 0;
  const float *src = S + ((size_t)mc * nk + q) * ntau;
  int s = 0;
  constexpr int CPR = TcGeom<MODE>::kRowB / 16;  // 16-byte chunks per row of a tau-block
  constexpr int BB = 2 * TcGeom<MODE>::kRowB;    // bytes of one source row's hi + lo in a block
  const int nch = nkbs * CPR;  // 16-byte chunks per row over all tau-blocks
  // loads one chunk's fp32 values (zero beyond ntau and for dead rows)
  auto load_chunk = [&](int ch, float *v) {
    const int t0 = ch * EPC;
    if (live && vec && t0 + EPC <= ntau) {
      const float4 *s4 = reinterpret_cast<const float4 *>(src + t0);
#pragma unroll
      for (int u = 0; u < EPC / 4; ++u) {
        const float4 f = __ldg(s4 + u);
        v[4 * u + 0] = f.x;
        v[4 * u + 1] = f.y;
        v[4 * u + 2] = f.z;
        v[4 * u + 3] = f.w;
      }
    } else {
#pragma unroll
      for (int u = 0; u < EPC; ++u) v[u] = (live && t0 + u < ntau) ? __ldg(src + t0 + u) : 0.f;
    }
  };
  // fp16 with a short row: keep the row in registers between the max and the split
  float cache[CACHE > 0 ? CACHE : 1][EPC];
  if constexpr (CACHE > 0) {
#pragma unroll
    for (int j = 0; j < CACHE; ++j)
      if (lane + 32 * j < nch) load_chunk(lane + 32 * j, cache[j]);
  }
  if constexpr (MODE == kF16) {
    float mx = 0.f;
    if constexpr (CACHE > 0) {
#pragma unroll
      for (int j = 0; j < CACHE; ++j)
#pragma unroll
        for (int u = 0; u < EPC; ++u)
          if (lane + 32 * j < nch) mx = fmaxf(mx, fabsf(cache[j][u]));
    } else if (live && vec) {
      // 16-byte loads, eight in flight per lane
      const float4 *s4 = reinterpret_cast<const float4 *>(src);
      const int n4 = ntau >> 2;
#pragma unroll 8
      for (int c = lane; c < n4; c += 32) {
        const float4 f = __ldg(s4 + c);
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(f.x), fabsf(f.y)), fmaxf(fabsf(f.z), fabsf(f.w))));
      }
    } else if (live) {
      for (int t = lane; t < ntau; t += 32) mx = fmaxf(mx, fabsf(__ldg(src + t)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (mx > 0.f) {
      int e;
      frexpf(mx, &e);  // mx < 2^e
      s = 14 - e;
      s = s < -40 ? -40 : (s > 80 ? 80 : s);
    }
  }
  char *base = sp + ((size_t)(q * n_mt + mt) * nkbs) * (size_t)(BB * NT);
  auto split_store = [&](int ch, const float *v) {
    uint4 hi, lo;
    uint32_t *h = reinterpret_cast<uint32_t *>(&hi), *l = reinterpret_cast<uint32_t *>(&lo);
    if constexpr (MODE == kTF32) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        h[u] = tf32_rna_u(v[u]);
        l[u] = tf32_rna_u(v[u] - __uint_as_float(h[u]));
      }
    } else if constexpr (MODE == kF16) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float a = ldexpf(v[2 * u], s), b = ldexpf(v[2 * u + 1], s);
        const __half2 hh = __floats2half2_rn(a, b);
        const __half2 ll = __floats2half2_rn(a - __low2float(hh), b - __high2float(hh));
        h[u] = *reinterpret_cast<const uint32_t *>(&hh);
        l[u] = *reinterpret_cast<const uint32_t *>(&ll);
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
        const __nv_bfloat162 ll =
            __floats2bfloat162_rn(v[2 * u] - __low2float(hh), v[2 * u + 1] - __high2float(hh));
        h[u] = *reinterpret_cast<const uint32_t *>(&hh);
        l[u] = *reinterpret_cast<const uint32_t *>(&ll);
      }
    }
    char *blk = base + (size_t)(ch / CPR) * (BB * NT);
    const uint32_t o = sw_off<MODE>(n, (ch % CPR) * 16);
    *reinterpret_cast<uint4 *>(blk + o) = hi;
    *reinterpret_cast<uint4 *>(blk + NT * TcGeom<MODE>::kRowB + o) = lo;
  };
  if constexpr (CACHE > 0) {
#pragma unroll
    for (int j = 0; j < CACHE; ++j)
      if (lane + 32 * j < nch) split_store(lane + 32 * j, cache[j]);
  } else {
    for (int ch = lane; ch < nch; ch += 32) {
      float v[EPC];
      load_chunk(ch, v);
      split_store(ch, v);
    }
  }
  if (lane == 0) {
    float w = 0.f;
    if (live) {
      const float root = sqrtf((float)(4.0 * 3.14159265358979323846 * prefix_weight(wk, kk, nk, nk_m[mfull], q) *
                                       Pk[(size_t)mc * nk + q]));
      w = MODE == kF16 ? ldexpf(root, -(sJ + s)) : root;
    }
    wq[row] = w;
  }
}

// Row scales and epilogue weights of the fused fp16 path (a uniform batch,
// sources in caller order): one warp per two adjacent (source, k) rows, taken
// in memory order so that the 4 KB rows stream; with vec, every lane has its
// eight 16-byte loads of the two rows in flight before it takes a maximum.
// Same scale rule as the split pass: 2^s with the row's largest |S| in
// [2^13, 2^14), s clamped to [-40, 80]; wq = sqrt(4 pi w_k P) 2^-(sJ + s).
__global__ void __launch_bounds__(256) rowscale_kernel(const float *__restrict__ S, const double *__restrict__ Pk,
                                                       const double *__restrict__ wk, int M, int nk, int ntau,
                                                       int mpad, int sJ, int vec, float *__restrict__ wq,
                                                       float *__restrict__ sc) {
  const int lane = threadIdx.x & 31;
  const size_t rows = (size_t)M * nk;
  const size_t r0 = ((size_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 2;  // m * nk + q of the first row
  if (r0 >= rows) return;
  const bool two = r0 + 1 < rows;
  const float *a = S + r0 * ntau, *b = a + ntau;  // the second row follows the first
  float mx0 = 0.f, mx1 = 0.f;
  if (vec) {
    const float4 *a4 = reinterpret_cast<const float4 *>(a), *b4 = reinterpret_cast<const float4 *>(b);
    const int n4 = ntau >> 2;
    for (int c0 = 0; c0 < n4; c0 += 128) {
      float4 fa[4], fb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + lane + 32 * u;
        fa[u] = c < n4 ? __ldg(a4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        fb[u] = (two && c < n4) ? __ldg(b4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        mx0 = fmaxf(mx0, fmaxf(fmaxf(fabsf(fa[u].x), fabsf(fa[u].y)), fmaxf(fabsf(fa[u].z), fabsf(fa[u].w))));
        mx1 = fmaxf(mx1, fmaxf(fmaxf(fabsf(fb[u].x), fabsf(fb[u].y)), fmaxf(fabsf(fb[u].z), fabsf(fb[u].w))));
      }
    }
  } else {
    for (int t = lane; t < ntau; t += 32) {
      mx0 = fmaxf(mx0, fabsf(__ldg(a + t)));
      if (two) mx1 = fmaxf(mx1, fabsf(__ldg(b + t)));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
    mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
  }
  if (lane < (two ? 2 : 1)) {  // lane j writes row r0 + j
    const size_t r = r0 + lane;
    const float mx = lane ? mx1 : mx0;
    const int m = (int)(r / nk), q = (int)(r - (size_t)m * nk);
    int s = 0;
    if (mx > 0.f) {
      int e;
      frexpf(mx, &e);
      s = 14 - e;
      s = s < -40 ? -40 : (s > 80 ? 80 : s);
    }
    const float root = sqrtf((float)(4.0 * 3.14159265358979323846 * wk[q] * Pk[r]));
    wq[(size_t)q * mpad + m] = ldexpf(root, -(sJ + s));
    sc[(size_t)q * mpad + m] = ldexpf(1.f, s);
  }
}

// Epilogue weights of the fused bf16 path (no row scale): one thread per
// (k, plan-order source) row, wq = sqrt(4 pi w_k P).
__global__ void __launch_bounds__(256) weights_kernel(const double *__restrict__ Pk, const double *__restrict__ wk,
                                                      const double *__restrict__ kk, int M, int nk, int mpad,
                                                      const int *__restrict__ perm, const int *__restrict__ nk_m,
                                                      float *__restrict__ wq) {
  const size_t row = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (size_t)nk * mpad) return;
  const int q = (int)(row / mpad), m = (int)(row - (size_t)q * mpad);
  float w = 0.f;
  if (m < M && q < nk_m[m]) {
    const int mc = perm[m];
    w = sqrtf((float)(4.0 * 3.14159265358979323846 * prefix_weight(wk, kk, nk, nk_m[m], q) * Pk[(size_t)mc * nk + q]));
  }
  wq[row] = w;
}

// Sum of FP32 values as an unevaluated pair hi + lo of FP32 numbers: each
// add is Knuth's TwoSum (s = hi + v and its exact rounding error), the
// errors gathered in lo; read out once as (double) hi + lo.  The result is
// within ~n^2 2^-48 of the exact sum (n terms), at FP32-pipe cost (this
// GPU's FP64 pipe runs at a small fraction of its FP32 rate).
struct PairSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float s = hi + v;
    const float b = s - hi;
    lo += (hi - (s - b)) + (v - b);
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// The partial-slot indices of a tile, kReduceIdx at a time, staged in shared
// memory by the block, so that each thread's partial loads wait on no index
// load of their own.
constexpr int kReduceIdx = 1024;

// C[m][row] = sum over the tile's items (fixed order) of the FP32 chunk sums
// (PairSum); zero above the source's own l_max.  row: output index, whose
// multipole is lrow[row].  A block takes one source of the tile (its 128
// rows); each thread keeps 16 partial loads in flight.
__global__ void __launch_bounds__(128) reduce_kernel(const float *__restrict__ partial, const int *__restrict__ tile_ptr,
                                                     const int *__restrict__ tile_items, int NT, int n_mt, int M,
                                                     int nl, const int *__restrict__ lrow,
                                                     const int *__restrict__ perm, const int *__restrict__ lmax_m,
                                                     double *__restrict__ Cl) {
  __shared__ int idx[kReduceIdx];
  const int r = threadIdx.x;
  const int ml = blockIdx.x;       // source within the tile
  const int tile = blockIdx.y;     // lt * n_mt + mt
  const int lt = tile / n_mt, mt = tile - lt * n_mt;
  const int m = mt * NT + ml;
  const int row = lt * kTileL + r;
  if (m >= M) return;  // the whole block
  const bool live = row < nl && lrow[row] <= lmax_m[m];
  const float *col = partial + (size_t)ml * 128 + r;
  PairSum acc;
  const int e0 = tile_ptr[tile], e1 = tile_ptr[tile + 1];
  for (int c0 = e0; c0 < e1; c0 += kReduceIdx) {
    const int n = min(kReduceIdx, e1 - c0);
    __syncthreads();
    for (int i = r; i < n; i += 128) idx[i] = tile_items[c0 + i];
    __syncthreads();
    if (!live) continue;
    // sequential order; the loads of sixteen items are issued together
    int i = 0;
    for (; i + 16 <= n; i += 16) {
      float v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = col[(size_t)idx[i + u] * NT * 128];
#pragma unroll
      for (int u = 0; u < 16; ++u) acc.add(v[u]);
    }
    for (; i < n; ++i) acc.add(col[(size_t)idx[i] * NT * 128]);
  }
  if (row < nl) Cl[(size_t)perm[m] * nl + row] = acc.value();
}

// 1/x^2 of every node, x = k (tau0 - tau_i), in FP32 for the converters:
// 0 below the small-x cut x_lo and on the padding beyond ntau (whose
// sources are zero).  [nk][npad], npad = 32 * the tau-blocks.
__global__ void __launch_bounds__(256) te_ix2_kernel(const double *__restrict__ kk, const double *__restrict__ tau,
                                                     double tau0, double xlo, int nk, int ntau, int npad,
                                                     float *__restrict__ ix2) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nk * npad) return;
  const int q = (int)(e / npad), i = (int)(e - (size_t)q * npad);
  float v = 0.f;
  if (i < ntau) {
    const double x = kk[q] * (tau0 - tau[i]);
    if (x >= xlo) v = (float)(1.0 / (x * x));
  }
  ix2[e] = v;
}

// TE inputs per (k, model) row, models in caller order: the epilogue weight
// wq = sqrt(4 pi w_k P) and the small-x tail of Delta_E at l = 2,
//   tail = sum over the nodes with x = k (tau0 - tau_i) < x_lo (the last
//          ones: x falls with tau) of w_i S_P[m][k][i] j_2(x)/x^2,
// with j_2(x)/x^2 = 1/15 - x^2/210 + x^4/7560 - x^6/498960 (x <= 0.2).  The
// test x < x_lo is the one te_ix2_kernel makes, so every node is either in
// the table sum or in the tail.
__global__ void __launch_bounds__(256) te_weights_kernel(const double *__restrict__ Pk, const double *__restrict__ wk,
                                                         const double *__restrict__ kk,
                                                         const double *__restrict__ tau, double tau0, double xlo,
                                                         const double *__restrict__ wtau,
                                                         const float *__restrict__ SP, int M, int nk, int ntau,
                                                         int mpad, float *__restrict__ wq, float *__restrict__ tail) {
  const size_t row = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (size_t)nk * mpad) return;
  const int q = (int)(row / mpad), m = (int)(row - (size_t)q * mpad);
  float w = 0.f, t = 0.f;
  if (m < M) {
    w = sqrtf((float)(4.0 * 3.14159265358979323846 * wk[q] * Pk[(size_t)m * nk + q]));
    const float *src = SP + ((size_t)m * nk + q) * ntau;
    double acc = 0.0;
    for (int i = ntau - 1; i >= 0; --i) {
      const double x = kk[q] * (tau0 - tau[i]);
      if (x >= xlo) break;
      const double x2 = x * x;
      acc += wtau[i] * (double)src[i] * (1.0 / 15.0 - x2 * (1.0 / 210.0 - x2 * (1.0 / 7560.0 - x2 / 498960.0)));
    }
    t = (float)acc;
  }
  wq[row] = w;
  tail[row] = t;
}

// TE reduce: per (model, l) the FP64 fixed-order sums of the three chunk
// partials; C^EE = c_l^2 sum, C^TE = c_l sum, c_l^2 = (l+2)(l+1)l(l-1).
__global__ void __launch_bounds__(128) reduce_te_kernel(const float *__restrict__ partial,
                                                        const int *__restrict__ tile_ptr,
                                                        const int *__restrict__ tile_items, int H, int n_mt, int M,
                                                        int nl, const int *__restrict__ lrow, int scale_cl,
                                                        double *__restrict__ ClTT, double *__restrict__ ClEE,
                                                        double *__restrict__ ClTE) {
  __shared__ int idx[kReduceIdx];
  const int r = threadIdx.x;
  const int ml = blockIdx.x;
  const int tile = blockIdx.y;
  const int lt = tile / n_mt, mt = tile - lt * n_mt;
  const int m = mt * H + ml;
  const int row = lt * kTileL + r;
  if (m >= M) return;  // the whole block
  const bool live = row < nl;
  const float *col = partial + (size_t)ml * 128 + r;
  const size_t slot = (size_t)3 * H * 128;
  PairSum tt, ee, te;
  const int e0 = tile_ptr[tile], e1 = tile_ptr[tile + 1];
  for (int c0 = e0; c0 < e1; c0 += kReduceIdx) {
    const int n = min(kReduceIdx, e1 - c0);
    __syncthreads();
    for (int i = r; i < n; i += 128) idx[i] = tile_items[c0 + i];
    __syncthreads();
    if (!live) continue;
    // sequential order; the loads of eight items (three sums each) are issued together
    int i = 0;
    for (; i + 8 <= n; i += 8) {
      float a[8], b[8], c[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float *pp = col + (size_t)idx[i + u] * slot;
        a[u] = pp[0];
        b[u] = pp[(size_t)H * 128];
        c[u] = pp[(size_t)2 * H * 128];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        tt.add(a[u]);
        ee.add(b[u]);
        te.add(c[u]);
      }
    }
    for (; i < n; ++i) {
      const float *pp = col + (size_t)idx[i] * slot;
      tt.add(pp[0]);
      ee.add(pp[(size_t)H * 128]);
      te.add(pp[(size_t)2 * H * 128]);
    }
  }
  if (!live) return;
  const int l = lrow[row];
  // E-mode (scale_cl): C^EE = c_l^2 sum, C^TE = c_l sum; pairs of kernel grids: none
  const double c2 = !scale_cl ? 1.0 : (l >= 2 ? (double)(l + 2) * (l + 1) * l * (l - 1) : 0.0);
  const size_t o = (size_t)m * nl + row;
  ClTT[o] = tt.value();
  ClEE[o] = c2 * ee.value();
  ClTE[o] = sqrt(c2) * te.value();
}

// ------------------------------------------------------------------ plan

// Work plan of one batched launch.  Sources are processed in plan order:
// sorted by l_max (then k prefix) descending, so that at every (k, l-tile)
// the sources that still need it form a prefix of the source tiles.  All
// integer arrays live in one blob, uploaded once (or written into the fixed
// buffer of the allocation-free entry point).
struct TcPlan {
  int mode = -1, M = 0, NT = 0, n_mt = 0, nkbs = 0, mpad = 0, nctas = 0, nitems = 0, ntile = 0;
  bool uniform = true;
  bool fused = false;  // sources converted inside the tensor-core kernel (no split pass)
  bool te = false;     // temperature + E-mode: NT models per tile, 2 NT operand rows
  int lp = 1;          // l-tiles per item (2: adjacent tiles share the item's source blocks)
  int ksub = kKSub;    // non-empty k per FP32 chunk sum
  int chain = 0;       // lp = 2: 1, chain records where an item's second tile is idle; 2, also l-tile 0 alone
  int nslots = 0;      // chunk slots (each lp tiles' partials)
  int tail = 0;        // the tail setting the items were cut with (as tail_key)
  int per_cta = 4;     // items of about equal cost per persistent CTA (kalign 0)
  int kalign = 0;      // items end at multiples of kalign k (0: at the cost target)
  int kalign_req = 0;  // the requested alignment (the plan cache's key; kalign may be half of it)
  std::vector<int> blob;
  size_t o_items = 0, o_tile_ptr = 0, o_tile_items = 0, o_perm = 0, o_nkm = 0, o_lmaxm = 0, o_tnk = 0;
  std::vector<double> cost;  // per item
  int *d_blob = nullptr;
  bool own_blob = false;
  float *d_ix2 = nullptr;  // te: 1/x^2 per node [nk][nkbs * 32], built with the plan
  size_t off_sp = 0, off_wp = 0, off_sc = 0, off_part = 0, off_ctr = 0, ws_bytes = 0;

  const TcItem *items(const int *base) const { return reinterpret_cast<const TcItem *>(base + o_items); }
  void release() {
    if (own_blob && d_blob) cudaFree(d_blob);
    d_blob = nullptr;
    own_blob = false;
    if (d_ix2) cudaFree(d_ix2);
    d_ix2 = nullptr;
  }
};

std::mutex g_plan_mu;
std::vector<std::pair<const gcamb_grid *, TcPlan *>> g_plans;

// Source-tile width of the uniform entry point: 64 for small batches, else
// 128 (double-buffered accumulator pairs); GCAMB_TC_NT=64|128|256 overrides it.
int pick_nt(int M) {
  int nt = M <= 64 ? 64 : 128;
  if (const char *e = getenv("GCAMB_TC_NT")) {
    const int v = atoi(e);
    if (v == 64 || v == 128 || v == 256) nt = v;
  }
  return nt;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The fused kernel reads the caller's FP32 sources by TMA as [M][nk][ntau]
// boxes of 32 tau x NT sources and splits them in shared memory.  It needs
// the sources in caller order (a uniform batch), a row pitch of whole 16-byte
// units (ntau % 4 == 0), a bf16 or fp16 split and NT <= 128
// (the in-place conversion holds a stage's tile in the converters' registers).
// GCAMB_TC_FUSED=0 selects the separate split pass instead.
bool want_fused(const gcamb_grid *g, int mode, int nt, bool uniform) {
  if (const char *e = getenv("GCAMB_TC_FUSED"))
    if (e[0] == '0') return false;
  return uniform && (mode == GCAMB_BF16X3 || mode == GCAMB_F16X3) && nt <= 128 && g->ntau % 4 == 0;
}

// l-tiles per item (not TE; bf16/fp16 with NT <= 128): 2, so that each source
// block is loaded (and, fused, split) once for two tiles; GCAMB_TC_LP=1
// selects one tile per item.
int want_lp(int mode, int nt, bool te) {
  if (te || mode == GCAMB_TF32X3 || nt > 128) return 1;
  if (const char *e = getenv("GCAMB_TC_LP"))
    if (e[0] == '1') return 1;
  return 2;
}

// Chain records of lp = 2 plans: 1 (the default), at every k where an
// item's second l-tile has no blocks, the first tile's hi*hi sum is spread
// over three accumulators (the second tile's pair is free); 2, l-tile 0 is
// also given items of its own, so that all of its k are chain records;
// 0, none (GCAMB_TC_CHAIN=0|1|2).
int want_chain() {
  if (const char *e = getenv("GCAMB_TC_CHAIN")) {
    if (e[0] == '0') return 0;
    if (e[0] == '2') return 2;
  }
  return 1;
}

// The tail of the work list: the share of the cost, handed out last, whose
// items are cut into pieces, and the pieces per item (GCAMB_TC_TAIL=frac:parts;
// 0:1 none).
void want_tail(double *frac, int *parts) {
  *frac = 0.1;
  *parts = 4;
  if (const char *e = getenv("GCAMB_TC_TAIL")) {
    double f = 0.0;
    int n = 1;
    if (sscanf(e, "%lf:%d", &f, &n) == 2 && f >= 0.0 && f <= 1.0 && n >= 1 && n <= 64) {
      *frac = f;
      *parts = n;
    }
  }
}

// k-aligned work items (GCAMB_TC_KALIGN=n, 0: items of equal cost instead):
// by default 12 k for uniform batches and 16 for uneven and temperature +
// E-mode plans (measured on the 256-source l_max = 2500 batch, F16X3:
// 1.535 ms per step with items of equal cost, 1.502 / 1.501 / 1.508 / 1.544 /
// 1.567 / 1.651 ms at 8 / 12 / 16 / 20 / 24 / 32 k; the 1000-source uneven
// batch 16.39 ms against 15.97 / 15.67 / 15.54 / 15.82 / 15.75 ms at 8 / 12 /
// 16 / 20 / 24 k; the TE batch 2.93 ms against 2.79 / 2.69 / 2.66 ms at 8 /
// 12 / 16 k).
int want_kalign(bool uniform, bool te = false) {
  if (const char *e = getenv("GCAMB_TC_KALIGN")) {
    const int v = atoi(e);
    if (v >= 0 && v <= kKChunkMax) return v;
  }
  return uniform && !te ? 12 : 16;
}

bool kalign_from_env() {
  const char *e = getenv("GCAMB_TC_KALIGN");
  if (!e) return false;
  const int v = atoi(e);
  return v >= 0 && v <= kKChunkMax;
}

int tail_key() {
  double f = 0.0;
  int n = 1;
  want_tail(&f, &n);
  return (int)(f * 1000.0 + 0.5) * 100 + n;
}

// Non-empty k per FP32 chunk sum of the epilogue (the partial-sum length):
// kKSub, or GCAMB_TC_KSUB = 1..64 (1: every k's term is its own partial, so
// the reduce's compensated sum is the FP64 sum of the FP32 terms).
int want_ksub() {
  if (const char *e = getenv("GCAMB_TC_KSUB")) {
    const int v = atoi(e);
    if (v >= 1 && v <= kKChunkMax) return v;
  }
  return kKSub;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

// Tensor map of the sources S[M][nk][ntau] (FP32): box 32 tau x 1 k x NT sources.
int encode_sources(CUtensorMap *tm, const float *S, int M, int nk, int ntau, int NT) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return fail(GCAMB_ECUDA, "los_cl: cuTensorMapEncodeTiled is not available from the driver");
  if (reinterpret_cast<uintptr_t>(S) % 16 != 0)
    return fail(GCAMB_EINVAL, "los_cl: S must be 16-byte aligned");
  const cuuint64_t dims[3] = {(cuuint64_t)ntau, (cuuint64_t)nk, (cuuint64_t)M};
  const cuuint64_t strides[2] = {(cuuint64_t)ntau * 4, (cuuint64_t)nk * ntau * 4};
  const cuuint32_t box[3] = {32, 1, (cuuint32_t)NT};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(S), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(GCAMB_ECUDA, "los_cl: tensor map of S rejected (" + std::to_string((int)r) + ")");
  return GCAMB_OK;
}

int num_sms() {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 148;
}

// Work-list settings a plan's autotuner chooses among (null: the defaults
// and the environment's switches): lp 1 forces one l-tile per item (0: the
// default, two where the mode allows); the tail (the share of the cost
// handed out last and the pieces each of its items is cut into); kalign,
// items cut at multiples of kalign k, or (0) per_cta items of about equal
// cost per persistent CTA.
struct PlanCfg {
  int lp = 0;
  double tail_frac = 0.1;
  int tail_parts = 4;
  int per_cta = 4;
  int kalign = 0;
};

// lmax_c / nk_c: per-source l_max and k-prefix length in the caller's order,
// or null for a uniform batch (every source uses the whole grid).
//
// te: a temperature + E-mode plan (uniform, fused bf16): nt models per tile,
// each with a temperature and a polarisation operand row.
void plan_build(const gcamb_grid *g, int M, int mode, int nt, const int *lmax_c, const int *nk_c, TcPlan &pl,
                bool te = false, const PlanCfg *cfg = nullptr, bool halve_if_few = false) {
  const ModeLayout lay = mode_layout(mode);
  const Table &t = g->tab[mode];
  pl.mode = mode;
  pl.M = M;
  pl.NT = nt;
  pl.te = te;
  pl.n_mt = (M + nt - 1) / nt;
  pl.mpad = pl.n_mt * nt;
  pl.nkbs = (g->ntau + lay.kb - 1) / lay.kb;
  pl.uniform = !lmax_c && !nk_c;
  std::vector<int> perm(M), nkm(M), lmm(M);
  for (int m = 0; m < M; ++m) perm[m] = m;
  auto lm_of = [&](int m) { return lmax_c ? lmax_c[m] : g->lmax; };
  auto nk_of = [&](int m) { return nk_c ? nk_c[m] : g->nk; };
  if (!pl.uniform)
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
      if (lm_of(a) != lm_of(b)) return lm_of(a) > lm_of(b);
      return nk_of(a) > nk_of(b);
    });
  // uneven batches take the split pass even when the caller's order is the
  // plan's: measured on the 1000-source batch, the split-source kernel plus
  // the pass beat the fused kernel (48.0k against 43.8k spectra/s)
  pl.fused = te || want_fused(g, mode, nt, pl.uniform);
  pl.lp = pl.nkbs < 32768 ? want_lp(mode, nt, te) : 1;  // LP = 2 records pack two block counts in 16 bits
  if (cfg && cfg->lp == 1) pl.lp = 1;
  const int lp = pl.lp;
  for (int j = 0; j < M; ++j) {
    nkm[j] = nk_of(perm[j]);
    lmm[j] = lm_of(perm[j]);
  }
  std::vector<int> tile_nk(pl.n_mt, 0), tile_lm(pl.n_mt, -1);
  for (int j = 0; j < M; ++j) {
    tile_nk[j / nt] = std::max(tile_nk[j / nt], nkm[j]);
    tile_lm[j / nt] = std::max(tile_lm[j / nt], lmm[j]);
  }
  // items: (l-tile, source tile, contiguous chunk of active k); lp = 2:
  // (first of two adjacent l-tiles, ...), active where either tile is, the
  // cost weighing the stages (the longer tile) and the second tile's MMAs
  // l-tiles of the item that starts at tile lt for source tile mt
  // chain items (lp = 2): l-tile 0 alone, its hi*hi sum spread over three
  // accumulators (the MMA warp's chain mode); the pairs then start at tile 1
  pl.chain = lp == 2 ? want_chain() : 0;
  std::vector<int> starts;
  for (int lt = 0; lt < g->nlt; lt += (pl.chain == 2 && lt == 0) ? 1 : lp) starts.push_back(lt);
  auto chain_of = [&](int lt) { return pl.chain == 2 && lt == 0; };
  auto ntl_of = [&](int lt, int mt) {
    return (lp == 2 && !chain_of(lt) && lt + 1 < g->nlt && tile_lm[mt] >= g->lrow[(size_t)(lt + 1) * kTileL]) ? 2
                                                                                                             : 1;
  };
  auto kcost = [&](int q, int lt, int ntl) -> double {
    const int a = t.nkb[(size_t)q * g->nlt + lt];
    const int b = ntl == 2 ? t.nkb[(size_t)q * g->nlt + lt + 1] : 0;
    if (a == 0 && b == 0) return 0.0;
    return std::max(a, b) + 0.5 * std::min(a, b) + 0.5;
  };
  double total = 0.0;
  for (int lt : starts)
    for (int mt = 0; mt < pl.n_mt; ++mt) {
      if (tile_lm[mt] < g->lrow[(size_t)lt * kTileL]) continue;
      for (int q = 0; q < tile_nk[mt]; ++q) total += kcost(q, lt, ntl_of(lt, mt));
    }
  const int sms = num_sms();
  pl.per_cta = cfg ? cfg->per_cta : 4;
  const double target = std::max(4.0, total / (sms * (double)pl.per_cta));
  // k-aligned items: every item ends at a multiple of kalign (then the items
  // of all l-tile pairs and source tiles that cover the same k run together
  // and share the source blocks in L2), or, with kalign 0, at the cost target
  const int kalign_req = cfg ? cfg->kalign : want_kalign(pl.uniform, te);
  pl.kalign_req = kalign_req;
  std::vector<TcItem> items;
  auto build_items = [&](int kalign) {
    items.clear();
    pl.cost.clear();
    for (int lt : starts)
      for (int mt = 0; mt < pl.n_mt; ++mt) {
        if (tile_lm[mt] < g->lrow[(size_t)lt * kTileL]) continue;
        // an item spans at most kKChunkMax k and starts and ends at a k with
        // stored blocks
        const int ntl = ntl_of(lt, mt);
        int qb = -1, qlast = -1;
        double c = 0.0;
        for (int q = 0; q < tile_nk[mt]; ++q) {
          const double kc = kcost(q, lt, ntl);
          if (kc == 0.0) continue;
          if (qb >= 0 && q - qb + 1 > kKChunkMax) {
            items.push_back({lt, mt, qb, qlast + 1, ntl, 0, chain_of(lt) ? 1 : 0, 0});
            pl.cost.push_back(c);
            qb = -1;
          }
          qlast = q;
          if (qb < 0) {
            qb = q;
            c = 0.0;
          }
          c += kc;
          if ((kalign > 0 ? (q + 1) % kalign == 0 : c >= target) || q - qb + 1 >= kKChunkMax) {
            items.push_back({lt, mt, qb, q + 1, ntl, 0, chain_of(lt) ? 1 : 0, 0});
            pl.cost.push_back(c);
            qb = -1;
          }
        }
        if (qb >= 0) {
          items.push_back({lt, mt, qb, qlast + 1, ntl, 0, chain_of(lt) ? 1 : 0, 0});
          pl.cost.push_back(c);
        }
      }
  };
  int kalign = kalign_req;
  build_items(kalign);
  // a uniform batch on one or two multipole tiles has few items per CTA, and
  // the CTAs run out of work unevenly: items of half the k range (130 sampled
  // multipoles, 256 sources: 310k -> 338k spectra/s at 6 k instead of 12).
  // Not for the fixed buffer of the allocation-free entry point, which would
  // hold twice the partials.
  if (halve_if_few && !cfg && pl.uniform && !te && !kalign_from_env() && kalign >= 12 &&
      (int)items.size() < 4 * sms) {
    kalign /= 2;
    build_items(kalign);
  }
  pl.kalign = kalign;
  pl.nitems = (int)items.size();
  // hand-out order: by k position (high k first), so that the CTAs working at
  // any moment share the source blocks of nearby k in L2; one persistent CTA
  // per SM takes the next item from a counter when it is free
  {
    std::vector<int> order(pl.nitems);
    for (int i = 0; i < pl.nitems; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return (items[a].qb + items[a].qe) > (items[b].qb + items[b].qe);
    });
    std::vector<TcItem> sorted(pl.nitems);
    std::vector<double> sc(pl.nitems);
    for (int i = 0; i < pl.nitems; ++i) {
      sorted[i] = items[order[i]];
      sc[i] = pl.cost[order[i]];
    }
    items.swap(sorted);
    pl.cost.swap(sc);
  }
  // the tail: the items handed out last (the last `frac` of the cost) are cut
  // into `parts` pieces of about equal cost, so that the persistent CTAs run
  // out of work closer together
  {
    double frac = 0.0;
    int parts = 1;
    if (cfg) {
      frac = cfg->tail_frac;
      parts = cfg->tail_parts;
    } else {
      want_tail(&frac, &parts);
    }
    pl.tail = (int)(frac * 1000.0 + 0.5) * 100 + parts;
    if (frac > 0.0 && parts > 1) {
      double tot = 0.0;
      for (double c : pl.cost) tot += c;
      std::vector<TcItem> out;
      std::vector<double> oc;
      double before = 0.0;
      for (int i = 0; i < pl.nitems; ++i) {
        const TcItem it = items[i];
        const double c = pl.cost[i];
        if (before < (1.0 - frac) * tot || c <= 0.0) {
          out.push_back(it);
          oc.push_back(c);
        } else {
          const double piece = c / parts;
          double acc = 0.0;
          int qb = it.qb;
          for (int q = it.qb; q < it.qe; ++q) {
            const double kc = kcost(q, it.lt, it.ntl);
            acc += kc;
            // cut after a k with blocks once a piece's cost is reached (the
            // next piece starts at the next k with blocks)
            if (kc > 0.0 && acc >= piece && q + 1 < it.qe) {
              int qn = q + 1;
              while (qn < it.qe && kcost(qn, it.lt, it.ntl) == 0.0) ++qn;
              if (qn >= it.qe) break;
              TcItem a = it;
              a.qb = qb;
              a.qe = q + 1;
              out.push_back(a);
              oc.push_back(acc);
              qb = qn;
              acc = 0.0;
              q = qn - 1;
            }
          }
          TcItem a = it;
          a.qb = qb;
          out.push_back(a);
          double rest = 0.0;
          for (int q = qb; q < it.qe; ++q) rest += kcost(q, it.lt, it.ntl);
          oc.push_back(rest);
        }
        before += c;
      }
      items.swap(out);
      pl.cost.swap(oc);
      pl.nitems = (int)items.size();
    }
  }
  pl.nctas = std::max(1, std::min(sms, pl.nitems));

  // chunk slots: an item's FP32 sums are flushed every ksub non-empty k (the
  // producer's records), each chunk to its own slot of lp tiles' partials
  pl.ksub = want_ksub();
  std::vector<int> nchunk(pl.nitems);
  pl.nslots = 0;
  for (int i = 0; i < pl.nitems; ++i) {
    int rec = 0;
    for (int q = items[i].qb; q < items[i].qe; ++q)
      if (kcost(q, items[i].lt, items[i].ntl) > 0.0) ++rec;
    nchunk[i] = (rec + pl.ksub - 1) / pl.ksub;
    items[i].pbase = pl.nslots;
    pl.nslots += nchunk[i];
  }
  // per (l-tile, source tile): its chunks' partials in increasing k (fixed
  // reduce order); chunk c of item i writes partial (pbase + c) * lp + s for
  // its tile lt + s
  pl.ntile = g->nlt * pl.n_mt;
  std::vector<int> tile_ptr(pl.ntile + 1, 0);
  for (int i = 0; i < pl.nitems; ++i)
    for (int sub = 0; sub < items[i].ntl; ++sub) tile_ptr[(items[i].lt + sub) * pl.n_mt + items[i].mt + 1] += nchunk[i];
  for (int i = 0; i < pl.ntile; ++i) tile_ptr[i + 1] += tile_ptr[i];
  std::vector<int> tile_items(tile_ptr[pl.ntile]);
  {
    std::vector<int> idx(pl.nitems), fill(tile_ptr.begin(), tile_ptr.end() - 1);
    for (int i = 0; i < pl.nitems; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return items[a].qb < items[b].qb; });
    for (int i : idx)
      for (int c = 0; c < nchunk[i]; ++c)
        for (int sub = 0; sub < items[i].ntl; ++sub)
          tile_items[fill[(items[i].lt + sub) * pl.n_mt + items[i].mt]++] = (items[i].pbase + c) * lp + sub;
  }
  // blob
  pl.blob.clear();
  auto put = [&](const int *p, size_t n) {
    const size_t o = pl.blob.size();
    pl.blob.insert(pl.blob.end(), p, p + n);
    while (pl.blob.size() % 4) pl.blob.push_back(0);  // 16-byte alignment of every array
    return o;
  };
  pl.o_items = put(reinterpret_cast<const int *>(items.data()), items.size() * (sizeof(TcItem) / sizeof(int)));
  pl.o_tile_ptr = put(tile_ptr.data(), tile_ptr.size());
  pl.o_tile_items = put(tile_items.data(), tile_items.size());
  pl.o_perm = put(perm.data(), perm.size());
  pl.o_nkm = put(nkm.data(), nkm.size());
  pl.o_lmaxm = put(lmm.data(), lmm.size());
  pl.o_tnk = put(tile_nk.data(), tile_nk.size());
  if (pl.blob.empty()) pl.blob.push_back(0);
  // workspace: split sources (not with the fused kernel), weights, fp16 row
  // scales (fused fp16), k-chunk partials
  // (te: the l = 2 tails in the scale slot, three partials per model)
  const size_t row_b = mode == GCAMB_TF32X3 ? 128 : 64;  // operand row bytes of a 32-tau block
  const size_t sp_bytes = pl.fused ? 0 : (size_t)g->nk * pl.n_mt * pl.nkbs * 2 * row_b * pl.NT;
  const size_t wp_bytes = (size_t)g->nk * pl.mpad * sizeof(float);
  const size_t sc_bytes = (te || (pl.fused && mode == GCAMB_F16X3)) ? wp_bytes : 0;
  const size_t part_bytes = std::max<size_t>(1, pl.nslots) * lp * (te ? 3 : 1) * pl.NT * 128 * sizeof(float);
  pl.off_sp = 0;
  pl.off_wp = align256(sp_bytes);
  pl.off_sc = pl.off_wp + align256(wp_bytes);
  pl.off_part = pl.off_sc + align256(sc_bytes);
  pl.off_ctr = pl.off_part + align256(part_bytes);
  pl.ws_bytes = pl.off_ctr + 256;
}

size_t blob_bytes(const TcPlan &pl) { return align256(pl.blob.size() * sizeof(int)); }

int upload_blob(TcPlan &pl) {
  cudaError_t e = cudaMalloc(&pl.d_blob, pl.blob.size() * sizeof(int));
  if (e != cudaSuccess) {
    pl.d_blob = nullptr;
    return cuda_fail(e, "plan: allocation");
  }
  pl.own_blob = true;
  e = cudaMemcpy(pl.d_blob, pl.blob.data(), pl.blob.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "plan: upload");
  return GCAMB_OK;
}

TcPlan *get_plan(const gcamb_grid *g, int M, int mode, int *rc) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  const int nt = pick_nt(M);
  for (auto &e : g_plans)
    if (e.first == g && !e.second->te && e.second->M == M && e.second->mode == mode && e.second->NT == nt &&
        e.second->fused == want_fused(g, mode, nt, true) && e.second->ksub == want_ksub() &&
        e.second->tail == tail_key() && e.second->kalign_req == want_kalign(true) &&
        e.second->chain == (e.second->lp == 2 ? want_chain() : 0) &&
        e.second->lp == (e.second->nkbs < 32768 ? want_lp(mode, nt, false) : 1))
      return e.second;
  TcPlan *pl = new TcPlan();
  plan_build(g, M, mode, nt, nullptr, nullptr, *pl, false, nullptr, true);
  if ((*rc = upload_blob(*pl)) != GCAMB_OK) {
    pl->release();
    delete pl;
    return nullptr;
  }
  g_plans.push_back({g, pl});
  return pl;
}

template <int NT, int MODE, bool FUSED, int TE = 0, int LP = 1>
int launch_tc_kernel(const gcamb_grid *g, const TcPlan &pl, const CUtensorMap &tm, const CUtensorMap &tm2,
                     const TcParams &prm, cudaStream_t st) {
  using Cfg = TcCfg<NT, MODE, (TE == 2 || LP == 2) ? 2 : 1, LP>;
  cudaError_t e = cudaFuncSetAttribute(los_cl_tc_kernel<NT, MODE, FUSED, TE, LP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmemBytes);
  if (e != cudaSuccess) return cuda_fail(e, "los_cl: smem attribute");
  e = cudaMemsetAsync(prm.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "los_cl: counter reset");
  ProfScope prof(GCAMB_K_TC, st);
  los_cl_tc_kernel<NT, MODE, FUSED, TE, LP>
      <<<(unsigned)pl.nctas, TcRoles<FUSED, TE, LP>::kThreadsT, Cfg::kSmemBytes, st>>>(tm, tm2, prm);
  return GCAMB_OK;
}

template <int NT, int MODE>
int launch_tc(const gcamb_grid *g, const TcPlan &pl, const float *S, const double *Pk, double *Cl, char *ws,
              cudaStream_t st, int *err_word = nullptr, bool use_err_word = false) {
  constexpr bool kCanFuse = NT <= 128 && MODE != kTF32;
  const Table &t = g->tab[pl.mode];
  char *sp = ws + pl.off_sp;
  float *wp = reinterpret_cast<float *>(ws + pl.off_wp);
  float *sc = reinterpret_cast<float *>(ws + pl.off_sc);
  float *part = reinterpret_cast<float *>(ws + pl.off_part);
  const int *B = pl.d_blob;
  const int *perm = B + pl.o_perm, *nkm = B + pl.o_nkm, *lmm = B + pl.o_lmaxm, *tnk = B + pl.o_tnk;
  const bool fused = kCanFuse && pl.fused;
  CUtensorMap tm;
  memset(&tm, 0, sizeof tm);
  if (fused) {
    if (int rc = encode_sources(&tm, S, pl.M, g->nk, g->ntau, NT)) return rc;
  }
  {
    const size_t rows = (size_t)g->nk * pl.mpad;
    const int vec = (g->ntau % 4 == 0) && (reinterpret_cast<uintptr_t>(S) % 16 == 0);
    const unsigned nblk = (unsigned)((rows + 7) / 8);
    // the fused kernel's inputs (weights; fp16: and the row scales) are
    // traced as weights, the split pass (which also writes the weights) as split
    ProfScope prof(fused ? GCAMB_K_WEIGHTS : GCAMB_K_SPLIT, st);
    if (fused && MODE == kBF16)
      weights_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(Pk, g->d_wk, g->d_k, pl.M, g->nk, pl.mpad, perm,
                                                                     nkm, wp);
    else if (fused) {
      // rows beyond M (the last tile's padding sources) get zero weights and scales
      if (pl.mpad > pl.M) {
        cudaError_t e = cudaMemsetAsync(wp, 0, (size_t)g->nk * pl.mpad * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(sc, 0, (size_t)g->nk * pl.mpad * sizeof(float), st);
        if (e != cudaSuccess) return cuda_fail(e, "los_cl: weight reset");
      }
      rowscale_kernel<<<(unsigned)(((size_t)pl.M * g->nk + 15) / 16), 256, 0, st>>>(
          S, Pk, g->d_wk, pl.M, g->nk, g->ntau, pl.mpad, t.scale_exp, vec, wp, sc);
    }
    else if (MODE == kF16 && pl.nkbs * (TcGeom<MODE>::kRowB / 16) <= 32 * 4)  // rows of up to 1024 tau
      split_rows_kernel<MODE, 4><<<nblk, 256, 0, st>>>(S, Pk, g->d_wk, g->d_k, pl.M, g->nk, g->ntau, NT, pl.n_mt,
                                                       pl.nkbs, pl.mpad, t.scale_exp, perm, nkm, tnk, vec, sp, wp);
    else if (MODE == kF16 && pl.nkbs * (TcGeom<MODE>::kRowB / 16) <= 32 * 8)
      split_rows_kernel<MODE, 8><<<nblk, 256, 0, st>>>(S, Pk, g->d_wk, g->d_k, pl.M, g->nk, g->ntau, NT, pl.n_mt,
                                                       pl.nkbs, pl.mpad, t.scale_exp, perm, nkm, tnk, vec, sp, wp);
    else
      split_rows_kernel<MODE, 0><<<nblk, 256, 0, st>>>(S, Pk, g->d_wk, g->d_k, pl.M, g->nk, g->ntau, NT, pl.n_mt,
                                                       pl.nkbs, pl.mpad, t.scale_exp, perm, nkm, tnk, vec, sp, wp);
  }
  if (pl.nitems > 0) {
    int *ctr = reinterpret_cast<int *>(ws + pl.off_ctr);
    TcParams prm{static_cast<const char *>(t.d_data), nullptr, t.d_off, t.d_nkb, sp, wp, sc, nullptr, -1,
                 pl.items(B), ctr, pl.nitems, pl.ksub, pl.chain >= 1 ? 1 : 0, part, use_err_word ? err_word : device_error_flag(), g->nlt, pl.n_mt,
                 pl.nkbs, pl.mpad};
    if (!prm.err && !use_err_word) return fail(GCAMB_ECUDA, "los_cl: error flag allocation");
    int rc;
    if constexpr (kCanFuse)
      rc = fused ? (pl.lp == 2 ? launch_tc_kernel<NT, MODE, true, 0, 2>(g, pl, tm, tm, prm, st)
                               : launch_tc_kernel<NT, MODE, true>(g, pl, tm, tm, prm, st))
                 : (pl.lp == 2 ? launch_tc_kernel<NT, MODE, false, 0, 2>(g, pl, tm, tm, prm, st)
                               : launch_tc_kernel<NT, MODE, false>(g, pl, tm, tm, prm, st));
    else
      rc = launch_tc_kernel<NT, MODE, false>(g, pl, tm, tm, prm, st);
    if (rc) return rc;
  }
  dim3 rgrid(NT, pl.ntile);
  ProfScope prof(GCAMB_K_REDUCE, st);
  reduce_kernel<<<rgrid, 128, 0, st>>>(part, B + pl.o_tile_ptr, B + pl.o_tile_items, NT, pl.n_mt, pl.M, g->nl,
                                       g->d_lrow, perm, lmm, Cl);
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

int launch_plan(const gcamb_grid *g, const TcPlan &pl, const float *S, const double *Pk, double *Cl, char *w,
                cudaStream_t st, int *err_word = nullptr, bool use_err_word = false) {
  switch (pl.mode) {
    case GCAMB_TF32X3: return launch_mode<kTF32>(g, pl, S, Pk, Cl, w, st, err_word, use_err_word);
    case GCAMB_F16X3: return launch_mode<kF16>(g, pl, S, Pk, Cl, w, st, err_word, use_err_word);
    default: return launch_mode<kBF16>(g, pl, S, Pk, Cl, w, st, err_word, use_err_word);
  }
}

// Models per tile of a temperature + E-mode batch (operand rows = twice
// that): 32 for small batches, else 64; GCAMB_TC_NT=64|128 (operand rows)
// overrides it.
int pick_h_te(int M) {
  int h = 2 * M <= 64 ? 32 : 64;
  if (const char *e = getenv("GCAMB_TC_NT")) {
    const int v = atoi(e);
    if (v == 64 || v == 128) h = v / 2;
  }
  return h;
}

// The grid's 1/x^2 per node for the converters of a TE plan (once per plan).
int build_ix2(const gcamb_grid *g, TcPlan &pl) {
  double xlo = 0.0;
  if (emode_x_lo(g, &xlo)) return fail(GCAMB_EINVAL, "los_cl_te: eps_cut too large for the l = 2 limit");
  const int npad = pl.nkbs * 32;
  const size_t n = (size_t)g->nk * npad;
  cudaError_t e = cudaMalloc(&pl.d_ix2, n * sizeof(float));
  if (e != cudaSuccess) {
    pl.d_ix2 = nullptr;
    return cuda_fail(e, "los_cl_te: 1/x^2 table allocation");
  }
  te_ix2_kernel<<<(unsigned)((n + 255) / 256), 256>>>(g->d_k, g->d_tau, g->tau0, xlo, g->nk, g->ntau, npad, pl.d_ix2);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "los_cl_te: 1/x^2 table");
  return GCAMB_OK;
}

TcPlan *get_plan_te(const gcamb_grid *g, int M, int *rc) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  const int h = pick_h_te(M);
  for (auto &e : g_plans)
    if (e.first == g && e.second->te && e.second->M == M && e.second->NT == h && e.second->ksub == want_ksub() &&
        e.second->kalign_req == want_kalign(true, true))
      return e.second;
  TcPlan *pl = new TcPlan();
  plan_build(g, M, GCAMB_BF16X3, h, nullptr, nullptr, *pl, true);
  if ((*rc = upload_blob(*pl)) == GCAMB_OK) *rc = build_ix2(g, *pl);
  if (*rc != GCAMB_OK) {
    pl->release();
    delete pl;
    return nullptr;
  }
  g_plans.push_back({g, pl});
  return pl;
}

// Temperature + E-mode batch: weights and l = 2 tails,
// the tensor-core kernel over NT = 2 H operand rows per tile, the TE reduce
// (1/x^2 per node was built with the plan).
template <int NT>
int launch_tc_te(const gcamb_grid *g, const TcPlan &pl, const float *ST, const float *SP, const double *Pk,
                 double *ClTT, double *ClEE, double *ClTE, char *ws, double xlo, cudaStream_t st) {
  constexpr int H = NT / 2;
  const Table &t = g->tab[GCAMB_BF16X3];
  const float *ix2 = pl.d_ix2;
  float *wp = reinterpret_cast<float *>(ws + pl.off_wp);
  float *tail = reinterpret_cast<float *>(ws + pl.off_sc);
  float *part = reinterpret_cast<float *>(ws + pl.off_part);
  const int *B = pl.d_blob;
  CUtensorMap tm1, tm2;
  memset(&tm1, 0, sizeof tm1);
  memset(&tm2, 0, sizeof tm2);
  if (int rc = encode_sources(&tm1, ST, pl.M, g->nk, g->ntau, H)) return rc;
  if (int rc = encode_sources(&tm2, SP, pl.M, g->nk, g->ntau, H)) return rc;
  {
    ProfScope prof(GCAMB_K_WEIGHTS, st);
    const size_t rows = (size_t)g->nk * pl.mpad;
    te_weights_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(Pk, g->d_wk, g->d_k, g->d_tau, g->tau0, xlo,
                                                                      g->d_wtau, SP, pl.M, g->nk, g->ntau, pl.mpad, wp,
                                                                      tail);
  }
  if (pl.nitems > 0) {
    int *ctr = reinterpret_cast<int *>(ws + pl.off_ctr);
    // the row of l = 2 if the first l-tile holds it (TMEM lane of the epilogue)
    const int r2 = (g->lmin <= 2 && g->lmax >= 2 && g->rowof[2 - g->lmin] >= 0 && g->rowof[2 - g->lmin] < kTileL)
                       ? g->rowof[2 - g->lmin]
                       : -1;
    TcParams prm{static_cast<const char *>(t.d_data), nullptr, t.d_off, t.d_nkb, nullptr, wp, tail, ix2, r2,
                 pl.items(B), ctr, pl.nitems, pl.ksub, pl.chain >= 1 ? 1 : 0, part, device_error_flag(), g->nlt, pl.n_mt, pl.nkbs, pl.mpad};
    if (!prm.err) return fail(GCAMB_ECUDA, "los_cl_te: error flag allocation");
    if (int rc = launch_tc_kernel<NT, kBF16, true, 1>(g, pl, tm1, tm2, prm, st)) return rc;
  }
  dim3 rgrid(H, pl.ntile);
  ProfScope prof(GCAMB_K_REDUCE, st);
  reduce_te_kernel<<<rgrid, 128, 0, st>>>(part, B + pl.o_tile_ptr, B + pl.o_tile_items, H, pl.n_mt, pl.M, g->nl,
                                          g->d_lrow, 1, ClTT, ClEE, ClTE);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "los_cl_te: launch");
  return GCAMB_OK;
}

// A pair of kernel grids X, Y with the same layout: C^XX, C^YY, C^XY of the
// sources SX (with X's table) and SY (with Y's table), e.g. tensor T and E.
template <int NT>
int launch_tc_pair(const gcamb_grid *gx, const gcamb_grid *gy, const TcPlan &pl, const float *SX, const float *SY,
                   const double *Pk, double *ClXX, double *ClYY, double *ClXY, char *ws, cudaStream_t st) {
  constexpr int H = NT / 2;
  const Table &tx = gx->tab[GCAMB_BF16X3], &ty = gy->tab[GCAMB_BF16X3];
  float *wp = reinterpret_cast<float *>(ws + pl.off_wp);
  float *tail = reinterpret_cast<float *>(ws + pl.off_sc);
  float *part = reinterpret_cast<float *>(ws + pl.off_part);
  const int *B = pl.d_blob;
  CUtensorMap tm1, tm2;
  memset(&tm1, 0, sizeof tm1);
  memset(&tm2, 0, sizeof tm2);
  if (int rc = encode_sources(&tm1, SX, pl.M, gx->nk, gx->ntau, H)) return rc;
  if (int rc = encode_sources(&tm2, SY, pl.M, gx->nk, gx->ntau, H)) return rc;
  {
    ProfScope prof(GCAMB_K_WEIGHTS, st);
    const size_t rows = (size_t)gx->nk * pl.mpad;
    // weights; no small-x tails (the kernel tables hold the series): x_lo < 0
    te_weights_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(Pk, gx->d_wk, gx->d_k, gx->d_tau, gx->tau0, -1.0,
                                                                      gx->d_wtau, SY, pl.M, gx->nk, gx->ntau, pl.mpad,
                                                                      wp, tail);
  }
  if (pl.nitems > 0) {
    int *ctr = reinterpret_cast<int *>(ws + pl.off_ctr);
    TcParams prm{static_cast<const char *>(tx.d_data), static_cast<const char *>(ty.d_data), tx.d_off, tx.d_nkb,
                 nullptr, wp, tail, nullptr, -1, pl.items(B), ctr, pl.nitems, pl.ksub, pl.chain >= 1 ? 1 : 0, part, device_error_flag(), gx->nlt,
                 pl.n_mt, pl.nkbs, pl.mpad};
    if (!prm.err) return fail(GCAMB_ECUDA, "los_cl_pair: error flag allocation");
    if (int rc = launch_tc_kernel<NT, kBF16, true, 2>(gx, pl, tm1, tm2, prm, st)) return rc;
  }
  dim3 rgrid(H, pl.ntile);
  ProfScope prof(GCAMB_K_REDUCE, st);
  reduce_te_kernel<<<rgrid, 128, 0, st>>>(part, B + pl.o_tile_ptr, B + pl.o_tile_items, H, pl.n_mt, pl.M, gx->nl,
                                          gx->d_lrow, 0, ClXX, ClYY, ClXY);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "los_cl_pair: launch");
  return GCAMB_OK;
}

}  // namespace

int launch_los_cl_pair(const gcamb_grid *gx, const gcamb_grid *gy, const float *SX, const float *SY,
                       const double *Pk, int M, double *ClXX, double *ClYY, double *ClXY, void *ws, size_t ws_bytes,
                       cudaStream_t st) {
  const Table &tx = gx->tab[GCAMB_BF16X3], &ty = gy->tab[GCAMB_BF16X3];
  if (gx->k != gy->k || gx->tau != gy->tau || gx->tau0 != gy->tau0 || gx->lrow != gy->lrow || tx.nkb != ty.nkb ||
      tx.off != ty.off)
    return fail(GCAMB_EINVAL, "los_cl_pair: the two grids must share k, tau, tau0, the multipoles and the table layout");
  int rc = 0;
  TcPlan *pl = get_plan_te(gx, M, &rc);
  if (!pl) return rc ? rc : fail(GCAMB_ECUDA, "los_cl_pair: plan");
  if (ws_bytes < pl->ws_bytes) return fail(GCAMB_EINVAL, "los_cl_pair: workspace too small");
  char *w = static_cast<char *>(ws);
  return pl->NT == 32 ? launch_tc_pair<64>(gx, gy, *pl, SX, SY, Pk, ClXX, ClYY, ClXY, w, st)
                      : launch_tc_pair<128>(gx, gy, *pl, SX, SY, Pk, ClXX, ClYY, ClXY, w, st);
}

size_t los_cl_te_workspace_bytes(const gcamb_grid *g, int M) {
  int rc = 0;
  TcPlan *p = get_plan_te(g, M, &rc);
  return p ? p->ws_bytes : 0;
}

int launch_los_cl_te(const gcamb_grid *g, const float *ST, const float *SP, const double *Pk, int M, double *ClTT,
                     double *ClEE, double *ClTE, void *ws, size_t ws_bytes, cudaStream_t st) {
  double xlo = 0.0;
  if (emode_x_lo(g, &xlo)) return fail(GCAMB_EINVAL, "los_cl_te: eps_cut too large for the l = 2 limit");
  int rc = 0;
  TcPlan *pl = get_plan_te(g, M, &rc);
  if (!pl) return rc ? rc : fail(GCAMB_ECUDA, "los_cl_te: plan");
  if (ws_bytes < pl->ws_bytes) return fail(GCAMB_EINVAL, "los_cl_te: workspace too small");
  char *w = static_cast<char *>(ws);
  return pl->NT == 32 ? launch_tc_te<64>(g, *pl, ST, SP, Pk, ClTT, ClEE, ClTE, w, xlo, st)
                      : launch_tc_te<128>(g, *pl, ST, SP, Pk, ClTT, ClEE, ClTE, w, xlo, st);
}

size_t los_cl_workspace_bytes(const gcamb_grid *g, int M, int mode) {
  if (!g->tab[mode].built) {
    // without the table: an upper bound from the extents
    const int nt = pick_nt(M), n_mt = (M + nt - 1) / nt;
    const ModeLayout lay = mode_layout(mode);
    const size_t nkbs = (g->ntau + lay.kb - 1) / lay.kb;
    const size_t sp_bytes = (size_t)g->nk * n_mt * nkbs * 256 * nt;
    const size_t wp_bytes = (size_t)g->nk * n_mt * nt * sizeof(float);
    const size_t max_items = (size_t)g->nk * (g->nlt + 1) * n_mt;  // partials: LP = 2 pads an odd tile count
    return align256(sp_bytes) + align256(wp_bytes) + align256(max_items * nt * 128 * sizeof(float));
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
  return launch_plan(g, *pl, S, Pk, Cl, static_cast<char *>(ws), st);
}

// Fixed-buffer variant for gcamb_los_cl_noalloc: the plan is computed on the
// host and its integer blob, the split sources, the weights and the chunk
// partials all live in the caller's buffer `scratch` (no device allocation).
size_t los_cl_fixed_bytes(const gcamb_grid *g, int M, int mode) {
  TcPlan pl;
  plan_build(g, M, mode, pick_nt(M), nullptr, nullptr, pl);
  return blob_bytes(pl) + pl.ws_bytes;
}

int launch_los_cl_fixed(const gcamb_grid *g, const float *S, const double *Pk, int M, int mode, double *Cl,
                        char *scratch, size_t cap, int *status, cudaStream_t st) {
  TcPlan pl;
  plan_build(g, M, mode, pick_nt(M), nullptr, nullptr, pl);
  const size_t b_blob = blob_bytes(pl);
  const size_t need = b_blob + pl.ws_bytes;
  if (need > cap)
    return fail(GCAMB_EINVAL, "los_cl_noalloc: needs " + std::to_string(need) + " bytes of scratch, the fixed buffer holds " +
                                  std::to_string(cap) + "; use gcamb_los_cl with a caller workspace");
  pl.d_blob = reinterpret_cast<int *>(scratch);
  // copies from pageable memory return once the host data is staged, so the
  // plan may go out of scope when this function returns
  cudaError_t e = cudaMemcpyAsync(pl.d_blob, pl.blob.data(), pl.blob.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "los_cl_noalloc: plan upload");
  // without a status word a timeout is reported through the library's error flag
  return launch_plan(g, pl, S, Pk, Cl, scratch + b_blob, st, status, status != nullptr);
}

void drop_plans(const gcamb_grid *g) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  for (auto it = g_plans.begin(); it != g_plans.end();) {
    if (it->first == g) {
      it->second->release();
      delete it->second;
      it = g_plans.erase(it);
    } else {
      ++it;
    }
  }
}

}  // namespace gcamb

// ------------------------------------------------------------------ plans (uneven batches)
//
// A gcamb_plan fixes a batch's composition (per-source l_max and k prefix),
// builds the work list once, can pick the source-tile width by timing the
// candidates on the first launch (autotuner, optionally cached on disk), and
// replays its three launches as one CUDA graph.

namespace gcamb {
namespace {

// The autotuner's candidates: source-tile width x l-tiles per item x work
// items (k-aligned at 16 or 8 k, or of equal cost, with the tail cut; and
// k-aligned at 16 k without it); at most kMaxCand.
constexpr int kMaxCand = 24;

struct Cand {
  int nt;
  PlanCfg cfg;
};

std::vector<Cand> tune_candidates(int M, int mode) {
  std::vector<Cand> out;
  for (int nt : {64, 128, 256}) {
    if (nt > 128 && M <= 128) continue;  // one tile would hold the whole batch at 128
    for (int lp : {2, 1}) {
      if (lp == 2 && (nt > 128 || mode == GCAMB_TF32X3)) continue;
      // (kalign, tail cut): 16, 8 and equal-cost items with the tail cut, 16 without
      const int ka[4] = {16, 8, 0, 16};
      for (int v = 0; v < 4; ++v) {
        Cand c{nt, PlanCfg()};
        c.cfg.lp = lp;
        c.cfg.kalign = ka[v];
        c.cfg.tail_frac = v == 3 ? 0.0 : 0.1;
        c.cfg.tail_parts = v == 3 ? 1 : 4;
        c.cfg.per_cta = 4;
        out.push_back(c);
      }
    }
  }
  return out;
}

uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
  const unsigned char *c = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace
}  // namespace gcamb

struct gcamb_plan {
  const gcamb_grid *g = nullptr;
  int M = 0, mode = 0;
  bool plain = false;                       // GCAMB_PLAIN32: the plain kernels, chunks of sources
  int *d_lmax = nullptr, *d_nk = nullptr;   // plain: device copies of the per-source l_max, k prefix
  bool tune = false, tuned = false;
  std::vector<int> lmax_c, nk_c;
  gcamb::TcPlan cand[gcamb::kMaxCand];
  gcamb::Cand spec[gcamb::kMaxCand];
  bool have[gcamb::kMaxCand] = {};
  int ncand = 0;
  int chosen = -1;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;  // private stream the graph is captured on
  const void *bS = nullptr, *bP = nullptr, *bC = nullptr, *bW = nullptr;
  int64_t captures = 0, replays = 0;
  std::string key;
};

namespace gcamb {
namespace {

std::string tune_cache_path() {
  const char *e = getenv("GCAMB_TUNE_CACHE");
  return e ? std::string(e) : std::string();
}

// One JSON object per line: {"key": "...", "nt": 128, "lp": 2, "tail_frac":
// 0.1, "tail_parts": 4, "per_cta": 4, "kalign": 16, "ms": 1.234}; the last
// line with the key wins.
bool tune_cache_lookup(const std::string &key, Cand *c) {
  const std::string path = tune_cache_path();
  if (path.empty()) return false;
  FILE *f = fopen(path.c_str(), "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  auto num = [](const std::string &s, const char *name, double *v) {
    const std::string pat = std::string("\"") + name + "\": ";
    const size_t n = s.find(pat);
    if (n == std::string::npos) return false;
    *v = atof(s.c_str() + n + pat.size());
    return true;
  };
  while (fgets(line, sizeof line, f)) {
    const std::string s(line);
    const size_t k = s.find("\"key\": \"");
    if (k == std::string::npos) continue;
    const size_t b = k + 8, e = s.find('"', b);
    if (e == std::string::npos || s.substr(b, e - b) != key) continue;
    double nt, lp, tf, tp, pc, ka;
    if (num(s, "nt", &nt) && num(s, "lp", &lp) && num(s, "tail_frac", &tf) && num(s, "tail_parts", &tp) &&
        num(s, "per_cta", &pc) && num(s, "kalign", &ka) && (nt == 64 || nt == 128 || nt == 256) &&
        (lp == 1 || lp == 2) && tf >= 0 && tf <= 1 && tp >= 1 && tp <= 64 && pc >= 1 && pc <= 64 && ka >= 0 &&
        ka <= kKChunkMax) {
      c->nt = (int)nt;
      c->cfg.lp = (int)lp;
      c->cfg.tail_frac = tf;
      c->cfg.tail_parts = (int)tp;
      c->cfg.per_cta = (int)pc;
      c->cfg.kalign = (int)ka;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void tune_cache_store(const std::string &key, const Cand &c, double ms) {
  const std::string path = tune_cache_path();
  if (path.empty()) return;
  FILE *f = fopen(path.c_str(), "a");
  if (!f) return;
  fprintf(f, "{\"key\": \"%s\", \"nt\": %d, \"lp\": %d, \"tail_frac\": %.3f, \"tail_parts\": %d, "
          "\"per_cta\": %d, \"kalign\": %d, \"ms\": %.6f}\n",
          key.c_str(), c.nt, c.cfg.lp, c.cfg.tail_frac, c.cfg.tail_parts, c.cfg.per_cta, c.cfg.kalign, ms);
  fclose(f);
}

int plan_time(gcamb_plan *p, int c, const float *S, const double *Pk, double *Cl, char *ws, cudaStream_t st,
              float *ms) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return fail(GCAMB_ECUDA, "plan: event");
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return fail(GCAMB_ECUDA, "plan: event");
  }
  int rc = launch_plan(p->g, p->cand[c], S, Pk, Cl, ws, st);  // warm-up
  if (!rc) {
    cudaEventRecord(a, st);
    for (int r = 0; r < 2 && !rc; ++r) rc = launch_plan(p->g, p->cand[c], S, Pk, Cl, ws, st);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(ms, a, b);
    *ms *= 0.5f;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

}  // namespace
}  // namespace gcamb

using namespace gcamb;

extern "C" {

int gcamb_plan_create(gcamb_grid *g, int M, const int *lmax_m, const int *nk_m, int mode, int tune,
                      gcamb_plan **out) {
  if (!out) return fail(GCAMB_EINVAL, "plan_create: out is NULL");
  *out = nullptr;
  if (!g) return fail(GCAMB_EINVAL, "plan_create: NULL grid");
  if (mode != GCAMB_BF16X3 && mode != GCAMB_TF32X3 && mode != GCAMB_F16X3 && mode != GCAMB_PLAIN32)
    return fail(GCAMB_EINVAL, "plan_create: mode must be GCAMB_BF16X3, GCAMB_F16X3, GCAMB_TF32X3 or GCAMB_PLAIN32");
  if (M < 1) return fail(GCAMB_EINVAL, "plan_create: M must be >= 1");
  if (!g->tab[mode].built) return fail(GCAMB_ESTATE, "plan_create: build the table for this mode first");
  if ((lmax_m == nullptr) != (nk_m == nullptr))
    return fail(GCAMB_EINVAL, "plan_create: give both lmax_m and nk_m, or neither");
  for (int m = 0; lmax_m && m < M; ++m) {
    if (lmax_m[m] < g->lmin || lmax_m[m] > g->lmax)
      return fail(GCAMB_EINVAL, "plan_create: lmax_m outside the grid's [lmin, lmax]");
    if (nk_m[m] < 1 || nk_m[m] > g->nk) return fail(GCAMB_EINVAL, "plan_create: nk_m outside [1, nk]");
  }
  gcamb_plan *p = new (std::nothrow) gcamb_plan();
  if (!p) return fail(GCAMB_ENOMEM, "plan_create: host allocation");
  p->g = g;
  p->M = M;
  p->mode = mode;
  p->tune = tune != 0;
  if (lmax_m) {
    p->lmax_c.assign(lmax_m, lmax_m + M);
    p->nk_c.assign(nk_m, nk_m + M);
  }
  if (mode == GCAMB_PLAIN32) {
    // FP32 on the plain kernels: per-source prefixes on the device, no work list
    p->plain = true;
    if (!lmax_m) {
      p->lmax_c.assign(M, g->lmax);
      p->nk_c.assign(M, g->nk);
    }
    cudaError_t e = cudaMalloc(&p->d_lmax, M * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_nk, M * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_lmax, p->lmax_c.data(), M * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_nk, p->nk_c.data(), M * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      const int rc = cuda_fail(e, "plan_create: per-source arrays");
      gcamb_plan_destroy(p);
      return rc;
    }
    p->chosen = 0;
    *out = p;
    return GCAMB_OK;
  }
  // the key identifies grid, batch and device for the tile cache
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, g->k.data(), g->k.size() * sizeof(double));
  h = fnv1a(h, g->tau.data(), g->tau.size() * sizeof(double));
  h = fnv1a(h, g->lrow.data(), g->lrow.size() * sizeof(int));
  h = fnv1a(h, &g->K, sizeof(double));
  if (lmax_m) {
    h = fnv1a(h, lmax_m, M * sizeof(int));
    h = fnv1a(h, nk_m, M * sizeof(int));
  }
  char kb[256];
  snprintf(kb, sizeof kb, "v3|sm%d|%d|%d|%d|%d|%g|%d|%d|%016llx", num_sms(), g->nk, g->ntau, g->lmin, g->lmax,
           g->eps_cut, M, mode, (unsigned long long)h);
  p->key = kb;
  // candidates: the cached choice, every tuning candidate, or the heuristic
  // width with the default settings (and the environment's switches)
  Cand cached{};
  const bool hit = p->tune && tune_cache_lookup(p->key, &cached);
  std::vector<Cand> list;
  if (hit) list.push_back(cached);
  else if (p->tune) list = tune_candidates(M, mode);
  else list.push_back(Cand{pick_nt(M), PlanCfg()});
  const bool defaults = !p->tune;  // heuristic plans keep the environment's switches (GCAMB_TC_LP, _TAIL)
  for (size_t c = 0; c < list.size() && (int)c < kMaxCand; ++c) {
    plan_build(g, M, mode, list[c].nt, lmax_m, nk_m, p->cand[c], false, defaults ? nullptr : &list[c].cfg,
               defaults);  // a default plan cuts its items as gcamb_los_cl's does
    int rc = upload_blob(p->cand[c]);
    if (rc) {
      gcamb_plan_destroy(p);
      return rc;
    }
    p->spec[c] = list[c];
    p->have[c] = true;
    p->ncand = (int)c + 1;
  }
  if (!p->tune || hit) p->chosen = 0;
  if (hit) p->tuned = true;
  *out = p;
  return GCAMB_OK;
}

int gcamb_plan_destroy(gcamb_plan *p) {
  if (!p) return GCAMB_OK;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->cap) cudaStreamDestroy(p->cap);
  cudaFree(p->d_lmax);
  cudaFree(p->d_nk);
  for (auto &c : p->cand) c.release();
  delete p;
  return GCAMB_OK;
}

int gcamb_plan_workspace(const gcamb_plan *p, size_t *bytes) {
  if (!p || !bytes) return fail(GCAMB_EINVAL, "plan_workspace: NULL argument");
  size_t b = 0;
  if (p->plain) b = plain_plan_workspace_bytes(p->g, p->M);
  for (int c = 0; c < p->ncand; ++c)
    if (p->have[c]) b = std::max(b, p->cand[c].ws_bytes);
  *bytes = b;
  return GCAMB_OK;
}

int gcamb_plan_info(const gcamb_plan *p, int64_t *info) {
  if (!p || !info) return fail(GCAMB_EINVAL, "plan_info: NULL argument");
  const TcPlan *c = (p->chosen >= 0 && !p->plain) ? &p->cand[p->chosen] : nullptr;
  info[0] = c ? c->NT : 0;
  info[1] = c ? c->nitems : (p->plain ? (p->M + 15) / 16 : 0);  // plain: source chunks
  info[2] = c ? c->nctas : 0;
  info[3] = p->captures;
  info[4] = p->replays;
  info[5] = p->tuned ? 1 : 0;
  info[6] = p->M;
  info[7] = c ? (int64_t)c->ws_bytes : (p->plain ? (int64_t)plain_plan_workspace_bytes(p->g, p->M) : 0);
  info[8] = c && c->fused ? 1 : 0;
  info[9] = c ? c->lp : 0;
  info[10] = c ? c->per_cta : 0;
  info[11] = c ? c->tail : 0;
  info[12] = c ? c->kalign : 0;
  return GCAMB_OK;
}

int gcamb_plan_launch(gcamb_plan *p, const float *S, const double *Pk, double *Cl, void *ws, size_t ws_bytes,
                      void *stream) {
  if (!p) return fail(GCAMB_EINVAL, "plan_launch: NULL plan");
  if (!S || !Pk || !Cl || !ws) return fail(GCAMB_EINVAL, "plan_launch: NULL pointer");
  size_t need = 0;
  gcamb_plan_workspace(p, &need);
  if (ws_bytes < need) return fail(GCAMB_EINVAL, "plan_launch: workspace too small");
  if (!p->g->tab[p->mode].built) return fail(GCAMB_ESTATE, "plan_launch: the grid's table is gone");
  cudaStream_t st = (cudaStream_t)stream;
  char *w = static_cast<char *>(ws);
  if (!device_error_flag()) return fail(GCAMB_ECUDA, "plan_launch: error flag allocation");
  if (!p->plain && p->chosen < 0) {
    // autotune: time every candidate tile on these inputs, keep the fastest
    float best = 1e30f;
    int bi = -1;
    for (int c = 0; c < p->ncand; ++c) {
      if (!p->have[c]) continue;
      float ms = 0.f;
      int rc = plan_time(p, c, S, Pk, Cl, w, st, &ms);
      if (rc) return rc;
      if (ms < best) {
        best = ms;
        bi = c;
      }
    }
    if (bi < 0) return fail(GCAMB_ESTATE, "plan_launch: no candidate tile");
    p->chosen = bi;
    p->tuned = true;
    tune_cache_store(p->key, p->spec[bi], best);
    for (int c = 0; c < p->ncand; ++c)
      if (c != bi && p->have[c]) {
        p->cand[c].release();
        p->have[c] = false;
      }
  }
  const bool rebind = !p->exec || p->bS != S || p->bP != Pk || p->bC != Cl || p->bW != ws;
  if (rebind) {
    if (p->exec) {
      cudaGraphExecDestroy(p->exec);
      p->exec = nullptr;
    }
    // capture on a private stream (the legacy default stream cannot be
    // captured); the graph is then launched on the caller's stream
    if (!p->cap) {
      cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        p->cap = nullptr;
        return cuda_fail(e, "plan_launch: capture stream");
      }
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "plan_launch: begin capture");
    const int rc = p->plain ? launch_plain_plan(p->g, S, Pk, p->M, p->lmax_c.data(), p->nk_c.data(), p->d_lmax,
                                                p->d_nk, Cl, w, p->cap)
                            : launch_plan(p->g, p->cand[p->chosen], S, Pk, Cl, w, p->cap);
    e = cudaStreamEndCapture(p->cap, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "plan_launch: end capture");
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      p->exec = nullptr;
      return cuda_fail(e, "plan_launch: instantiate");
    }
    p->bS = S;
    p->bP = Pk;
    p->bC = Cl;
    p->bW = ws;
    ++p->captures;
  }
  cudaError_t e = cudaGraphLaunch(p->exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "plan_launch: graph launch");
  ++p->replays;
  return GCAMB_OK;
}

}  // extern "C"
