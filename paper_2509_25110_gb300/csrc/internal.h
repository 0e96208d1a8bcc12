// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gcamb.h"

namespace gcamb {

constexpr int kTileL = 128;      // multipoles per l-tile (UMMA M)
constexpr int kMaxL = 20000;
constexpr int kNumModes = 5;

// Table layout of one mode: blocks of [planes][128 rows][kb cols], one block
// per (k, l-tile, tau-block of kb nodes).  Rows are multipoles, columns tau.
// Split modes store their rows in the swizzled order the tensor cores read
// K-major operands in: bf16/fp16 64-byte rows (32 tau) in the 64-byte
// swizzle (16-byte chunk index XOR (row / 2) % 4), tf32 128-byte rows
// (32 tau) in the 128-byte swizzle (chunk index XOR row % 8).
struct ModeLayout {
  int kb;        // tau nodes per block
  int planes;    // 1 (plain) or 2 (hi, lo)
  int esize;     // bytes per element
  bool swizzle;  // 128B swizzle within each 8-row group
  size_t block_bytes() const { return (size_t)planes * kTileL * kb * esize; }
};

inline ModeLayout mode_layout(int mode) {
  switch (mode) {
    case GCAMB_PLAIN64: return {64, 1, 8, false};
    case GCAMB_PLAIN32: return {64, 1, 4, false};
    case GCAMB_BF16X3: return {32, 2, 2, true};
    case GCAMB_TF32X3: return {32, 2, 4, true};
    case GCAMB_F16X3: return {32, 2, 2, true};
    default: return {0, 0, 0, false};
  }
}

struct Table {
  bool built = false;
  ModeLayout lay{};
  std::vector<int32_t> nkb;   // [nk][nlt] tau-blocks stored per (k, l-tile)
  std::vector<int64_t> off;   // [nk][nlt] first block of the chunk
  int64_t nblocks = 0;
  void *d_data = nullptr;     // table blocks
  int32_t *d_nkb = nullptr;
  int64_t *d_off = nullptr;
  size_t bytes = 0;
  int scale_exp = 0;          // F16X3: entries are w_i j_l 2^scale_exp
  // d_data from the driver's virtual-memory API with generic compression
  // (table_alloc): the allocation handle and the mapped size; 0 for cudaMalloc
  unsigned long long vmm = 0;
  size_t mapped = 0;
};

// Table memory: compressible device memory where the device grants it
// (GCAMB_TABLE_COMPRESS=0 asks for cudaMalloc), else cudaMalloc.  table_free
// waits for the device before it unmaps, as cudaFree does.
int table_alloc(Table &t, size_t bytes);
void table_free(Table &t);

}  // namespace gcamb

struct gcamb_grid {
  int nk = 0, ntau = 0, lmin = 0, lmax = 0, nl = 0, nlt = 0;
  // multipole of each table row (output index): lmin + r, or the caller's
  // sampled list; rowof[l - lmin] is the row of l or -1 (sampled grids)
  std::vector<int> lrow, rowof;
  bool lsampled = false;
  int *d_lrow = nullptr, *d_rowof = nullptr;
  // curvature: 0 flat (j_l), 1 open (K < 0), 2 closed (K > 0): hyperspherical
  // Bessel functions with beta = k / rk, chi = rk (tau0 - tau), rk = sqrt|K|;
  // the tau-prefixes of a curved grid come from a device pass (ext_ready)
  int kernel = 0;  // 0: j_l; GCAMB_KERNEL_* (flat grids): the table holds that kernel
  int curved = 0;
  double K = 0.0, rk = 0.0;
  bool ext_ready = true;
  double tau0 = 0.0, eps_cut = 1e-30;
  std::vector<double> k, tau, wtau, wk;
  std::vector<int32_t> ext;       // [nk][nlt] active tau-prefix per (k, l-tile)
  std::vector<double> xstart;     // [nxs] Miller start thresholds per order
  // [nl] per row: Watson threshold below which |j_l| < eps_cut (flat grids;
  // empty on curved ones)
  std::vector<double> xthr;
  int64_t active = 0;             // active (l,k,tau) entries
  // device copies (made lazily)
  double *d_k = nullptr, *d_tau = nullptr, *d_wtau = nullptr, *d_wk = nullptr;
  double *d_xstart = nullptr;
  double *d_xthr = nullptr;
  int nxs = 0;
  gcamb::Table tab[gcamb::kNumModes];
};

namespace gcamb {

// Thread-local error text; returns the code for convenient `return fail(...)`.
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
int *device_error_flag();  // device pointer of the mapped error word

// Device-side error code written to the flag word (or a caller's status
// word) when a bounded wait gives up: the public status itself.
constexpr int kDevErrTimeout = GCAMB_ETIMEOUT;

int ensure_device_grid(gcamb_grid *g);

// Bessel table construction (bessel.cu).
int launch_bessel_table(gcamb_grid *g, int mode, cudaStream_t st);
int launch_sph_bessel(const double *x, int n, int lmax, double *out, cudaStream_t st);

// Plain FP64/FP32 path (plain.cu).
int launch_los_plain(const gcamb_grid *g, const void *S, int M, int mode, void *Delta, cudaStream_t st,
                     bool emode = false);
int launch_los_tensor(const gcamb_grid *g, const void *ST, const void *SP, int M, int mode, void *DT, void *DE,
                      void *DB, cudaStream_t st);
// Source interpolation onto the grid's k nodes (interp.cu).
size_t interp_workspace_bytes(int M, int nk_in, int ntau, int nk_out);
int launch_interp_sources(const double *k_in, int nk_in, const void *S_in, int M, int ntau, int dtype,
                          const gcamb_grid *g, void *S_out, void *ws, size_t ws_bytes, cudaStream_t st);
// E-mode small-x cut x_lo of the grid (plain.cu); -1 if it would exceed 0.2.
int emode_x_lo(const gcamb_grid *g, double *x_lo);
int launch_cl_cross(const gcamb_grid *g, const void *DX, const void *DY, int d_dtype, const double *Pk, int M,
                    double *Cl, cudaStream_t st);
int launch_cl(const gcamb_grid *g, const void *Delta, int d_dtype, const double *Pk, int M, double *Cl,
              cudaStream_t st);
// Uneven batch in FP32 on the plain kernels (plain.cu): per-source k prefix
// and l_max (host copies lmax_c, nk_c; device copies d_lmax, d_nk).
size_t plain_plan_workspace_bytes(const gcamb_grid *g, int M);
int launch_plain_plan(const gcamb_grid *g, const float *S, const double *Pk, int M, const int *lmax_c,
                      const int *nk_c, const int *d_lmax, const int *d_nk, double *Cl, void *ws, cudaStream_t st);

// Tensor-core batched path (tc.cu).
size_t los_cl_workspace_bytes(const gcamb_grid *g, int M, int mode);
size_t los_cl_te_workspace_bytes(const gcamb_grid *g, int M);
int launch_los_cl_pair(const gcamb_grid *gx, const gcamb_grid *gy, const float *SX, const float *SY,
                       const double *Pk, int M, double *ClXX, double *ClYY, double *ClXY, void *ws, size_t ws_bytes,
                       cudaStream_t st);
int launch_los_cl_te(const gcamb_grid *g, const float *ST, const float *SP, const double *Pk, int M, double *ClTT,
                     double *ClEE, double *ClTE, void *ws, size_t ws_bytes, cudaStream_t st);
int launch_los_cl(const gcamb_grid *g, const float *S, const double *Pk, int M, int mode, double *Cl,
                  void *ws, size_t ws_bytes, cudaStream_t st);
void drop_plans(const gcamb_grid *g);
size_t los_cl_fixed_bytes(const gcamb_grid *g, int M, int mode);
int launch_los_cl_fixed(const gcamb_grid *g, const float *S, const double *Pk, int M, int mode, double *Cl,
                        char *scratch, size_t cap, int *status, cudaStream_t st);

// Probes (probe.cu).
int run_probe_flops(int what, double *flops);
int run_wait_selftest(int *status, cudaStream_t st);

// Event tracer: brackets one kernel launch when profiling is on.
struct ProfScope {
  int id;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(int id, cudaStream_t st);
  ~ProfScope();
};

// Watson's bound (A&S 9.1.63) on log|j_l(x)| for x < l + 1/2.
double log_watson_bound(int l, double x);
// Smallest x > 0 at which the bound on |j_l| reaches `logeps` (0 for l == 0).
double watson_threshold(int l, double logeps);

}  // namespace gcamb
