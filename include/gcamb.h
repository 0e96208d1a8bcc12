/*
 * gcamb.h -- C ABI of the GB300 line-of-sight projection library (libgcamb.so).
 *
 * The library computes, on one GPU, the two sums that the paper
 * (arXiv 2509.25110, "gCAMB") offloads and assembles:
 *
 *   Eq. (2), flat space, discretised on the conformal-time nodes tau_i:
 *       Delta_l(k) = sum_i w_i S(k, tau_i) j_l(k (tau0 - tau_i))
 *   Eq. (1), for X = Y = T, discretised on the wavenumber nodes k_j:
 *       C_l = 4 pi sum_j w_j P(k_j) Delta_l(k_j)^2
 *
 * w_i are trapezoid weights in tau and w_j trapezoid weights in u = ln k (the
 * dk/k measure of Eq. 1).  The paper does not state its quadrature; this is
 * the library's reading.  The paper's kernel phi_l is "related to spherical
 * Bessel functions" in flat space (Sec. 2.1); the library uses j_l.
 *
 * Conventions for every entry point:
 *  - Return value: GCAMB_OK (0) or a negative GCAMB_E* code.  The text of the
 *    last error of the calling thread is returned by gcamb_last_error().
 *    No C++ exception and no abort crosses this boundary.
 *  - Arrays documented "host" are read (or written) before the call returns.
 *  - Arrays documented "device" are caller-owned CUDA device memory, C
 *    contiguous in the stated layout; they must stay valid until the work
 *    enqueued on `stream` has finished.  The library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is enqueued asynchronously on it.  Errors raised on the
 *    device (a bounded wait that gave up) are reported by gcamb_sync().
 *  - Handles (gcamb_grid*) are owned by the library and released with the
 *    matching *_destroy call.
 */
#ifndef GCAMB_H
#define GCAMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define GCAMB_OK            0
#define GCAMB_EINVAL      (-1)  /* bad argument (size, order, pointer, mode) */
#define GCAMB_ENOMEM      (-2)  /* device or host allocation failed */
#define GCAMB_ECUDA       (-3)  /* a CUDA runtime call failed */
#define GCAMB_ESTATE      (-4)  /* call out of order, e.g. table not built for this mode */
#define GCAMB_EUNSUPPORTED (-5) /* feature not available on this device */
#define GCAMB_ETIMEOUT    (-6)  /* a device-side bounded wait gave up */

/* Arithmetic modes (the form in which the Bessel table is stored and the
 * tau-contraction of Eq. 2 is computed). */
#define GCAMB_PLAIN64 0  /* FP64 table, FP64 sums */
#define GCAMB_PLAIN32 1  /* FP32 table, FP32 sums */
#define GCAMB_BF16X3  2  /* tensor cores: bf16 hi/lo split, hi*hi + hi*lo + lo*hi, FP32 accumulate */
#define GCAMB_TF32X3  3  /* tensor cores: tf32 hi/lo split, same three products, FP32 accumulate */
#define GCAMB_F16X3   4  /* tensor cores: fp16 hi/lo split of power-of-two scaled operands, FP32 accumulate */

/* Element types of Delta arrays. */
#define GCAMB_F64 0
#define GCAMB_F32 1

/* Number of int64 fields written by gcamb_grid_info. */
#define GCAMB_INFO_N 8

typedef struct gcamb_grid gcamb_grid;

/* Library version string (static storage). */
const char *gcamb_version(void);

/* Text of the calling thread's last error ("" if none); valid until the next
 * gcamb call on the same thread. */
const char *gcamb_last_error(void);

/*
 * Creates the integration grid of Eqs. (1)-(2): the k nodes, the tau nodes,
 * tau0 and the multipole range l = lmin..lmax (every l, no l-sampling).
 * Plays the role of CAMB's IntegrationVars_init (Sec. 3.2).
 *
 *   k[nk]      host, strictly increasing, > 0                      [1/Mpc]
 *   tau[ntau]  host, strictly increasing, tau[ntau-1] <= tau0      [Mpc]
 *   lmin, lmax 0 <= lmin <= lmax <= 20000
 *   eps_cut    activity threshold (> 0, <= 1e-3; 0 selects 1e-30): for each
 *              (k, 128-multipole tile) only the tau-prefix on which Watson's
 *              bound (Abramowitz & Stegun 9.1.63) allows |j_l| >= eps_cut for
 *              some l of the tile is summed.  This prefix is Algorithm 1's
 *              n_min..n_max window.
 *   out        receives the handle.
 *
 * Computes the quadrature weights and the active extents on the host; the
 * host arrays are copied.  No device memory is touched (device copies are
 * made by the first call that needs them).  Errors: GCAMB_EINVAL for bad
 * sizes, non-increasing nodes, tau beyond tau0 or a NULL pointer.
 */
int gcamb_grid_create(const double *k, int nk, const double *tau, int ntau, double tau0,
                      int lmin, int lmax, double eps_cut, gcamb_grid **out);

/* Releases the grid, its tables and its device copies.  NULL is accepted. */
int gcamb_grid_destroy(gcamb_grid *g);

/*
 * Grid summary (host, int64[GCAMB_INFO_N]):
 *   [0] nk  [1] ntau  [2] nl = lmax-lmin+1  [3] n_ltile = ceil(nl/128)
 *   [4] active (l, k, tau) entries (sum over k and l of the per-l prefix)
 *   [5] stored (l, k, tau) entries of the PLAIN64 table (tile granularity)
 *   [6] lmin  [7] lmax
 */
int gcamb_grid_info(const gcamb_grid *g, int64_t *info);

/* Active tau-prefix length per (k, l-tile), host int32[nk][n_ltile]. */
int gcamb_grid_extents(const gcamb_grid *g, int32_t *ext);

/* Quadrature weights the grid uses (host): wtau[ntau] trapezoid in tau,
 * wk[nk] trapezoid in ln k.  Either pointer may be NULL. */
int gcamb_grid_weights(const gcamb_grid *g, double *wtau, double *wk);

/*
 * Builds (or rebuilds) the grid's table of w_i j_l(k (tau0 - tau_i)) over the
 * active extents, in the layout of `mode`, by an FP64 recurrence on the
 * device (Miller's backward recurrence above x = k(tau0-tau), the forward
 * recurrence at and below it).  This is the "calculation of the spherical
 * Bessel-function" inside the line-of-sight loop (Sec. 3.2), hoisted out of
 * it because the table is shared by all sources on the grid.
 * The table is device memory owned by the grid (size: gcamb_table_bytes).
 * Errors: GCAMB_EINVAL (mode), GCAMB_ENOMEM, GCAMB_ECUDA.
 */
int gcamb_bessel_table(gcamb_grid *g, int mode, void *stream);

/* Bytes the table of `mode` occupies (host size_t*). */
int gcamb_table_bytes(const gcamb_grid *g, int mode, size_t *bytes);

/*
 * Whether the built table of `mode` lives in compressible device memory
 * (host int*: 1 yes, 0 no).  The table kernels' output is the same either
 * way; compression only changes how the memory system moves the table's
 * zero-padded blocks (the rows of a 128-multipole tile beyond their own
 * tau-prefix, Algorithm 1's window per multipole) between DRAM and L2.
 * The library asks for it where the device supports generic compression;
 * GCAMB_TABLE_COMPRESS=0 in the environment asks for plain cudaMalloc.
 * Errors: GCAMB_EINVAL (NULL argument, unknown mode), GCAMB_ESTATE (table
 * not built).
 */
int gcamb_table_compressed(const gcamb_grid *g, int mode, int *compressed);

/*
 * Spherical Bessel functions by the table's device routine:
 *   x[n]              device double, x >= 0
 *   out[n][lmax+1]    device double, j_0..j_lmax at each x
 * Entries below 1e-300 in magnitude may be returned as 0.
 * Errors: GCAMB_EINVAL (n < 0, lmax < 0 or > 20000, NULL with n > 0).
 */
int gcamb_sph_bessel(const double *x, int n, int lmax, double *out, void *stream);

/*
 * Line-of-sight transfer, Eq. (2), for M sources on the grid (Algorithm 1:
 * every k, every l, the tau-window sum).
 *   S[M][nk][ntau]      device; double for GCAMB_PLAIN64, float for GCAMB_PLAIN32
 *   Delta[M][nk][nl]    device; same type as S; every entry is written
 *                       (zero where the whole tile is inactive)
 * Requires gcamb_bessel_table(g, mode) first (else GCAMB_ESTATE).
 * mode must be GCAMB_PLAIN64 or GCAMB_PLAIN32 (else GCAMB_EINVAL).
 */
int gcamb_los_transfer(const gcamb_grid *g, const void *S, int M, int mode, void *Delta, void *stream);

/*
 * E-mode polarisation transfer functions, Eq. (3) (Sec. 2.1), on the CUDA
 * cores, with the flat-space kernel
 *   eps_l(x) = sqrt((l+2)!/(l-2)!) j_l(x) / x^2   (l >= 2; 0 for l < 2):
 *   DeltaE[m][k][l - lmin] = sum_i w_i S_P[m][k][i] eps_l(k (tau0 - tau_i)).
 * It uses the same j_l table as gcamb_los_transfer (the x^-2 factor is
 * applied to the source, the prefactor to the row).  Nodes with x below a
 * small cut x_lo (x = 0 included; x_lo is 1e-12 or the largest x at which the
 * table may hold j_2 as zero, at most 0.2) contribute to l = 2 only, through
 * the power series of j_2(x)/x^2 (-> 1/15); for l >= 3 their terms are below
 * c_l x_lo^(l-2)/(2l+1)!!.  GCAMB_EINVAL if eps_cut is so large that x_lo
 * would exceed 0.2.  Arguments, layout, modes, dtypes and other errors as for
 * gcamb_los_transfer.
 */
int gcamb_los_transfer_e(const gcamb_grid *g, const void *SP, int M, int mode, void *DeltaE, void *stream);

/*
 * Tensor modes on the CUDA cores: the projection the paper runs a second time
 * for tensor perturbations (Sec. 3.1, 3.3; Sec. 2.1 says equations like
 * Eqs. (2)-(3) hold for them), with the flat-space line-of-sight kernels
 *   T: t_l(x) = sqrt((l+2)!/(l-2)!) j_l(x) / x^2        (source ST)
 *   E: e_l(x) = -j_l + j_l'' + 2 j_l/x^2 + 4 j_l'/x
 *             = (l (l-1)/x^2 - 2) j_l + 2 j_(l-1)/x     (source SP)
 *   B: b_l(x) = 2 j_l' + 4 j_l/x = 2 j_(l-1) - 2 (l-1) j_l/x   (source SP)
 * (l >= 2; 0 below).  The shared j_l table gives the sums D_p[l] =
 * sum_i w_i j_l S_P x^-p (p = 0, 1, 2) and the kernels combine rows l and
 * l-1 (for l = lmin >= 2, row l-1 from j_(l-1) = (2l+1)/x j_l - j_(l+1)).
 * Nodes below the small cut x_lo of gcamb_los_transfer_e take the power
 * series of the kernels for l = 2..5 (e_2 -> 4/5, t_2 -> sqrt(24)/15).
 *   ST, SP                [M][nk][ntau] device, FP64 (PLAIN64) or FP32 (PLAIN32)
 *   DeltaT, DeltaE, DeltaB [M][nk][nl] device, same dtype; DeltaT is also used
 *                         as scratch (the three must not overlap)
 * C_l (TT, EE, BB, TE of the tensor spectrum) follow from gcamb_cl and
 * gcamb_cl_cross with the tensor P(k).  Errors: as gcamb_los_transfer_e, and
 * GCAMB_EINVAL for lmin >= 2 with lmax == lmin.
 */
int gcamb_los_transfer_tensor(const gcamb_grid *g, const void *ST, const void *SP, int M, int mode, void *DeltaT,
                              void *DeltaE, void *DeltaB, void *stream);

/*
 * Kernel grids.  By default a grid's table holds w_i j_l (Eq. 2).  Before its
 * first table, a flat grid can be switched to one of the other kernels of the
 * line-of-sight projection, evaluated in FP64 while the table is built:
 *   GCAMB_KERNEL_EPS       c_l j_l(x) / x^2, c_l = sqrt((l+2)!/(l-2)!): the
 *                          E-mode kernel of Eq. (3) and the tensor T kernel
 *   GCAMB_KERNEL_TENSOR_E  (l(l-1)/x^2 - 2) j_l + 2 j_(l-1)/x (tensor E)
 *   GCAMB_KERNEL_TENSOR_B  2 j_(l-1) - 2 (l-1) j_l / x      (tensor B)
 * (zero below l = 2; the power series below the small-x cut of
 * gcamb_los_transfer_e; every tau node stays in the first l-tile when
 * lmin <= 5, since the l = 2 kernels do not vanish at x = 0).  Every path
 * that reads the table then projects with that kernel: gcamb_los_transfer,
 * gcamb_cl, gcamb_los_cl (the batched tensor-core path: one kernel grid per
 * field, no cancellation between j_l and j_(l-1) in split precision), plans,
 * sampled grids.  gcamb_los_transfer_e, gcamb_los_transfer_tensor and
 * gcamb_los_cl_te, which derive their kernels from j_l, reject kernel grids.
 * Errors: GCAMB_ESTATE (a table exists), GCAMB_EUNSUPPORTED (curved grid),
 * GCAMB_EINVAL.
 */
#define GCAMB_KERNEL_J 0
#define GCAMB_KERNEL_EPS 1
#define GCAMB_KERNEL_TENSOR_E 2
#define GCAMB_KERNEL_TENSOR_B 3
int gcamb_grid_set_kernel(gcamb_grid *g, int kernel);

/*
 * Curved space (the non-flat integration the paper names as its next step,
 * Sec. 2.1, 5): as gcamb_grid_create, with curvature K [Mpc^-2] != 0 and
 * the wavenumbers q[nq] of the curved-space modes; the kernel phi_l of
 * Eq. (2) becomes the hyperspherical Bessel function Phi^beta_l(chi),
 * beta = q / sqrt|K|, chi = sqrt|K| (tau0 - tau) (open space for K < 0,
 * closed for K > 0, where every beta must be an integer >= 3 and Phi_l = 0
 * for l >= beta).  Eq. (1)'s measure is unchanged (trapezoid in ln q).
 * gcamb_bessel_table evaluates Phi by its three-term recurrence (forward
 * below the turning order beta |sh chi|, Miller's downward recurrence above)
 * and, on the first build, finds each (q, l-tile) tau-prefix on the device
 * from where some |Phi_l| of the tile reaches eps_cut.  The temperature
 * paths (plain, batched, plans, emulator) take such grids; the E-mode and
 * tensor kernels are flat-space only (GCAMB_EUNSUPPORTED).
 */
int gcamb_grid_create_curved(const double *q, int nq, const double *tau, int ntau, double tau0, int lmin, int lmax,
                             double K, double eps_cut, gcamb_grid **out);

/*
 * Sampled multipoles (the output l-sampling of the paper's accuracy settings,
 * Sec. 3.1, Table 1: l_sample_boost = 50 computes every l).
 *
 * gcamb_grid_create_lsampled: as gcamb_grid_create, with the table rows,
 * transfer functions and C_l rows on the listed multipoles lval[0..nl)
 * (strictly increasing, 0..20000) instead of every l; lmin = lval[0],
 * lmax = lval[nl-1], and the row index r of every output holds l = lval[r].
 * Every path accepts such a grid except the tensor modes (GCAMB_EUNSUPPORTED:
 * they combine rows l and l-1).
 *
 * gcamb_l_sampling: a list for such a grid (host; lval NULL returns the
 * count in *n): every l below 20 boost, then steps of round(l / (20 boost)),
 * at most ceil(50 / boost); boost >= 50 keeps every l; lmax is always listed.
 *
 * gcamb_cl_interp: C_l of every multipole lmin..lmax from the sampled rows:
 * the natural cubic spline in l of l (l+1) C_l through the samples (FP64);
 * sampled multipoles are copied.  Cl_s [M][nl] device, Cl [M][lmax-lmin+1]
 * device, ws of gcamb_cl_interp_workspace bytes.
 */
int gcamb_grid_create_lsampled(const double *k, int nk, const double *tau, int ntau, double tau0, const int *lval,
                               int nl, double eps_cut, gcamb_grid **out);
int gcamb_l_sampling(int lmin, int lmax, double boost, int *lval, int *n);
int gcamb_cl_interp_workspace(const gcamb_grid *g, int M, size_t *bytes);
int gcamb_cl_interp(const gcamb_grid *g, const double *Cl_s, int M, double *Cl, void *ws, size_t ws_bytes,
                    void *stream);

/*
 * Source interpolation onto the grid's k nodes (the step that prepares the
 * sources before the projection, Sec. 3.3): the natural cubic spline in k of
 * every (source, tau) column (second derivatives zero at both ends), solved
 * and evaluated in the sources' precision (FP64 or FP32).
 *   k_in[nk_in]          host, strictly increasing, nk_in >= 2; the grid's k
 *                        range must lie inside [k_in[0], k_in[nk_in-1]]
 *   S_in[M][nk_in][ntau] device, dtype GCAMB_F64 or GCAMB_F32 (ntau: the grid's)
 *   S_out[M][nk][ntau]   device, same dtype
 *   ws, ws_bytes         device workspace of gcamb_interp_sources_workspace bytes
 * Errors: GCAMB_EINVAL (arguments), GCAMB_ECUDA.
 */
int gcamb_interp_sources_workspace(const gcamb_grid *g, int M, int nk_in, size_t *bytes);
int gcamb_interp_sources(const gcamb_grid *g, const double *k_in, int nk_in, const void *S_in, int M, int dtype,
                         void *S_out, void *ws, size_t ws_bytes, void *stream);

/*
 * Cross spectrum, Eq. (1) with X, Y in {T, E}:
 *   C^XY[m][l] = 4 pi sum_k w_k P[m][k] DX[m][k][l] DY[m][k][l]
 * DX, DY [M][nk][nl] device, both of d_dtype (GCAMB_F64 or GCAMB_F32);
 * Pk[M][nk], Cl[M][nl] device double.  Summed in FP64 in increasing k.
 */
int gcamb_cl_cross(const gcamb_grid *g, const void *DX, const void *DY, int d_dtype, const double *Pk, int M,
                   double *Cl, void *stream);

/*
 * C_l from transfer functions, Eq. (1) with X = Y = T:
 *   Delta[M][nk][nl]   device, d_dtype = GCAMB_F64 or GCAMB_F32
 *   Pk[M][nk]          device double, P_R(k) per source
 *   Cl[M][nl]          device double, C_l for l = lmin..lmax
 * Summed in FP64 in increasing k (deterministic).
 */
int gcamb_cl(const gcamb_grid *g, const void *Delta, int d_dtype, const double *Pk, int M,
             double *Cl, void *stream);

/*
 * Device workspace (bytes) that gcamb_los_cl needs for M sources in `mode`.
 */
int gcamb_los_cl_workspace(const gcamb_grid *g, int M, int mode, size_t *bytes);

/*
 * Fused, batched Eqs. (1)-(2) on the tensor cores for M sources sharing the
 * grid: per k, the tau-contraction D_k[l][m] = sum_i (w_i j_l)(k,tau_i) S_m(k,tau_i)
 * is a dense product over the active tau-blocks, computed from hi/lo splits
 * of both operands (three products, FP32 accumulate); D_k is squared,
 * weighted by 4 pi w_k P_m(k) and summed over k without being stored.
 * hi*hi is accumulated apart from hi*lo + lo*hi (two TMEM accumulators), so
 * the main chain takes a third of the accumulate steps.  Partial sums over
 * k-chunks of at most 16 nodes with stored blocks are FP32 (each within
 * 15 * 2^-24 of the exact sum of its positive terms, relative); the final sum
 * over chunks runs in a fixed order (deterministic) as a TwoSum pair of FP32
 * numbers, read out in FP64.  Two adjacent 128-multipole tiles share each loaded and split source
 * block (bf16/fp16 with 64- or 128-source tiles).  GCAMB_F16X3 scales the table by one power
 * of two per grid and each (k, source) row of S by its own power of two so
 * that both land in fp16's normal range; the scales are removed exactly.
 *   S[M][nk][ntau]   device float
 *   Pk[M][nk]        device double, >= 0 (a power spectrum; the epilogue
 *                    weights by sqrt(4 pi w_k P))
 *   Cl[M][nl]        device double
 *   ws, ws_bytes     device workspace of at least gcamb_los_cl_workspace bytes,
 *                    16-byte aligned (GCAMB_EINVAL otherwise)
 * mode: GCAMB_BF16X3, GCAMB_F16X3 or GCAMB_TF32X3; requires
 * gcamb_bessel_table(g, mode).  For GCAMB_F16X3 the per-row scale is clamped
 * to 2^-40..2^80, so rows whose largest |S| is below ~1e-20 lose precision.
 * M = 0 returns GCAMB_OK and writes nothing.
 * Environment (tuning switches, read when a plan is built; the results agree
 * within the bounds the tests state): GCAMB_TC_NT=64|128|256 source-tile
 * width; GCAMB_TC_FUSED=0 splits the sources in a separate pass instead of in
 * shared memory; GCAMB_TC_LP=1 one multipole tile per work item instead of two;
 * GCAMB_TC_KSUB=1..64 k nodes per FP32 chunk sum instead of 16 (1: every k's
 * term is its own partial, and C_l is the FP64 sum of the FP32 terms);
 * GCAMB_TC_CHAIN=0|1|2 chain records (a tile's hi*hi tau-sum spread over three
 * TMEM accumulators): none, where an item's second l-tile is idle (default),
 * or also l-tile 0 in items of its own; GCAMB_TC_TAIL=frac:parts the share of
 * the cost handed out last whose items are cut into parts (default 0.1:4);
 * GCAMB_TC_KALIGN=n work items end at multiples of n k nodes (0: items of
 * equal cost; default 12, or 6 where items of 12 k would give a CTA fewer
 * than four; gcamb_los_cl_noalloc keeps 12).
 * Errors: GCAMB_EINVAL, GCAMB_ESTATE, GCAMB_EUNSUPPORTED (device is not
 * sm_103), GCAMB_ECUDA; GCAMB_ETIMEOUT is reported by gcamb_sync.
 */
int gcamb_los_cl(const gcamb_grid *g, const float *S, const double *Pk, int M, int mode,
                 double *Cl, void *ws, size_t ws_bytes, void *stream);

/*
 * Temperature and E-mode polarisation together, batched on the tensor cores:
 * for M models sharing the grid, Eq. (2) for S_T and Eq. (3) for S_P (the
 * E-mode kernel eps_l(x) = c_l j_l(x)/x^2 of gcamb_los_transfer_e, with its
 * small-x treatment) and Eq. (1) for XY = TT, EE, TE, without storing Delta.
 * The two sources of a model are adjacent operand rows of one product with
 * the shared bf16 hi/lo table (the table is read once for both); the
 * polarisation rows are scaled by 1/x^2 while they are split in shared
 * memory, and the row sums by c_l (EE: c_l^2) in the reduce, which adds
 * the FP32 k-chunk sums as compensated pairs and reads them out in FP64.
 *   ST, SP[M][nk][ntau]   device float, 16-byte aligned, ntau % 4 == 0
 *   Pk[M][nk]             device double, >= 0
 *   ClTT, ClEE, ClTE[M][nl]  device double
 *   ws, ws_bytes          device workspace of at least
 *                         gcamb_los_cl_te_workspace bytes, 16-byte aligned
 * mode: GCAMB_BF16X3 (the only one); requires gcamb_bessel_table(g, mode).
 * Errors: GCAMB_EINVAL (mode, pointers, alignment, workspace, eps_cut too
 * large for the l = 2 limit), GCAMB_ESTATE (no table), GCAMB_EUNSUPPORTED
 * (ntau % 4 != 0, or not sm_103), GCAMB_ECUDA; GCAMB_ETIMEOUT by gcamb_sync.
 */
int gcamb_los_cl_te_workspace(const gcamb_grid *g, int M, int mode, size_t *bytes);
int gcamb_los_cl_te(const gcamb_grid *g, const float *ST, const float *SP, const double *Pk, int M, int mode,
                    double *ClTT, double *ClEE, double *ClTE, void *ws, size_t ws_bytes, void *stream);

/*
 * Two fields batched together on the tensor cores, each with its own kernel
 * grid (gcamb_grid_set_kernel; e.g. the tensor T and E kernels): for M
 * models, C^XX, C^YY and C^XY of Eq. (1) with Delta_X from the sources SX
 * and gx's table, Delta_Y from SY and gy's table, without storing Delta.
 * Each stage carries a block of both tables; the epilogue accumulates the
 * three spectra per model (the kernels' own factors are in the tables: no
 * c_l here).  gx and gy must share k, tau, tau0, the multipoles and the
 * table layout (the same grid arguments and kernels with the same
 * activity); both need gcamb_bessel_table(., GCAMB_BF16X3).  Arguments and
 * errors as for gcamb_los_cl_te; workspace from gcamb_los_cl_te_workspace(gx).
 */
int gcamb_los_cl_pair(const gcamb_grid *gx, const gcamb_grid *gy, const float *SX, const float *SY, const double *Pk,
                      int M, int mode, double *ClXX, double *ClYY, double *ClXY, void *ws, size_t ws_bytes,
                      void *stream);

/*
 * Plans: batches of sources with their own l_max and k range on one grid
 * (the uneven batch), run as one persistent tensor-core kernel replayed from
 * a CUDA graph.  Eq. (1) is summed for source m over its own k prefix
 * k[0..nk_m[m]) (trapezoid in ln k on that prefix) and Eq. (2) for its own
 * multipoles l <= lmax_m[m]; C_l above lmax_m[m] is written as 0.  The
 * paper's counterpart is Algorithm 1's gang loop over modes, which runs one
 * cosmology at a time.
 *
 *   lmax_m[M], nk_m[M]  host int, or both NULL (every source uses the whole
 *                       grid, as gcamb_los_cl); lmin <= lmax_m <= lmax,
 *                       1 <= nk_m <= nk.  Copied.
 *   mode                GCAMB_BF16X3, GCAMB_F16X3 or GCAMB_TF32X3 (the
 *                       tensor-core kernel), or GCAMB_PLAIN32 (FP32 on the
 *                       plain CUDA-core kernels, in chunks of 16 sources in
 *                       the caller's order: each chunk's transfer functions
 *                       over its longest k prefix and highest l-tile, then
 *                       each source's C_l over its own prefix; tune is
 *                       ignored, the plan info's "items" is the number of
 *                       chunks); the grid's table for this mode must be built.
 *   tune                0: source-tile width from a heuristic, the default
 *                       work-list settings (items ending at multiples of 16
 *                       k nodes; 12 for a uniform batch, 6 where that would
 *                       give a CTA fewer than four items; the tail cut);
 *                       1: the first gcamb_plan_launch times every
 *                       candidate on its inputs and keeps the fastest:
 *                       source-tile width (64, 128, 256 sources) x multipole
 *                       tiles per item (2 where the mode allows, 1) x work
 *                       items (ending at multiples of 16 or 8 k nodes, or of
 *                       equal cost, with the last 10% of the cost cut into
 *                       items of a quarter size; or at multiples of 16
 *                       without that cut): up to 20 candidates.  If
 *                       the environment variable GCAMB_TUNE_CACHE names a
 *                       file, choices are appended there (one JSON object
 *                       per line, keyed by device, grid and batch) and
 *                       reused by later plans.
 * Sources are processed sorted by l_max (descending), so that at each (k,
 * l-tile) the sources that need it are a prefix of the source tiles; work
 * items are spread over one persistent CTA per SM, longest first.
 * A plan refers to its grid and the grid's table: destroy the plan before
 * the grid (a plan used after its grid is destroyed reads freed memory).
 */
typedef struct gcamb_plan gcamb_plan;

#define GCAMB_PLAN_INFO_N 13

int gcamb_plan_create(gcamb_grid *g, int M, const int *lmax_m, const int *nk_m, int mode, int tune,
                      gcamb_plan **out);

/* Releases the plan and its graph.  NULL is accepted. */
int gcamb_plan_destroy(gcamb_plan *p);

/* Device workspace bytes gcamb_plan_launch needs (the largest candidate's
 * when tuning). */
int gcamb_plan_workspace(const gcamb_plan *p, size_t *bytes);

/*
 * Runs the plan: S[M][nk][ntau] device float (rows k >= nk_m[m] are
 * ignored), Pk[M][nk] device double (>= 0), Cl[M][nl] device double, ws a
 * 16-byte aligned device workspace of gcamb_plan_workspace bytes.
 * The first launch (and any launch whose pointers or stream differ from the
 * previous one) captures the split, contraction and reduction launches into a
 * CUDA graph; later launches replay it.  The first launch of a tuning plan
 * runs each candidate three times before capturing.  Must not itself be
 * called inside a stream capture.
 */
int gcamb_plan_launch(gcamb_plan *p, const float *S, const double *Pk, double *Cl, void *ws, size_t ws_bytes,
                      void *stream);

/*
 * Plan summary (host, int64[GCAMB_PLAN_INFO_N]): [0] source-tile width in use
 * (0 before tuning), [1] work items, [2] persistent CTAs, [3] graph captures,
 * [4] graph replays, [5] 1 if the width came from timing (now or cached),
 * [6] M, [7] workspace bytes of the width in use, [8] 1 if the sources are
 * read in place (fused kernel, no split pass: uniform batches only), [9]
 * multipole tiles per work item (2 when adjacent 128-multipole tiles share
 * each loaded and split source block; else 1), [10] work items of about
 * equal cost per persistent CTA (used when [12] is 0), [11] the tail of the
 * work list, 100 x round(1000 x share) + pieces (10004: the last 10% of the
 * cost in items cut into 4 pieces; 1: no tail cut), [12] kalign: every work
 * item ends at a multiple of kalign k nodes (0: items of equal cost).
 */
int gcamb_plan_info(const gcamb_plan *p, int64_t *info);

/*
 * Emulator of log C_l with a projection fallback.  The paper builds none; it
 * motivates fast spectra as training sets for emulators (Sec. 1, Sec. 5).
 * An MLP maps the 9 features of the synthetic source generator
 *   x = (tau*, sigma, r_s, cos phi, sin phi, k_D, b, n_s, ln(1e10 A_s))
 * to the standardised log C_l of the grid's multipoles (n_out = nl), with
 * `depth` hidden layers of `width` units and GELU.  It is trained on the
 * device by the library's kernels: tcgen05 GEMMs with bf16 operands and FP32
 * accumulation, FP32 parameters and Adam moments.  Parameter layout (host
 * arrays of gcamb_emu_params / gcamb_emu_grads): for each layer l, W_l
 * [out][in] row-major, then b_l [out].
 *
 * All pointers below are device memory unless marked host.
 */
typedef struct gcamb_emu gcamb_emu;

#define GCAMB_EMU_INFO_N 8
#define GCAMB_EMU_CHECK_N 6

/* n_in must be 9; 16 <= width <= 4096, 1 <= depth <= 8; batches up to
 * max_batch.  Parameters U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64
 * on (seed, index); identity normalisation. */
int gcamb_emu_create(gcamb_grid *g, int n_in, int width, int depth, int max_batch, uint64_t seed, gcamb_emu **out);
int gcamb_emu_destroy(gcamb_emu *e);
/* Number of parameters (host size_t*). */
int gcamb_emu_num_params(const gcamb_emu *e, size_t *n);
/* Copies host_in into the parameters (if not NULL), then the parameters into
 * host_out (if not NULL); host float arrays of gcamb_emu_num_params entries. */
int gcamb_emu_params(gcamb_emu *e, float *host_out, const float *host_in);
/* Gradients of the last gcamb_emu_train_step (host float array). */
int gcamb_emu_grads(gcamb_emu *e, float *host_out);
/* Normalisation (host float arrays, n_in and n_out long): set = 1 writes
 * them, set = 0 reads them.  Inputs enter as (x - mu_x) / sd_x (sd_x = 0: the
 * feature is dropped), outputs leave as log C_l = y sd_y + mu_y + (x_8 -
 * mu_x[8]): C_l is proportional to A_s (Eq. 1 is linear in P), so the
 * amplitude feature x_8 = ln(1e10 A_s) enters exactly, not through the
 * network. */
int gcamb_emu_norm(gcamb_emu *e, float *mu_x, float *sd_x, float *mu_y, float *sd_y, int set);
/* Fits the normalisation on N training samples X[N][9], Cl[N][n_out] (>0)
 * and writes the standardised targets
 * Y[N][n_out] = (log Cl - (x_8 - mu_x[8]) - mu_y) / sd_y:
 * mu_y per multipole; sd_y per multipole (per_l = 1) or one scale for all,
 * the root mean square of the per-multipole ones (per_l = 0, so that the loss
 * weighs the error of log C_l, i.e. the relative error of C_l, alike at every
 * l).  Synchronises the stream. */
int gcamb_emu_fit_norm(gcamb_emu *e, const float *X, const double *Cl, int N, int per_l, float *Y, void *stream);
/* One Adam step (lr; beta 0.9, 0.999; eps 1e-8) on the mean squared error of
 * the batch X[idx[b]], Y[idx[b]] (idx[B] device int, or NULL for the first B
 * rows); the batch loss goes to *loss (device float, may be NULL). */
int gcamb_emu_train_step(gcamb_emu *e, const float *X, const float *Y, const int *idx, int B, float lr, float *loss,
                         void *stream);
/* Standardised network output Y[B][n_out] for X[B][9]. */
int gcamb_emu_forward(gcamb_emu *e, const float *X, int B, float *Y, void *stream);
/*
 * Held-out check against reference spectra Cl_ref[N][n_out] (from the
 * projection path) for X[N][9]: per spectrum the max over l of
 * |C_emu/C_ref - 1|.  Parameter space is cut into at most 16 cells by
 * splitting, at its held-out median, each of the (at most 4) features whose
 * two halves differ most in mean log error; a cell is trusted when it holds at
 * least max(1, min_count) held-out spectra and all are within tol.  report (host double[GCAMB_EMU_CHECK_N]): max error, mean error,
 * fraction within tol, fraction of cells trusted, fraction of held-out
 * spectra in trusted cells, number of cells.  Synchronises the stream.
 */
int gcamb_emu_check(gcamb_emu *e, const float *X, const double *Cl_ref, int N, double tol, int min_count,
                    double *report, void *stream);
/*
 * C_l[B][n_out] (double) for X[B][9]: requests in trusted cells from the
 * network (exp of the de-standardised output plus the amplitude term of
 * gcamb_emu_norm), the others (all of them before
 * any check) from the batched projection, gcamb_los_cl in GCAMB_F16X3 on
 * sources regenerated by gcamb_synth_sources; used_fallback[B] (device int)
 * marks those.  Synchronises the stream; builds the F16X3 table if needed.
 */
int gcamb_emulate(gcamb_emu *e, const float *X, int B, double *Cl, int *used_fallback, void *stream);
/* Summary (host double[GCAMB_EMU_INFO_N]): parameters, Adam steps, last check's
 * max error, its tol, fraction of cells trusted, n_out, device error flag,
 * width. */
int gcamb_emu_info(const gcamb_emu *e, double *info);
/* Checkpoint: architecture, step, parameters, Adam moments, normalisation,
 * trust cells, FNV-1a checksum.  Load requires the same architecture. */
int gcamb_emu_save(const gcamb_emu *e, const char *path);
int gcamb_emu_load(gcamb_emu *e, const char *path);

/*
 * The synthetic source family (input synthesis, not the method): for
 * features X[M][9] as above,
 *   S(k, tau) = N(tau; tau*, sigma) cos(k r_s + phi) exp(-(k/k_D)^2)
 *             + b exp(-(tau - 11000)^2 / (2 * 2000^2)) exp(-k / 0.01)
 *   P(k) = A_s (k / 0.05)^(n_s - 1),  phi = atan2(sin phi, cos phi)
 * on the grid's nodes, evaluated in FP64: S[M][nk][ntau] float, Pk[M][nk]
 * double.
 */
int gcamb_synth_sources(const gcamb_grid *g, const float *X, int M, float *S, double *Pk, void *stream);

/*
 * gcamb_los_cl without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory,
 * such as a likelihood callback running inside a sampler or host framework
 * that owns the device's memory budget, or code that cannot afford
 * cudaMalloc's implicit device-wide synchronisation.
 *
 * Same arguments and result as gcamb_los_cl, without the workspace: every
 * scratch byte (the work list, the split sources, the weights and the
 * k-chunk partial sums) lives in one statically allocated 64 MiB device
 * buffer inside the library, which every device that loads the library
 * holds until the process exits.  The call makes no cudaMalloc, cudaFree or
 * other allocating call.
 *   status   device int, or NULL: set to GCAMB_ETIMEOUT if a bounded wait
 *            on the device gave up (left untouched otherwise); with NULL
 *            the timeout is reported by the next gcamb_sync instead
 * Limits and behaviour:
 *  - Problems whose scratch exceeds 64 MiB are rejected with GCAMB_EINVAL
 *    (the message gives the bytes needed); use gcamb_los_cl for them.  The
 *    scratch holds the k-chunk partial sums, 64 KB per (chunk of up to 16 k,
 *    l-tile, source tile) at 128 sources per tile, and 4-8 bytes per
 *    (k, source) of weights.
 *    When the sources cannot be read in place (ntau not a multiple of 4, or
 *    the TF32X3 mode) it also holds the split sources, about 4 bytes per
 *    (k, tau, source), which with 1000 tau nodes limits nk * M to about
 *    15,000.
 *  - Every call looks up the buffer's device address on the current device
 *    (cudaGetSymbolAddress).  The first call on a device may load the
 *    library's device code there (lazy module loading), which sets the
 *    buffer up; make it before any stream capture on that device.
 *  - A call on a stream that is being captured is refused with
 *    GCAMB_EUNSUPPORTED: the work list is copied up from host memory that
 *    lives only for the call.
 *  - The device error word used when status is NULL is set up by the grid's
 *    first device call (gcamb_bessel_table), not here.
 *  - All calls share the one buffer, and each call overwrites all of the
 *    scratch it uses before reading it, so nothing has to start at zero.
 *    Calls whose device work overlaps (on different streams, or from
 *    different host threads) race on the buffer and give wrong results:
 *    serialise them.
 */
int gcamb_los_cl_noalloc(const gcamb_grid *g, const float *S, const double *Pk, int M, int mode,
                         double *Cl, int *status, void *stream);

/*
 * Waits for `stream` and reports any error the library's kernels raised on
 * the device since the last gcamb_sync (GCAMB_ETIMEOUT for a bounded wait
 * that gave up), or a CUDA error (GCAMB_ECUDA).  Clears the device flag.
 */
int gcamb_sync(void *stream);

/* Kernel identifiers of the event tracer. */
#define GCAMB_K_TABLE     0  /* Bessel table generation */
#define GCAMB_K_LOS_PLAIN 1  /* plain transfer, Eq. (2) */
#define GCAMB_K_CL        2  /* Eq. (1) k-sum of stored transfers */
#define GCAMB_K_SPLIT     3  /* split pass: hi/lo planes and weights of the sources (batched path) */
#define GCAMB_K_WEIGHTS   4  /* sqrt(4 pi w_k P(k)) weights, fp16 row scales, TE tails (batched path) */
#define GCAMB_K_TC        5  /* tensor-core contraction + square + k-chunk sum */
#define GCAMB_K_REDUCE    6  /* fixed-order sum of the k-chunk partials (compensated), read out in FP64 */
#define GCAMB_K_INTERP    7  /* splines: sources onto the transfer k grid, C_l onto every l */
#define GCAMB_K_COUNT     8

/*
 * Event tracer.  While enabled, every kernel the library launches is
 * bracketed by CUDA events recorded on its launch stream.  Enabling clears
 * the accumulators.  gcamb_profile_read waits for the recorded events and
 * returns, for one kernel id, the summed device time in milliseconds and the
 * number of launches (host double*, int64_t*).  Not thread-safe with respect
 * to concurrent launches from several host threads.
 */
int gcamb_profile_enable(int on);
int gcamb_profile_read(int kernel, double *total_ms, int64_t *launches);

/*
 * Throughput probe of the device's plain arithmetic pipes (no tensor cores):
 *   what = 0: FP64 fused multiply-add, 1: FP32 fused multiply-add.
 * Runs a fixed dependent-chain kernel over all SMs and writes the measured
 * rate in FLOP/s (2 per FMA) to *flops (host).  Synchronous.
 */
int gcamb_probe_flops(int what, double *flops);

/*
 * Self-test of the tensor cores' FP32 accumulation (no counterpart in the
 * paper; it documents what the batched path's chain records correct).  One
 * 128 x 128 tile
 *   C[i][n] = sum_{k < K} A[i][k] B[n][k]
 * through the library's tcgen05 GEMM (kind::f16): A[128][K], B[128][K]
 * device float, row-major, rounded to bf16 by the loaders; C[128][128]
 * device float.  1 <= K <= 2^20.  Asynchronous on `stream`; a device-side
 * timeout is reported by gcamb_sync.  Errors: GCAMB_EINVAL, GCAMB_ECUDA.
 */
int gcamb_probe_mma(const float *A, const float *B, int K, float *C, void *stream);

/*
 * Self-test of the device-side failure path (no counterpart in the paper).
 * Launches one thread that waits, with the bounded wait every tensor-core
 * kernel of the library uses, on an mbarrier that nothing ever arrives on.
 * After the wait limit (one second) it gives up and reports GCAMB_ETIMEOUT
 * exactly as a stalled kernel would: in *status (device int) if status is not
 * NULL, else through the library's error flag, so that the next
 * gcamb_sync(stream) returns GCAMB_ETIMEOUT.  Nothing faults, traps or
 * hangs; the CUDA context stays usable.  Asynchronous on `stream`.
 */
int gcamb_selftest_wait(int *status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GCAMB_H */
