// C ABI entry points and host runtime: argument checks, grid set-up
// (quadrature weights, active extents, Miller start thresholds), device
// copies, table bookkeeping, error reporting.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "internal.h"

namespace gcamb {

static thread_local std::string t_err;

int fail(int code, const std::string &msg) {
  t_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  t_err = std::string(what) + ": " + cudaGetErrorString(e);
  return GCAMB_ECUDA;
}

static std::mutex g_flag_mu;
static int *g_flag_host = nullptr;
static int *g_flag_dev = nullptr;

int *device_error_flag() {
  std::lock_guard<std::mutex> lk(g_flag_mu);
  if (!g_flag_dev) {
    void *h = nullptr;
    if (cudaHostAlloc(&h, 64, cudaHostAllocMapped) != cudaSuccess) return nullptr;
    std::memset(h, 0, 64);
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
      cudaFreeHost(h);
      return nullptr;
    }
    g_flag_host = static_cast<int *>(h);
    g_flag_dev = static_cast<int *>(d);
  }
  return g_flag_dev;
}

static int read_and_clear_flag() {
  std::lock_guard<std::mutex> lk(g_flag_mu);
  if (!g_flag_host) return 0;
  volatile int *p = g_flag_host;
  int v = *p;
  *p = 0;
  return v;
}

// ------------------------------------------------------------ event tracer
namespace {
struct ProfRec {
  int id;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pending;
std::vector<cudaEvent_t> g_ev_pool;
double g_prof_ms[GCAMB_K_COUNT];
int64_t g_prof_n[GCAMB_K_COUNT];

cudaEvent_t take_event() {
  if (!g_ev_pool.empty()) {
    cudaEvent_t e = g_ev_pool.back();
    g_ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void drain_pending() {
  for (auto &r : g_prof_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      g_prof_ms[r.id] += ms;
      g_prof_n[r.id] += 1;
    }
    g_ev_pool.push_back(r.a);
    g_ev_pool.push_back(r.b);
  }
  g_prof_pending.clear();
}
}  // namespace

ProfScope::ProfScope(int id_, cudaStream_t st_) : id(id_), st(st_) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  if (g_prof_pending.size() > 4096) drain_pending();
  a = take_event();
  b = take_event();
  if (a && b) cudaEventRecord(a, st);
}

ProfScope::~ProfScope() {
  if (!a || !b) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(b, st);
  g_prof_pending.push_back({id, a, b});
}

// log of Watson's bound on |j_l(x)| = sqrt(pi/(2x)) |J_nu(x)|, nu = l + 1/2:
// |J_nu(nu z)| <= exp(-nu (alpha - tanh alpha)), z = sech(alpha) <= 1
// (Abramowitz & Stegun 9.1.63).  Written with s = tanh(alpha) = sqrt(1 - z^2).
double log_watson_bound(int l, double x) {
  const double nu = l + 0.5;
  const double z = x / nu;
  const double pre = 0.5 * std::log(M_PI / (2.0 * x));
  if (z >= 1.0) return pre;  // beyond the turning point: no decay
  const double s = std::sqrt((1.0 - z) * (1.0 + z));
  return pre + nu * (std::log(z) + s - std::log1p(s));
}

double watson_threshold(int l, double logeps) {
  if (l <= 0) return 0.0;
  const double nu = l + 0.5;
  // the bound increases on (0, xpk], xpk = nu sqrt(1 - 1/(4 nu^2))
  const double xpk = nu * std::sqrt(1.0 - 1.0 / (4.0 * nu * nu));
  if (log_watson_bound(l, xpk) < logeps) return xpk;
  double lo = std::log(1e-300), hi = std::log(xpk);
  if (log_watson_bound(l, std::exp(lo)) >= logeps) return 0.0;
  for (int it = 0; it < 90; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (log_watson_bound(l, std::exp(mid)) < logeps) lo = mid;
    else hi = mid;
  }
  return std::exp(lo);  // the bound is below eps for every x < this value
}

int ensure_device_grid(gcamb_grid *g) {
  if (g->d_k) return GCAMB_OK;
  auto up = [](double **dst, const std::vector<double> &src) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, src.size()) * sizeof(double));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice);
  };
  cudaError_t e;
  if ((e = up(&g->d_k, g->k)) != cudaSuccess) return cuda_fail(e, "grid upload");
  if ((e = up(&g->d_tau, g->tau)) != cudaSuccess) return cuda_fail(e, "grid upload");
  if ((e = up(&g->d_wtau, g->wtau)) != cudaSuccess) return cuda_fail(e, "grid upload");
  if ((e = up(&g->d_wk, g->wk)) != cudaSuccess) return cuda_fail(e, "grid upload");
  if ((e = up(&g->d_xstart, g->xstart)) != cudaSuccess) return cuda_fail(e, "grid upload");
  if (!g->xthr.empty() && (e = up(&g->d_xthr, g->xthr)) != cudaSuccess) return cuda_fail(e, "grid upload");
  auto upi = [](int **dst, const std::vector<int> &src) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, src.size()) * sizeof(int));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice);
  };
  if ((e = upi(&g->d_lrow, g->lrow)) != cudaSuccess) return cuda_fail(e, "grid upload");
  if ((e = upi(&g->d_rowof, g->rowof)) != cudaSuccess) return cuda_fail(e, "grid upload");
  // the mapped error word is set up here, with the grid's first device copy,
  // so that no later call (the allocation-free entry point in particular)
  // has to allocate it
  if (!device_error_flag()) return fail(GCAMB_ECUDA, "grid upload: error flag allocation");
  return GCAMB_OK;
}

static void trapezoid(const std::vector<double> &x, std::vector<double> &w) {
  const size_t n = x.size();
  w.assign(n, 0.0);
  if (n < 2) return;
  w[0] = 0.5 * (x[1] - x[0]);
  for (size_t i = 1; i + 1 < n; ++i) w[i] = 0.5 * (x[i + 1] - x[i - 1]);
  w[n - 1] = 0.5 * (x[n - 1] - x[n - 2]);
}

static bool is_sm103() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  int maj = 0, min = 0;
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev);
  return maj == 10 && min == 3;
}

}  // namespace gcamb

using namespace gcamb;

extern "C" {

const char *gcamb_version(void) { return "gcamb-gb300 0.1 (sm_103a)"; }

const char *gcamb_last_error(void) { return t_err.c_str(); }

static int grid_build(const double *k, int nk, const double *tau, int ntau, double tau0, std::vector<int> lrow,
                      bool sampled, double eps_cut, gcamb_grid **out, double K = 0.0);

int gcamb_grid_create(const double *k, int nk, const double *tau, int ntau, double tau0, int lmin, int lmax,
                      double eps_cut, gcamb_grid **out) {
  if (!out) return fail(GCAMB_EINVAL, "grid_create: out is NULL");
  *out = nullptr;
  if (lmin < 0 || lmax < lmin || lmax > kMaxL) return fail(GCAMB_EINVAL, "grid_create: need 0 <= lmin <= lmax <= 20000");
  std::vector<int> lrow(lmax - lmin + 1);
  for (int r = 0; r <= lmax - lmin; ++r) lrow[r] = lmin + r;
  return grid_build(k, nk, tau, ntau, tau0, std::move(lrow), false, eps_cut, out);
}

int gcamb_grid_create_lsampled(const double *k, int nk, const double *tau, int ntau, double tau0, const int *lval,
                               int nl, double eps_cut, gcamb_grid **out) {
  if (!out) return fail(GCAMB_EINVAL, "grid_create_lsampled: out is NULL");
  *out = nullptr;
  if (!lval || nl < 1) return fail(GCAMB_EINVAL, "grid_create_lsampled: need a list of at least one multipole");
  for (int r = 0; r < nl; ++r) {
    if (lval[r] < 0 || lval[r] > kMaxL) return fail(GCAMB_EINVAL, "grid_create_lsampled: need 0 <= l <= 20000");
    if (r && lval[r] <= lval[r - 1]) return fail(GCAMB_EINVAL, "grid_create_lsampled: l must be strictly increasing");
  }
  return grid_build(k, nk, tau, ntau, tau0, std::vector<int>(lval, lval + nl), true, eps_cut, out);
}

int gcamb_grid_create_curved(const double *q, int nq, const double *tau, int ntau, double tau0, int lmin, int lmax,
                             double K, double eps_cut, gcamb_grid **out) {
  if (!out) return fail(GCAMB_EINVAL, "grid_create_curved: out is NULL");
  *out = nullptr;
  if (!(K != 0.0) || !std::isfinite(K)) return fail(GCAMB_EINVAL, "grid_create_curved: K must be finite and nonzero");
  if (lmin < 0 || lmax < lmin || lmax > kMaxL)
    return fail(GCAMB_EINVAL, "grid_create_curved: need 0 <= lmin <= lmax <= 20000");
  if (K > 0.0 && q) {
    const double rk = std::sqrt(K);
    for (int j = 0; j < nq; ++j) {
      const double b = q[j] / rk;
      if (!(std::fabs(b - std::nearbyint(b)) <= 1e-6 * std::max(1.0, b)) || b < 3.0)
        return fail(GCAMB_EINVAL, "grid_create_curved: closed space needs integer beta = q / sqrt(K) >= 3");
    }
  }
  std::vector<int> lrow(lmax - lmin + 1);
  for (int r = 0; r <= lmax - lmin; ++r) lrow[r] = lmin + r;
  return grid_build(q, nq, tau, ntau, tau0, std::move(lrow), false, eps_cut, out, K);
}

int gcamb_grid_set_kernel(gcamb_grid *g, int kernel) {
  if (!g) return fail(GCAMB_EINVAL, "grid_set_kernel: NULL grid");
  if (kernel < GCAMB_KERNEL_J || kernel > GCAMB_KERNEL_TENSOR_B) return fail(GCAMB_EINVAL, "grid_set_kernel: unknown kernel");
  for (const auto &t : g->tab)
    if (t.d_data) return fail(GCAMB_ESTATE, "grid_set_kernel: the grid already has a table");
  if (g->curved && kernel) return fail(GCAMB_EUNSUPPORTED, "grid_set_kernel: kernel grids are flat-space only");
  g->kernel = kernel;
  if (kernel && g->lmin <= 5)  // the l = 2 kernels do not vanish at x = 0: keep every node in the first tile
    for (int q = 0; q < g->nk; ++q) g->ext[(size_t)q * g->nlt] = g->ntau;
  return GCAMB_OK;
}

int gcamb_l_sampling(int lmin, int lmax, double boost, int *lval, int *n) {
  if (!n) return fail(GCAMB_EINVAL, "l_sampling: n is NULL");
  if (lmin < 0 || lmax < lmin || lmax > kMaxL || !(boost > 0.0))
    return fail(GCAMB_EINVAL, "l_sampling: need 0 <= lmin <= lmax <= 20000 and boost > 0");
  // every l below 20 boost, then steps of round(l / (20 boost)), at most
  // ceil(50 / boost); boost >= 50 keeps every l; lmax is always a sample
  const int cap = std::max(1, (int)std::ceil(50.0 / boost));
  int cnt = 0;
  for (int l = lmin; l <= lmax;) {
    if (lval) lval[cnt] = l;
    ++cnt;
    if (l == lmax) break;
    int step = boost >= 50.0 ? 1 : std::max(1, std::min(cap, (int)std::lround(l / (20.0 * boost))));
    l = std::min(lmax, l + step);
  }
  *n = cnt;
  return GCAMB_OK;
}

static int grid_build(const double *k, int nk, const double *tau, int ntau, double tau0, std::vector<int> lrow,
                      bool sampled, double eps_cut, gcamb_grid **out, double K) {
  const int lmin = lrow.front(), lmax = lrow.back();
  if (!k || !tau) return fail(GCAMB_EINVAL, "grid_create: k or tau is NULL");
  if (nk < 1 || ntau < 1) return fail(GCAMB_EINVAL, "grid_create: nk and ntau must be >= 1");
  if (nk > (1 << 24) || ntau > (1 << 20)) return fail(GCAMB_EINVAL, "grid_create: grid too large");
  if (!(eps_cut >= 0.0) || eps_cut > 1e-3) return fail(GCAMB_EINVAL, "grid_create: eps_cut must be in [0, 1e-3]");
  if (eps_cut == 0.0) eps_cut = 1e-30;
  eps_cut = std::max(eps_cut, 1e-200);
  if (!std::isfinite(tau0)) return fail(GCAMB_EINVAL, "grid_create: tau0 not finite");
  for (int i = 0; i < nk; ++i) {
    if (!(k[i] > 0.0) || !std::isfinite(k[i])) return fail(GCAMB_EINVAL, "grid_create: k must be finite and > 0");
    if (i && !(k[i] > k[i - 1])) return fail(GCAMB_EINVAL, "grid_create: k must be strictly increasing");
  }
  for (int i = 0; i < ntau; ++i) {
    if (!std::isfinite(tau[i])) return fail(GCAMB_EINVAL, "grid_create: tau not finite");
    if (i && !(tau[i] > tau[i - 1])) return fail(GCAMB_EINVAL, "grid_create: tau must be strictly increasing");
  }
  if (tau[ntau - 1] > tau0) return fail(GCAMB_EINVAL, "grid_create: tau must not exceed tau0");

  gcamb_grid *g = new (std::nothrow) gcamb_grid();
  if (!g) return fail(GCAMB_ENOMEM, "grid_create: host allocation");
  g->nk = nk;
  g->ntau = ntau;
  g->lmin = lmin;
  g->lmax = lmax;
  g->nl = (int)lrow.size();
  g->nlt = (g->nl + kTileL - 1) / kTileL;
  g->lsampled = sampled;
  g->rowof.assign((size_t)(lmax - lmin + 1), -1);
  for (int r = 0; r < g->nl; ++r) g->rowof[lrow[r] - lmin] = r;
  g->lrow = std::move(lrow);
  if (K != 0.0) {
    g->curved = K < 0.0 ? 1 : 2;
    g->K = K;
    g->rk = std::sqrt(std::fabs(K));
    g->ext_ready = false;  // the tau-prefixes come from the first table build
  }
  g->tau0 = tau0;
  g->eps_cut = eps_cut;
  g->k.assign(k, k + nk);
  g->tau.assign(tau, tau + ntau);
  trapezoid(g->tau, g->wtau);
  {
    std::vector<double> u(nk);
    for (int i = 0; i < nk; ++i) u[i] = std::log(k[i]);
    trapezoid(u, g->wk);
  }

  // Active extents: tau-prefix with x = k (tau0 - tau) >= x_eps(l0) per tile.
  const double logeps = std::log(eps_cut);
  auto prefix = [&](int q, double xe) -> int {
    // x decreases with i: count i with x_i >= xe
    int lo = 0, hi = ntau;  // invariant: x_i >= xe for i < lo, < xe for i >= hi
    while (lo < hi) {
      int mid = (lo + hi) / 2;
      double x = g->k[q] * (tau0 - g->tau[mid]);
      if (x >= xe) lo = mid + 1;
      else hi = mid;
    }
    return lo;
  };
  g->ext.assign((size_t)nk * g->nlt, 0);
  for (int lt = 0; lt < g->nlt; ++lt) {
    const int l0 = g->lrow[(size_t)lt * kTileL];  // the tile's lowest multipole
    const double xe = watson_threshold(l0, logeps);
    for (int q = 0; q < nk; ++q)
      g->ext[(size_t)q * g->nlt + lt] = (l0 == 0 || g->curved) ? ntau : prefix(q, xe);
  }
  // Active (l, k, tau) entries with the per-l prefix.
  {
    std::vector<double> xe(g->nl);
    for (int r = 0; r < g->nl; ++r) xe[r] = watson_threshold(g->lrow[r], logeps);
    if (!g->curved) g->xthr = xe;
    int64_t act = 0;
    for (int q = 0; q < nk; ++q) {
      int i = ntau;  // boundary moves towards 0 as l grows
      for (int r = 0; r < g->nl; ++r) {
        if (g->lrow[r] == 0) { act += ntau; continue; }
        while (i > 0 && g->k[q] * (tau0 - g->tau[i - 1]) < xe[r]) --i;
        act += i;
      }
    }
    g->active = act;
  }
  // Miller start thresholds: xstart[l] = x below which |j_l| < delta.
  {
    const double logdelta = std::log(std::max(eps_cut * 1e-10, 1e-290));
    const int cap = lmax + 4096;
    g->xstart.clear();
    for (int l = 0; l <= cap; ++l) {
      double xs = watson_threshold(l, logdelta);
      g->xstart.push_back(xs);
      if (l > lmax && xs > (double)lmax + 2.0) break;
    }
    g->nxs = (int)g->xstart.size();
  }
  *out = g;
  return GCAMB_OK;
}

int gcamb_grid_destroy(gcamb_grid *g) {
  if (!g) return GCAMB_OK;
  drop_plans(g);
  for (auto &t : g->tab) {
    table_free(t);
    cudaFree(t.d_nkb);
    cudaFree(t.d_off);
  }
  cudaFree(g->d_k);
  cudaFree(g->d_tau);
  cudaFree(g->d_wtau);
  cudaFree(g->d_wk);
  cudaFree(g->d_xstart);
  cudaFree(g->d_xthr);
  cudaFree(g->d_lrow);
  cudaFree(g->d_rowof);
  delete g;
  return GCAMB_OK;
}

int gcamb_grid_info(const gcamb_grid *g, int64_t *info) {
  if (!g || !info) return fail(GCAMB_EINVAL, "grid_info: NULL argument");
  int64_t stored = 0;
  for (int q = 0; q < g->nk; ++q)
    for (int lt = 0; lt < g->nlt; ++lt) {
      int e = g->ext[(size_t)q * g->nlt + lt];
      stored += (int64_t)((e + 63) / 64) * 64 * kTileL;
    }
  info[0] = g->nk;
  info[1] = g->ntau;
  info[2] = g->nl;
  info[3] = g->nlt;
  info[4] = g->active;
  info[5] = stored;
  info[6] = g->lmin;
  info[7] = g->lmax;
  return GCAMB_OK;
}

int gcamb_grid_extents(const gcamb_grid *g, int32_t *ext) {
  if (!g || !ext) return fail(GCAMB_EINVAL, "grid_extents: NULL argument");
  std::memcpy(ext, g->ext.data(), g->ext.size() * sizeof(int32_t));
  return GCAMB_OK;
}

int gcamb_grid_weights(const gcamb_grid *g, double *wtau, double *wk) {
  if (!g) return fail(GCAMB_EINVAL, "grid_weights: NULL grid");
  if (wtau) std::memcpy(wtau, g->wtau.data(), g->wtau.size() * sizeof(double));
  if (wk) std::memcpy(wk, g->wk.data(), g->wk.size() * sizeof(double));
  return GCAMB_OK;
}

int gcamb_table_compressed(const gcamb_grid *g, int mode, int *compressed) {
  if (!g || !compressed) return fail(GCAMB_EINVAL, "table_compressed: NULL argument");
  if (!mode_layout(mode).kb) return fail(GCAMB_EINVAL, "table_compressed: unknown mode");
  const Table &t = g->tab[mode];
  if (!t.built) return fail(GCAMB_ESTATE, "table_compressed: build the table for this mode first");
  *compressed = t.vmm ? 1 : 0;
  return GCAMB_OK;
}

int gcamb_table_bytes(const gcamb_grid *g, int mode, size_t *bytes) {
  if (!g || !bytes) return fail(GCAMB_EINVAL, "table_bytes: NULL argument");
  ModeLayout lay = mode_layout(mode);
  if (!lay.kb) return fail(GCAMB_EINVAL, "table_bytes: unknown mode");
  int64_t nb = 0;
  for (size_t e = 0; e < g->ext.size(); ++e) nb += (g->ext[e] + lay.kb - 1) / lay.kb;
  *bytes = (size_t)nb * lay.block_bytes();
  return GCAMB_OK;
}

int gcamb_bessel_table(gcamb_grid *g, int mode, void *stream) {
  if (!g) return fail(GCAMB_EINVAL, "bessel_table: NULL grid");
  if (!mode_layout(mode).kb) return fail(GCAMB_EINVAL, "bessel_table: unknown mode");
  int rc = ensure_device_grid(g);
  if (rc) return rc;
  return launch_bessel_table(g, mode, (cudaStream_t)stream);
}

int gcamb_sph_bessel(const double *x, int n, int lmax, double *out, void *stream) {
  if (n < 0 || lmax < 0 || lmax > kMaxL) return fail(GCAMB_EINVAL, "sph_bessel: bad n or lmax");
  if (n == 0) return GCAMB_OK;
  if (!x || !out) return fail(GCAMB_EINVAL, "sph_bessel: NULL pointer");
  return launch_sph_bessel(x, n, lmax, out, (cudaStream_t)stream);
}

int gcamb_los_transfer(const gcamb_grid *g, const void *S, int M, int mode, void *Delta, void *stream) {
  if (!g) return fail(GCAMB_EINVAL, "los_transfer: NULL grid");
  if (mode != GCAMB_PLAIN64 && mode != GCAMB_PLAIN32)
    return fail(GCAMB_EINVAL, "los_transfer: mode must be GCAMB_PLAIN64 or GCAMB_PLAIN32");
  if (M < 0) return fail(GCAMB_EINVAL, "los_transfer: M < 0");
  if (M == 0) return GCAMB_OK;
  if (!S || !Delta) return fail(GCAMB_EINVAL, "los_transfer: NULL S or Delta");
  if (!g->tab[mode].built) return fail(GCAMB_ESTATE, "los_transfer: build the table for this mode first");
  return launch_los_plain(g, S, M, mode, Delta, (cudaStream_t)stream);
}

int gcamb_los_transfer_e(const gcamb_grid *g, const void *SP, int M, int mode, void *DeltaE, void *stream) {
  if (!g) return fail(GCAMB_EINVAL, "los_transfer_e: NULL grid");
  if (g->curved) return fail(GCAMB_EUNSUPPORTED, "los_transfer_e: the E-mode kernel is flat-space only");
  if (g->kernel) return fail(GCAMB_EUNSUPPORTED, "los_transfer_e: needs a j_l grid (use gcamb_los_transfer on a kernel grid)");
  if (mode != GCAMB_PLAIN64 && mode != GCAMB_PLAIN32)
    return fail(GCAMB_EINVAL, "los_transfer_e: mode must be GCAMB_PLAIN64 or GCAMB_PLAIN32");
  if (M < 0) return fail(GCAMB_EINVAL, "los_transfer_e: M < 0");
  if (M == 0) return GCAMB_OK;
  if (!SP || !DeltaE) return fail(GCAMB_EINVAL, "los_transfer_e: NULL S_P or Delta_E");
  if (!g->tab[mode].built) return fail(GCAMB_ESTATE, "los_transfer_e: build the table for this mode first");
  return launch_los_plain(g, SP, M, mode, DeltaE, (cudaStream_t)stream, true);
}

int gcamb_los_transfer_tensor(const gcamb_grid *g, const void *ST, const void *SP, int M, int mode, void *DeltaT,
                              void *DeltaE, void *DeltaB, void *stream) {
  if (!g) return fail(GCAMB_EINVAL, "los_transfer_tensor: NULL grid");
  if (g->curved) return fail(GCAMB_EUNSUPPORTED, "los_transfer_tensor: the tensor kernels are flat-space only");
  if (g->kernel) return fail(GCAMB_EUNSUPPORTED, "los_transfer_tensor: needs a j_l grid");
  if (mode != GCAMB_PLAIN64 && mode != GCAMB_PLAIN32)
    return fail(GCAMB_EINVAL, "los_transfer_tensor: mode must be GCAMB_PLAIN64 or GCAMB_PLAIN32");
  if (M < 0) return fail(GCAMB_EINVAL, "los_transfer_tensor: M < 0");
  if (M == 0) return GCAMB_OK;
  if (!ST || !SP || !DeltaT || !DeltaE || !DeltaB) return fail(GCAMB_EINVAL, "los_transfer_tensor: NULL pointer");
  if (DeltaT == DeltaE || DeltaT == DeltaB || DeltaE == DeltaB)
    return fail(GCAMB_EINVAL, "los_transfer_tensor: the three outputs must be distinct");
  if (!g->tab[mode].built) return fail(GCAMB_ESTATE, "los_transfer_tensor: build the table for this mode first");
  return launch_los_tensor(g, ST, SP, M, mode, DeltaT, DeltaE, DeltaB, (cudaStream_t)stream);
}

int gcamb_cl_cross(const gcamb_grid *g, const void *DX, const void *DY, int d_dtype, const double *Pk, int M,
                   double *Cl, void *stream) {
  if (!g) return fail(GCAMB_EINVAL, "cl_cross: NULL grid");
  if (d_dtype != GCAMB_F64 && d_dtype != GCAMB_F32) return fail(GCAMB_EINVAL, "cl_cross: d_dtype must be F64 or F32");
  if (M < 0) return fail(GCAMB_EINVAL, "cl_cross: M < 0");
  if (M == 0) return GCAMB_OK;
  if (!DX || !DY || !Pk || !Cl) return fail(GCAMB_EINVAL, "cl_cross: NULL pointer");
  int rc = ensure_device_grid(const_cast<gcamb_grid *>(g));
  if (rc) return rc;
  return launch_cl_cross(g, DX, DY, d_dtype, Pk, M, Cl, (cudaStream_t)stream);
}

int gcamb_cl(const gcamb_grid *g, const void *Delta, int d_dtype, const double *Pk, int M, double *Cl,
             void *stream) {
  if (!g) return fail(GCAMB_EINVAL, "cl: NULL grid");
  if (d_dtype != GCAMB_F64 && d_dtype != GCAMB_F32) return fail(GCAMB_EINVAL, "cl: d_dtype must be F64 or F32");
  if (M < 0) return fail(GCAMB_EINVAL, "cl: M < 0");
  if (M == 0) return GCAMB_OK;
  if (!Delta || !Pk || !Cl) return fail(GCAMB_EINVAL, "cl: NULL pointer");
  int rc = ensure_device_grid(const_cast<gcamb_grid *>(g));
  if (rc) return rc;
  return launch_cl(g, Delta, d_dtype, Pk, M, Cl, (cudaStream_t)stream);
}

int gcamb_los_cl_workspace(const gcamb_grid *g, int M, int mode, size_t *bytes) {
  if (!g || !bytes) return fail(GCAMB_EINVAL, "los_cl_workspace: NULL argument");
  if (mode != GCAMB_BF16X3 && mode != GCAMB_TF32X3 && mode != GCAMB_F16X3)
    return fail(GCAMB_EINVAL, "los_cl_workspace: bad mode");
  if (M < 1) return fail(GCAMB_EINVAL, "los_cl_workspace: M must be >= 1");
  *bytes = los_cl_workspace_bytes(g, M, mode);
  return GCAMB_OK;
}

int gcamb_los_cl(const gcamb_grid *g, const float *S, const double *Pk, int M, int mode, double *Cl, void *ws,
                 size_t ws_bytes, void *stream) {
  if (!g) return fail(GCAMB_EINVAL, "los_cl: NULL grid");
  if (mode != GCAMB_BF16X3 && mode != GCAMB_TF32X3 && mode != GCAMB_F16X3)
    return fail(GCAMB_EINVAL, "los_cl: mode must be GCAMB_BF16X3, GCAMB_F16X3 or GCAMB_TF32X3");
  if (M < 0) return fail(GCAMB_EINVAL, "los_cl: M < 0");
  if (M == 0) return GCAMB_OK;
  if (!S || !Pk || !Cl) return fail(GCAMB_EINVAL, "los_cl: NULL pointer");
  if (!g->tab[mode].built) return fail(GCAMB_ESTATE, "los_cl: build the table for this mode first");
  if (!is_sm103()) return fail(GCAMB_EUNSUPPORTED, "los_cl: the tensor-core path needs an sm_103 device");
  size_t need = los_cl_workspace_bytes(g, M, mode);
  if (!ws || ws_bytes < need) return fail(GCAMB_EINVAL, "los_cl: workspace missing or too small");
  if (reinterpret_cast<uintptr_t>(ws) % 16) return fail(GCAMB_EINVAL, "los_cl: workspace must be 16-byte aligned");
  return launch_los_cl(g, S, Pk, M, mode, Cl, ws, ws_bytes, (cudaStream_t)stream);
}

static int te_check(const gcamb_grid *g, int M, int mode, const char *who) {
  if (!g) return fail(GCAMB_EINVAL, std::string(who) + ": NULL grid");
  if (g->curved) return fail(GCAMB_EUNSUPPORTED, std::string(who) + ": the E-mode kernel is flat-space only");
  if (g->kernel) return fail(GCAMB_EUNSUPPORTED, std::string(who) + ": needs a j_l grid");
  if (mode != GCAMB_BF16X3) return fail(GCAMB_EINVAL, std::string(who) + ": mode must be GCAMB_BF16X3");
  if (M < 0) return fail(GCAMB_EINVAL, std::string(who) + ": M < 0");
  if (!g->tab[mode].built) return fail(GCAMB_ESTATE, std::string(who) + ": build the table for this mode first");
  if (g->ntau % 4 != 0)
    return fail(GCAMB_EUNSUPPORTED, std::string(who) + ": needs ntau % 4 == 0 (sources read by TMA in place)");
  return GCAMB_OK;
}

int gcamb_los_cl_te_workspace(const gcamb_grid *g, int M, int mode, size_t *bytes) {
  if (!bytes) return fail(GCAMB_EINVAL, "los_cl_te_workspace: bytes is NULL");
  *bytes = 0;
  if (g && g->kernel && !g->curved && mode == GCAMB_BF16X3 && M >= 0 && g->tab[mode].built && g->ntau % 4 == 0) {
    // a kernel grid: the workspace of gcamb_los_cl_pair
    *bytes = M ? los_cl_te_workspace_bytes(g, M) : 0;
    return (*bytes || !M) ? GCAMB_OK : fail(GCAMB_ECUDA, "los_cl_te_workspace: plan");
  }
  if (int rc = te_check(g, M, mode, "los_cl_te_workspace")) return rc;
  if (M == 0) return GCAMB_OK;
  *bytes = los_cl_te_workspace_bytes(g, M);
  return *bytes ? GCAMB_OK : fail(GCAMB_ECUDA, "los_cl_te_workspace: plan");
}

int gcamb_los_cl_te(const gcamb_grid *g, const float *ST, const float *SP, const double *Pk, int M, int mode,
                    double *ClTT, double *ClEE, double *ClTE, void *ws, size_t ws_bytes, void *stream) {
  if (int rc = te_check(g, M, mode, "los_cl_te")) return rc;
  if (M == 0) return GCAMB_OK;
  if (!ST || !SP || !Pk || !ClTT || !ClEE || !ClTE) return fail(GCAMB_EINVAL, "los_cl_te: NULL pointer");
  if (!is_sm103()) return fail(GCAMB_EUNSUPPORTED, "los_cl_te: the tensor-core path needs an sm_103 device");
  if (!ws) return fail(GCAMB_EINVAL, "los_cl_te: workspace missing");
  if (reinterpret_cast<uintptr_t>(ws) % 16) return fail(GCAMB_EINVAL, "los_cl_te: workspace must be 16-byte aligned");
  return launch_los_cl_te(g, ST, SP, Pk, M, ClTT, ClEE, ClTE, ws, ws_bytes, (cudaStream_t)stream);
}

int gcamb_los_cl_pair(const gcamb_grid *gx, const gcamb_grid *gy, const float *SX, const float *SY, const double *Pk,
                      int M, int mode, double *ClXX, double *ClYY, double *ClXY, void *ws, size_t ws_bytes,
                      void *stream) {
  if (!gx || !gy) return fail(GCAMB_EINVAL, "los_cl_pair: NULL grid");
  if (mode != GCAMB_BF16X3) return fail(GCAMB_EINVAL, "los_cl_pair: mode must be GCAMB_BF16X3");
  if (M < 0) return fail(GCAMB_EINVAL, "los_cl_pair: M < 0");
  if (!gx->tab[mode].built || !gy->tab[mode].built)
    return fail(GCAMB_ESTATE, "los_cl_pair: build both grids' tables for this mode first");
  if (gx->ntau % 4 != 0) return fail(GCAMB_EUNSUPPORTED, "los_cl_pair: needs ntau % 4 == 0");
  if (M == 0) return GCAMB_OK;
  if (!SX || !SY || !Pk || !ClXX || !ClYY || !ClXY || !ws) return fail(GCAMB_EINVAL, "los_cl_pair: NULL pointer");
  if (!is_sm103()) return fail(GCAMB_EUNSUPPORTED, "los_cl_pair: the tensor-core path needs an sm_103 device");
  if (reinterpret_cast<uintptr_t>(ws) % 16) return fail(GCAMB_EINVAL, "los_cl_pair: workspace must be 16-byte aligned");
  return launch_los_cl_pair(gx, gy, SX, SY, Pk, M, ClXX, ClYY, ClXY, ws, ws_bytes, (cudaStream_t)stream);
}

int gcamb_sync(void *stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  int f = read_and_clear_flag();
  if (f == kDevErrTimeout) return fail(GCAMB_ETIMEOUT, "a device-side bounded wait gave up");
  if (f) return fail(GCAMB_ECUDA, "device error flag " + std::to_string(f));
  return GCAMB_OK;
}

int gcamb_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  drain_pending();
  g_prof_on = on != 0;
  for (int i = 0; i < GCAMB_K_COUNT; ++i) {
    g_prof_ms[i] = 0.0;
    g_prof_n[i] = 0;
  }
  return GCAMB_OK;
}

int gcamb_profile_read(int kernel, double *total_ms, int64_t *launches) {
  if (kernel < 0 || kernel >= GCAMB_K_COUNT || !total_ms || !launches)
    return fail(GCAMB_EINVAL, "profile_read: bad argument");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  drain_pending();
  *total_ms = g_prof_ms[kernel];
  *launches = g_prof_n[kernel];
  return GCAMB_OK;
}

int gcamb_probe_flops(int what, double *flops) {
  if (!flops || (what != 0 && what != 1)) return fail(GCAMB_EINVAL, "probe_flops: bad argument");
  return run_probe_flops(what, flops);
}

int gcamb_selftest_wait(int *status, void *stream) { return run_wait_selftest(status, (cudaStream_t)stream); }

}  // extern "C"
