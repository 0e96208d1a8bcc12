/*
 * FP64 CPU oracle for the line-of-sight projection and the C_l k-integral.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * What it computes (arXiv 2509.25110, Sec. 2.1):
 *   Eq. (2), discretised on the tau nodes with trapezoid weights w_i:
 *       Delta_l(k) = sum_i  w_i S(k, tau_i) j_l(k (tau0 - tau_i))
 *   Eq. (1), for X = Y = T, discretised on the k nodes with trapezoid weights
 *   in u = ln k (the dk/k measure), P = P_R:
 *       C_l = 4 pi sum_j  w_j P(k_j) Delta_l(k_j)^2
 * The sums are dense: every tau node is used, no activity cut.
 *
 * E-mode polarisation (Eq. 3, and Eq. (1) for X, Y in {T, E}):
 *       Delta^E_l(k) = sum_i  w_i S_P(k, tau_i) eps_l(k (tau0 - tau_i)),
 *       C^XY_l = 4 pi sum_j  w_j P(k_j) Delta^X_l(k_j) Delta^Y_l(k_j).
 * The paper calls eps_l a kernel "related to spherical Bessel functions"
 * (Sec. 2.1); this oracle takes the flat-space line-of-sight form
 *       eps_l(x) = sqrt((l+2)! / (l-2)!) j_l(x) / x^2     (l >= 2; 0 below),
 * with its limit at x = 0: sqrt(24) / 15 for l = 2 and 0 above.
 *
 * Tensor modes (the second projection the paper runs, Sec. 3.1 and 3.3; it
 * says only that equations like Eqs. (2)-(3) hold for tensors and B modes,
 * Sec. 2.1).  This oracle takes the flat-space line-of-sight kernels of
 * tensor perturbations:
 *       T: t_l(x) = sqrt((l+2)!/(l-2)!) j_l(x) / x^2            (= eps_l)
 *       E: e_l(x) = -j_l + j_l'' + 2 j_l / x^2 + 4 j_l' / x
 *       B: b_l(x) = 2 j_l' + 4 j_l / x
 * (l >= 2; 0 below), evaluated through the Bessel equation and
 * j_l' = j_{l-1} - (l+1) j_l / x as
 *       e_l = (l (l-1) / x^2 - 2) j_l + 2 j_{l-1} / x,
 *       b_l = 2 j_{l-1} - 2 (l-1) j_l / x,
 * with their limits at x = 0: e_2 = 4/5, all others 0.  Each projection is
 * the dense sum of Eq. (2) with the tensor sources S_T^t, S_P^t.
 *
 * Non-flat space (the curved-space kernels the paper names as next, Sec. 2.1
 * and 5): phi_l becomes the hyperspherical Bessel function Phi^beta_l(chi)
 * of curvature K, beta = q / sqrt|K|, chi = sqrt|K| (tau0 - tau), with
 * (open, K < 0: sh = sinh, ct = coth, s_l = sqrt(beta^2 + l^2);
 *  closed, K > 0: sh = sin, ct = cot, s_l = sqrt(beta^2 - l^2), beta an
 *  integer, Phi_l = 0 for l >= beta)
 *       Phi_0 = sin(beta chi) / (beta sh(chi)),
 *       Phi_1 = Phi_0 (ct(chi) - beta cot(beta chi)) / s_1
 *             = (sin(beta chi) ct(chi) - beta cos(beta chi)) / (beta sh(chi) s_1),
 *       s_(l+1) Phi_(l+1) = (2l+1) ct(chi) Phi_l - s_l Phi_(l-1),
 * which tends to j_l(q r) as K -> 0.  This oracle runs the recurrence
 * downwards from far above the order range and the turning point (Miller;
 * in closed space from l = beta - 1 with Phi_beta = 0, which is exact) and
 * normalises to the larger of the closed forms of Phi_0, Phi_1.
 *
 * The paper fixes neither the Bessel kernel's evaluation nor the quadrature
 * (it names phi_l only as "related to spherical Bessel functions", Sec. 2.1,
 * and evaluates it inside the line-of-sight loop, Sec. 3.2 / Algorithm 1).
 * This oracle takes phi_l = j_l (flat space) and evaluates j_l(x) for all
 * l = 0..lmax at once by
 *   - Miller's backward recurrence (J. C. P. Miller, British Association
 *     Mathematical Tables vol. X, 1952; stability: W. Gautschi, SIAM Review 9,
 *     1967) started far above max(lmax, x), for the orders above x;
 *   - the forward recurrence from the closed forms of j_0 and j_1 for the
 *     orders at or below x (x >= 1), where the forward direction is stable;
 *   - for x < 1, the backward sequence normalised to j_0 = sin(x)/x.
 * Three-term recurrence used in both directions:
 *       j_{l-1}(x) + j_{l+1}(x) = (2l+1)/x j_l(x).
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC -o liboracle.so gcamb_oracle.c -lm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Quadrature weights                                                       */
/* ------------------------------------------------------------------------ */

/* Trapezoid weights on arbitrary increasing nodes x[0..n-1]:
 * w_0 = (x_1-x_0)/2, w_i = (x_{i+1}-x_{i-1})/2, w_{n-1} = (x_{n-1}-x_{n-2})/2.
 * n == 1 gives w_0 = 0 (a single node spans no interval). */
void orc_trapz_weights(int n, const double *x, double *w)
{
    if (n <= 0) return;
    if (n == 1) { w[0] = 0.0; return; }
    w[0] = 0.5 * (x[1] - x[0]);
    for (int i = 1; i < n - 1; ++i) w[i] = 0.5 * (x[i + 1] - x[i - 1]);
    w[n - 1] = 0.5 * (x[n - 1] - x[n - 2]);
}

/* Trapezoid weights in u = ln k, for the dk/k measure of Eq. (1). */
void orc_lnk_weights(int n, const double *k, double *w)
{
    if (n <= 0) return;
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) u[i] = log(k[i]);
    orc_trapz_weights(n, u, w);
    free(u);
}

/* ------------------------------------------------------------------------ */
/* Spherical Bessel functions j_0..j_lmax at one argument                   */
/* ------------------------------------------------------------------------ */

/* j[l], l = 0..lmax, for x >= 0. */
void orc_sph_bessel(int lmax, double x, double *j)
{
    if (lmax < 0) return;
    if (x == 0.0) {
        j[0] = 1.0;
        for (int l = 1; l <= lmax; ++l) j[l] = 0.0;
        return;
    }
    if (x < 1e-3) {
        /* Power series (the definition):
         * j_l(x) = x^l/(2l+1)!! [1 - x^2/(2(2l+3)) + x^4/(8(2l+3)(2l+5)) - ...];
         * the dropped terms are below 1e-21 relative.  The backward recurrence
         * would overflow here, its step factor (2l+1)/x being huge. */
        double t = 1.0, x2 = x * x;  /* t = x^l / (2l+1)!! */
        for (int l = 0; l <= lmax; ++l) {
            if (l > 0) t *= x / (2.0 * l + 1.0);
            double a = 2.0 * l + 3.0, b = 2.0 * l + 5.0;
            j[l] = t * (1.0 - x2 / (2.0 * a) + x2 * x2 / (8.0 * a * b));
        }
        return;
    }
    /* Orders at or below ls come from the forward recurrence (x >= 1). */
    int ls = -1;
    if (x >= 1.0) {
        double fl = floor(x);
        ls = fl > (double)lmax ? lmax : (int)fl;
        double s = sin(x), c = cos(x);
        j[0] = s / x;
        if (lmax >= 1) j[1] = (s / x - c) / x;
        for (int l = 1; l < ls; ++l) j[l + 1] = (2.0 * l + 1.0) / x * j[l] - j[l - 1];
        if (ls == lmax) return;
    }
    /* Backward recurrence from a start far above max(lmax, x). */
    double big = x > (double)lmax ? ceil(x) : (double)lmax;
    int Lstart = (int)big + 30 + (int)ceil(2.0 * cbrt(big)) + (int)ceil(sqrt(40.0 * big));
    int lo = (x < 1.0) ? 0 : ls - 1;      /* lowest order the backward pass reaches */
    double fhi = 0.0;                      /* f_{l+1} */
    double f = 1e-300;                     /* f_l, starting at l = Lstart */
    double f_at_ls = 0.0, f_at_lsm1 = 0.0; /* backward values at the matching pair */
    /* The backward values for orders above ls are stored straight into j[];
     * orders ls and ls-1 keep their forward values, their backward values are
     * kept aside for the normalisation. */
    for (int l = Lstart; l >= lo; --l) {
        if (l <= lmax && l > ls) j[l] = f;
        if (l == ls) f_at_ls = f;
        if (l == ls - 1) f_at_lsm1 = f;
        if (x < 1.0 && l <= lmax) j[l] = f;
        if (l == lo) break;
        double fm = (2.0 * l + 1.0) / x * f - fhi;   /* f_{l-1} */
        fhi = f;
        f = fm;
        if (fabs(f) > 1e250) {                        /* rescale everything kept */
            f *= 1e-250;
            fhi *= 1e-250;
            int top = Lstart < lmax ? Lstart : lmax;
            for (int q = l; q <= top; ++q)
                if (q > ls || x < 1.0) j[q] *= 1e-250;
            if (l <= ls) f_at_ls *= 1e-250;
        }
    }
    double scale;
    if (x < 1.0) {
        double j0 = sin(x) / x;
        scale = j0 / j[0];
        int top = Lstart < lmax ? Lstart : lmax;
        for (int l = 0; l <= top; ++l) j[l] *= scale;
        for (int l = top + 1; l <= lmax; ++l) j[l] = 0.0;
        return;
    }
    /* Match at whichever of (ls-1, ls) has the larger forward magnitude. */
    if (fabs(j[ls]) >= fabs(j[ls - 1])) scale = j[ls] / f_at_ls;
    else scale = j[ls - 1] / f_at_lsm1;
    int top = Lstart < lmax ? Lstart : lmax;
    for (int l = ls + 1; l <= top; ++l) j[l] *= scale;
    for (int l = top + 1; l <= lmax; ++l) j[l] = 0.0;
}

/* out[n][lmax+1] for many arguments. */
void orc_sph_bessel_many(int n, const double *x, int lmax, double *out)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) orc_sph_bessel(lmax, x[i], out + (size_t)i * (size_t)(lmax + 1));
}

/* ------------------------------------------------------------------------ */
/* Line-of-sight transfer (Eq. 2) and C_l (Eq. 1)                           */
/* ------------------------------------------------------------------------ */

/*
 * S     [M][nk][ntau]   source function on the nodes
 * Pk    [M][nk]         primordial spectrum (may be NULL if Cl == NULL)
 * Delta [M][nk][nl]     output transfer functions, nl = lmax-lmin+1 (may be NULL)
 * Cl    [M][nl]         output spectra (may be NULL)
 * wtau, wk: optional caller weights (NULL = trapezoid in tau / in ln k).
 * Returns 0 on success, -1 on bad arguments.
 *
 * Parallel over k; each thread keeps private C_l partial sums, which are added
 * in thread order at the end.
 */
int orc_los_cl(int nk, const double *k, int ntau, const double *tau, double tau0,
               int lmin, int lmax, int M, const double *S, const double *Pk,
               const double *wtau_in, const double *wk_in,
               double *Delta, double *Cl, int nthreads)
{
    if (nk < 0 || ntau < 0 || lmin < 0 || lmax < lmin || M < 0) return -1;
    const int nl = lmax - lmin + 1;
    double *wtau = (double *)malloc(sizeof(double) * (size_t)(ntau > 0 ? ntau : 1));
    double *wk = (double *)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    if (wtau_in) memcpy(wtau, wtau_in, sizeof(double) * (size_t)ntau);
    else orc_trapz_weights(ntau, tau, wtau);
    if (wk_in) memcpy(wk, wk_in, sizeof(double) * (size_t)nk);
    else orc_lnk_weights(nk, k, wk);
    if (Cl) memset(Cl, 0, sizeof(double) * (size_t)M * (size_t)nl);

    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    double *clpart = NULL;
    if (Cl) clpart = (double *)calloc((size_t)nt * (size_t)M * (size_t)nl, sizeof(double));

    #pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *jl = (double *)malloc(sizeof(double) * (size_t)(lmax + 1));
        double *dk = (double *)malloc(sizeof(double) * (size_t)M * (size_t)nl);
        #pragma omp for schedule(static)
        for (int q = 0; q < nk; ++q) {
            memset(dk, 0, sizeof(double) * (size_t)M * (size_t)nl);
            for (int i = 0; i < ntau; ++i) {
                double x = k[q] * (tau0 - tau[i]);
                orc_sph_bessel(lmax, x, jl);
                for (int m = 0; m < M; ++m) {
                    double ws = wtau[i] * S[((size_t)m * nk + q) * ntau + i];
                    double *d = dk + (size_t)m * nl;
                    for (int l = lmin; l <= lmax; ++l) d[l - lmin] += ws * jl[l];
                }
            }
            if (Delta)
                for (int m = 0; m < M; ++m)
                    memcpy(Delta + ((size_t)m * nk + q) * nl, dk + (size_t)m * nl, sizeof(double) * (size_t)nl);
            if (Cl) {
                double *cp = clpart + (size_t)tid * M * nl;
                for (int m = 0; m < M; ++m) {
                    double f = 4.0 * M_PI * wk[q] * Pk[(size_t)m * nk + q];
                    const double *d = dk + (size_t)m * nl;
                    for (int l = 0; l < nl; ++l) cp[(size_t)m * nl + l] += f * d[l] * d[l];
                }
            }
        }
        free(jl);
        free(dk);
    }
    if (Cl) {
        for (int t = 0; t < nt; ++t)
            for (size_t e = 0; e < (size_t)M * nl; ++e) Cl[e] += clpart[(size_t)t * M * nl + e];
        free(clpart);
    }
    free(wtau);
    free(wk);
    return 0;
}

/* C_l from given transfer functions: Cl[m][l] = 4 pi sum_j wk_j P[m][j] Delta[m][j][l]^2,
 * summed in increasing j.  wk_in NULL = trapezoid in ln k. */
int orc_cl(int nk, const double *k, int nl, int M, const double *Delta, const double *Pk,
           const double *wk_in, double *Cl)
{
    if (nk < 0 || nl < 0 || M < 0) return -1;
    double *wk = (double *)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    if (wk_in) memcpy(wk, wk_in, sizeof(double) * (size_t)nk);
    else orc_lnk_weights(nk, k, wk);
    for (int m = 0; m < M; ++m)
        for (int l = 0; l < nl; ++l) {
            double acc = 0.0;
            for (int q = 0; q < nk; ++q) {
                double d = Delta[((size_t)m * nk + q) * nl + l];
                acc += 4.0 * M_PI * wk[q] * Pk[(size_t)m * nk + q] * d * d;
            }
            Cl[(size_t)m * nl + l] = acc;
        }
    free(wk);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* E-mode polarisation                                                      */
/* ------------------------------------------------------------------------ */

/* eps_l(x) for l = 0..lmax into e[0..lmax] (see the header). */
void orc_eps(int lmax, double x, double *e)
{
    double *jl = (double *)malloc(sizeof(double) * (size_t)(lmax + 1));
    orc_sph_bessel(lmax, x, jl);
    for (int l = 0; l <= lmax; ++l) {
        if (l < 2) {
            e[l] = 0.0;
            continue;
        }
        double c = sqrt((double)(l + 2) * (double)(l + 1) * (double)l * (double)(l - 1));
        if (x == 0.0)
            e[l] = (l == 2) ? c / 15.0 : 0.0;  /* j_2(x)/x^2 -> 1/15; higher orders vanish */
        else
            e[l] = c * jl[l] / (x * x);
    }
    free(jl);
}

void orc_eps_many(int n, const double *x, int lmax, double *out)
{
    for (int i = 0; i < n; ++i) orc_eps(lmax, x[i], out + (size_t)i * (lmax + 1));
}

/* Delta^E[m][q][l - lmin] = sum_i w_i S_P[m][q][i] eps_l(k_q (tau0 - tau_i)),
 * dense over the tau nodes.  wtau_in NULL = trapezoid.  Returns 0 or -1. */
int orc_los_e(int nk, const double *k, int ntau, const double *tau, double tau0,
              int lmin, int lmax, int M, const double *SP, const double *wtau_in,
              double *DeltaE, int nthreads)
{
    if (nk < 0 || ntau < 0 || lmin < 0 || lmax < lmin || M < 0 || !DeltaE) return -1;
    const int nl = lmax - lmin + 1;
    double *wtau = (double *)malloc(sizeof(double) * (size_t)(ntau > 0 ? ntau : 1));
    if (wtau_in) memcpy(wtau, wtau_in, sizeof(double) * (size_t)ntau);
    else orc_trapz_weights(ntau, tau, wtau);
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    #pragma omp parallel num_threads(nt)
    {
        double *el = (double *)malloc(sizeof(double) * (size_t)(lmax + 1));
        #pragma omp for schedule(static)
        for (int q = 0; q < nk; ++q) {
            for (int m = 0; m < M; ++m)
                memset(DeltaE + ((size_t)m * nk + q) * nl, 0, sizeof(double) * (size_t)nl);
            for (int i = 0; i < ntau; ++i) {
                orc_eps(lmax, k[q] * (tau0 - tau[i]), el);
                for (int m = 0; m < M; ++m) {
                    double ws = wtau[i] * SP[((size_t)m * nk + q) * ntau + i];
                    double *d = DeltaE + ((size_t)m * nk + q) * nl;
                    for (int l = lmin; l <= lmax; ++l) d[l - lmin] += ws * el[l];
                }
            }
        }
        free(el);
    }
    free(wtau);
    return 0;
}

/* Hyperspherical Bessel Phi^beta_l(chi), l = 0..lmax, open (closed = 0) or
 * closed (closed = 1) space; see the header. */
void orc_hyper_bessel(int lmax, double beta, double chi, int closed, double *out)
{
    for (int l = 0; l <= lmax; ++l) out[l] = 0.0;
    if (chi == 0.0) {
        out[0] = 1.0;
        return;
    }
    const double sh = closed ? sin(chi) : sinh(chi);
    const double ct = closed ? cos(chi) / sin(chi) : cosh(chi) / sinh(chi);
    const double p0 = sin(beta * chi) / (beta * sh);
    const double s1 = closed ? sqrt(beta * beta - 1.0) : sqrt(beta * beta + 1.0);
    const double p1 = (sin(beta * chi) * ct - beta * cos(beta * chi)) / (beta * sh * s1);
    /* start far above the order range and the classical turning order
     * beta |sh(chi)|; above it the decaying solution falls by about
     * tanh(chi/2) per order in open space (the recurrence's roots tend to
     * (cosh chi -+ 1)/sinh chi), so the start also clears
     * 46 / -ln tanh(chi/2) orders (a factor e^-46); in closed space at most
     * l = beta - 1, where Phi_beta = 0 makes the start exact */
    const double turn = beta * fabs(sh);
    const double hi = lmax > turn ? (double)lmax : turn;
    double extra = 0.0;
    if (!closed) extra = fmin(46.0 / -log(tanh(0.5 * chi)), 1e6);
    int top = (int)(hi + 60.0 + 8.0 * sqrt(hi) + extra) + 10;
    if (closed && top > (int)llround(beta) - 1) top = (int)llround(beta) - 1;
    if (top < 1) {
        if (lmax >= 0) out[0] = p0;
        return;
    }
    /* downward: s_l Phi_(l-1) = (2l+1) ct Phi_l - s_(l+1) Phi_(l+1) */
    int n = top + 1;
    double *f = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    f[n] = 0.0;
    f[top] = 1e-300;
    for (int l = top; l >= 1; --l) {
        const double sl = closed ? sqrt(beta * beta - (double)l * l) : sqrt(beta * beta + (double)l * l);
        const double sl1 = closed ? sqrt(fmax(beta * beta - (double)(l + 1) * (l + 1), 0.0))
                                  : sqrt(beta * beta + (double)(l + 1) * (l + 1));
        f[l - 1] = ((2.0 * l + 1.0) * ct * f[l] - sl1 * f[l + 1]) / sl;
        if (fabs(f[l - 1]) > 1e250) {  /* rescale what is still needed: the outputs and f[l], f[l+1] */
            const int hi2 = (l + 1 > lmax ? l + 1 : lmax);
            for (int j = l - 1; j <= hi2 && j <= n; ++j) f[j] *= 1e-250;
        }
    }
    const double norm = fabs(p0) >= fabs(p1) ? p0 / f[0] : p1 / f[1];
    for (int l = 0; l <= lmax && l <= top; ++l) out[l] = f[l] * norm;
    free(f);
}

void orc_hyper_bessel_many(int n, const double *beta, const double *chi, int lmax, int closed, double *out)
{
    for (int i = 0; i < n; ++i) orc_hyper_bessel(lmax, beta[i], chi[i], closed, out + (size_t)i * (lmax + 1));
}

/* Curved-space transfer functions Delta[M][q][l - lmin] = sum_i w_i S[m][q][i]
 * Phi^(q/sqrt|K|)_l(sqrt|K| (tau0 - tau_i)), K != 0; dense over the nodes. */
int orc_los_curved(int nq, const double *q, int ntau, const double *tau, double tau0, double K,
                   int lmin, int lmax, int M, const double *S, const double *wtau_in, double *Delta, int nthreads)
{
    if (nq < 0 || ntau < 0 || lmin < 0 || lmax < lmin || M < 0 || !Delta || K == 0.0) return -1;
    const int nl = lmax - lmin + 1;
    const int closed = K > 0.0;
    const double rk = sqrt(fabs(K));
    double *wtau = (double *)malloc(sizeof(double) * (size_t)(ntau > 0 ? ntau : 1));
    if (wtau_in) memcpy(wtau, wtau_in, sizeof(double) * (size_t)ntau);
    else orc_trapz_weights(ntau, tau, wtau);
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    #pragma omp parallel num_threads(nt)
    {
        double *ph = (double *)malloc(sizeof(double) * (size_t)(lmax + 1));
        #pragma omp for schedule(dynamic)
        for (int j = 0; j < nq; ++j) {
            for (int m = 0; m < M; ++m) memset(Delta + ((size_t)m * nq + j) * nl, 0, sizeof(double) * (size_t)nl);
            for (int i = 0; i < ntau; ++i) {
                orc_hyper_bessel(lmax, q[j] / rk, rk * (tau0 - tau[i]), closed, ph);
                for (int m = 0; m < M; ++m) {
                    const double ws = wtau[i] * S[((size_t)m * nq + j) * ntau + i];
                    double *d = Delta + ((size_t)m * nq + j) * nl;
                    for (int l = lmin; l <= lmax; ++l) d[l - lmin] += ws * ph[l];
                }
            }
        }
        free(ph);
    }
    free(wtau);
    return 0;
}

/* Tensor kernels t_l, e_l, b_l at one x for l = 0..lmax (zero below l = 2). */
void orc_tensor_kernels(int lmax, double x, double *t, double *e, double *b)
{
    double *jl = (double *)malloc(sizeof(double) * (size_t)(lmax + 1));
    orc_sph_bessel(lmax, x, jl);
    for (int l = 0; l <= lmax; ++l) {
        t[l] = e[l] = b[l] = 0.0;
        if (l < 2) continue;
        double c = sqrt((double)(l + 2) * (double)(l + 1) * (double)l * (double)(l - 1));
        if (x == 0.0) {
            if (l == 2) {
                t[l] = c / 15.0;
                e[l] = 0.8;
            }
            continue;
        }
        t[l] = c * jl[l] / (x * x);
        e[l] = ((double)l * (double)(l - 1) / (x * x) - 2.0) * jl[l] + 2.0 * jl[l - 1] / x;
        b[l] = 2.0 * jl[l - 1] - 2.0 * (double)(l - 1) * jl[l] / x;
    }
    free(jl);
}

void orc_tensor_kernels_many(int n, const double *x, int lmax, double *t, double *e, double *b)
{
    for (int i = 0; i < n; ++i) {
        size_t o = (size_t)i * (lmax + 1);
        orc_tensor_kernels(lmax, x[i], t + o, e + o, b + o);
    }
}

/* Tensor transfer functions DT, DE, DB [M][q][l - lmin] = sum_i w_i S[m][q][i]
 * kernel_l(k_q (tau0 - tau_i)), S = ST for t_l and SP for e_l, b_l; dense
 * over the tau nodes.  wtau_in NULL = trapezoid.  Returns 0 or -1. */
int orc_los_tensor(int nk, const double *k, int ntau, const double *tau, double tau0,
                   int lmin, int lmax, int M, const double *ST, const double *SP,
                   const double *wtau_in, double *DT, double *DE, double *DB, int nthreads)
{
    if (nk < 0 || ntau < 0 || lmin < 0 || lmax < lmin || M < 0 || !DT || !DE || !DB) return -1;
    const int nl = lmax - lmin + 1;
    double *wtau = (double *)malloc(sizeof(double) * (size_t)(ntau > 0 ? ntau : 1));
    if (wtau_in) memcpy(wtau, wtau_in, sizeof(double) * (size_t)ntau);
    else orc_trapz_weights(ntau, tau, wtau);
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    #pragma omp parallel num_threads(nt)
    {
        double *kt = (double *)malloc(sizeof(double) * 3 * (size_t)(lmax + 1));
        double *ke = kt + (lmax + 1), *kb = ke + (lmax + 1);
        #pragma omp for schedule(static)
        for (int q = 0; q < nk; ++q) {
            for (int m = 0; m < M; ++m) {
                size_t o = ((size_t)m * nk + q) * nl;
                memset(DT + o, 0, sizeof(double) * (size_t)nl);
                memset(DE + o, 0, sizeof(double) * (size_t)nl);
                memset(DB + o, 0, sizeof(double) * (size_t)nl);
            }
            for (int i = 0; i < ntau; ++i) {
                orc_tensor_kernels(lmax, k[q] * (tau0 - tau[i]), kt, ke, kb);
                for (int m = 0; m < M; ++m) {
                    size_t s = ((size_t)m * nk + q) * ntau + i, o = ((size_t)m * nk + q) * nl;
                    double wt = wtau[i] * ST[s], wp = wtau[i] * SP[s];
                    for (int l = lmin; l <= lmax; ++l) {
                        DT[o + l - lmin] += wt * kt[l];
                        DE[o + l - lmin] += wp * ke[l];
                        DB[o + l - lmin] += wp * kb[l];
                    }
                }
            }
        }
        free(kt);
    }
    free(wtau);
    return 0;
}

/* Cross spectrum Cl[m][l] = 4 pi sum_j wk_j P[m][j] DX[m][j][l] DY[m][j][l],
 * summed in increasing j.  wk_in NULL = trapezoid in ln k. */
int orc_cl_cross(int nk, const double *k, int nl, int M, const double *DX, const double *DY,
                 const double *Pk, const double *wk_in, double *Cl)
{
    if (nk < 0 || nl < 0 || M < 0) return -1;
    double *wk = (double *)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    if (wk_in) memcpy(wk, wk_in, sizeof(double) * (size_t)nk);
    else orc_lnk_weights(nk, k, wk);
    for (int m = 0; m < M; ++m)
        for (int l = 0; l < nl; ++l) {
            double acc = 0.0;
            for (int q = 0; q < nk; ++q) {
                size_t e = ((size_t)m * nk + q) * nl + l;
                acc += 4.0 * M_PI * wk[q] * Pk[(size_t)m * nk + q] * DX[e] * DY[e];
            }
            Cl[(size_t)m * nl + l] = acc;
        }
    free(wk);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
