"""Pins for the oracle's line-of-sight transfer (Eq. 2) and C_l k-integral
(Eq. 1): quadrature exactness and error bounds, a delta-function source,
closed-form integrals of j_0 and j_1, linearity, the Sachs-Wolfe plateau, and
brute force against mpmath on tiny grids."""
import math

import numpy as np
import pytest

from paper_2509_25110_gb300 import synth
from tests.conftest import jl_mpmath


# ---------------------------------------------------------------- weights

def test_trapz_exact_on_linear(orc):
    rng = np.random.default_rng(0)
    for n in (2, 3, 7, 50):
        x = np.sort(rng.uniform(-3, 5, n))
        w = orc.trapz_weights(x)
        a, b = rng.normal(size=2)
        exact = a * (x[-1] - x[0]) + b * (x[-1] ** 2 - x[0] ** 2) / 2
        assert abs(np.dot(w, a + b * x) - exact) <= 1e-13 * (abs(exact) + 1)
        assert abs(w.sum() - (x[-1] - x[0])) <= 1e-14 * (x[-1] - x[0])
    assert orc.trapz_weights(np.array([4.0]))[0] == 0.0
    assert np.allclose(orc.trapz_weights(np.array([1.0, 3.0])), [1.0, 1.0])


def test_lnk_weights_are_trapezoid_in_lnk(orc):
    k = synth.log_grid(1e-4, 0.3, 300)
    w = orc.lnk_weights(k)
    u = np.log(k)
    # exact for integrands linear in u = ln k (dk/k measure)
    assert abs(w.sum() - (u[-1] - u[0])) <= 1e-13
    assert abs(np.dot(w, u) - (u[-1] ** 2 - u[0] ** 2) / 2) <= 1e-12
    # non-uniform grid
    k2 = synth.master_linear_k(50)
    w2 = orc.lnk_weights(k2)
    u2 = np.log(k2)
    assert abs(np.dot(w2, 2 - 3 * u2) - (2 * (u2[-1] - u2[0]) - 1.5 * (u2[-1] ** 2 - u2[0] ** 2))) < 1e-12


# ---------------------------------------------------------------- transfer

def test_delta_source_gives_bessel(orc):
    """S_i = delta_{i,i*} / w_{i*}  =>  Delta_l(k) = j_l(k (tau0 - tau_{i*}))."""
    tau = np.linspace(200.0, 14000.0, 40)
    k = synth.log_grid(1e-3, 0.3, 12)
    w = orc.trapz_weights(tau)
    istar = 17
    S = np.zeros((k.size, tau.size))
    S[:, istar] = 1.0 / w[istar]
    delta, _ = orc.los_cl(k, tau, 14000.0, 2, 300, S, want_cl=False)
    for q in range(k.size):
        x = k[q] * (14000.0 - tau[istar])
        ref = orc.sph_bessel(300, x)[2:]
        assert np.allclose(delta[q], ref, rtol=1e-15, atol=1e-300)
    # tie two of them to mpmath
    for q, l in ((5, 2), (11, 250)):
        x = k[q] * (14000.0 - tau[istar])
        r = jl_mpmath(l, x)
        assert abs(delta[q, l - 2] - r) <= 1e-12 * abs(r)


def test_constant_source_closed_forms(orc):
    """S = 1 on [ta, tb]: Delta_0 = (Si(xa) - Si(xb))/k and Delta_1 = (j0(xb) - j0(xa))/k,
    x = k (tau0 - tau).  Trapezoid error <= (tb-ta) h^2 max|f''| / 12 with |j_l''| <= 1."""
    sp = pytest.importorskip("scipy.special")
    tau0, ta, tb = 14000.0, 200.0, 14000.0
    k = np.array([1e-4, 3e-3, 0.02, 0.05])
    errs = []
    for n in (201, 401, 801):
        tau = np.linspace(ta, tb, n)
        h = tau[1] - tau[0]
        delta, _ = orc.los_cl(k, tau, tau0, 0, 1, np.ones((k.size, n)), want_cl=False)
        e = []
        for q, kk in enumerate(k):
            xa, xb = kk * (tau0 - ta), kk * (tau0 - tb)
            si_a, si_b = sp.sici(xa)[0], sp.sici(xb)[0]
            d0 = (si_a - si_b) / kk
            j0 = lambda x: 1.0 if x == 0 else math.sin(x) / x
            d1 = (j0(xb) - j0(xa)) / kk
            bound = (tb - ta) * h * h * kk * kk / 12 + 1e-12 * (tb - ta)
            assert abs(delta[q, 0] - d0) <= bound
            assert abs(delta[q, 1] - d1) <= bound
            e.append(abs(delta[q, 1] - d1))
        errs.append(e)
    errs = np.array(errs)
    # second-order convergence where the error is well above rounding (k = 0.05)
    r = errs[:-1, 3] / errs[1:, 3]
    assert np.all((r > 3.5) & (r < 4.5)), r


def test_linearity(orc):
    rng = np.random.default_rng(5)
    tau = np.linspace(200.0, 14000.0, 60)
    k = synth.log_grid(1e-3, 0.2, 9)
    S1 = rng.normal(size=(k.size, tau.size))
    S2 = rng.normal(size=(k.size, tau.size))
    d1, _ = orc.los_cl(k, tau, 14000.0, 2, 120, S1, want_cl=False)
    d2, _ = orc.los_cl(k, tau, 14000.0, 2, 120, S2, want_cl=False)
    d3, _ = orc.los_cl(k, tau, 14000.0, 2, 120, 2 * S1 - 3 * S2, want_cl=False)
    scale = np.abs(d1).max() + np.abs(d2).max()
    assert np.abs(d3 - (2 * d1 - 3 * d2)).max() <= 1e-12 * scale


# ---------------------------------------------------------------- C_l

def test_cl_scales_with_primordial_amplitude(orc):
    wl = synth.workload("plain_lmax500")
    p = synth.model_params(2, seed=1)
    k, tau = wl.k[::10], wl.tau[::8]
    S = synth.sources(k, tau, p)
    P = synth.primordial(k, p)
    _, c1 = orc.los_cl(k, tau, wl.tau0, 2, 60, S, P)
    _, c3 = orc.los_cl(k, tau, wl.tau0, 2, 60, S, 3.0 * P)
    assert np.allclose(c3, 3.0 * c1, rtol=1e-14, atol=0)
    d, _ = orc.los_cl(k, tau, wl.tau0, 2, 60, S, want_cl=False)
    assert np.allclose(orc.cl_from_delta(k, d, P), c1, rtol=1e-13, atol=0)


def test_sachs_wolfe_plateau(orc):
    """Delta source at r* with P = A (n_s = 1):
    C_l = 4 pi A int j_l(k r*)^2 dk/k = 2 pi A / (l (l+1))."""
    tau0 = 14000.0
    tau = np.array([13000.0, 13500.0, 13900.0])
    istar = 1
    rstar = tau0 - tau[istar]
    w = orc.trapz_weights(tau)
    xs_log = np.exp(np.arange(math.log(1e-3), math.log(10.0), 0.004))
    xs_lin = np.arange(10.0, 2e4 + 1e-9, 0.05)
    x = np.concatenate([xs_log, xs_lin[1:] if xs_log[-1] >= 10.0 else xs_lin])
    k = x / rstar
    S = np.zeros((k.size, tau.size))
    S[:, istar] = 1.0 / w[istar]
    A = 2.1e-9
    _, cl = orc.los_cl(k, tau, tau0, 2, 50, S, np.full(k.size, A))
    l = np.arange(2, 51)
    ref = 2 * math.pi * A / (l * (l + 1))
    assert np.abs(cl / ref - 1).max() <= 1e-4


def test_brute_force_tiny_grid(orc):
    """The discrete sums of Eqs. 1-2 evaluated in 30-digit mpmath on a tiny grid."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    rng = np.random.default_rng(9)
    tau0 = 14000.0
    tau = np.sort(rng.uniform(200.0, 13990.0, 6))
    k = np.sort(rng.uniform(1e-3, 0.05, 7))
    M, lmin, lmax = 2, 0, 4
    S = rng.normal(size=(M, k.size, tau.size))
    P = rng.uniform(1e-9, 3e-9, size=(M, k.size))
    delta, cl = orc.los_cl(k, tau, tau0, lmin, lmax, S, P)
    T = [mp.mpf(t) for t in tau]
    U = [mp.log(mp.mpf(q)) for q in k]

    def trap(nodes):
        n = len(nodes)
        return [(nodes[1] - nodes[0]) / 2] + [(nodes[i + 1] - nodes[i - 1]) / 2 for i in range(1, n - 1)] + \
               [(nodes[-1] - nodes[-2]) / 2]
    wt, wk = trap(T), trap(U)
    for m in range(M):
        for l in range(lmin, lmax + 1):
            c = mp.mpf(0)
            for q in range(k.size):
                d = mp.mpf(0)
                mag = mp.mpf(0)
                for i in range(tau.size):
                    # the argument at the FP64 node (j_l(x) amplifies x's rounding by ~x)
                    x = mp.mpf(float(k[q] * (tau0 - tau[i])))
                    jv = mp.besselj(l + mp.mpf(1) / 2, x) * mp.sqrt(mp.pi / (2 * x))
                    d += wt[i] * mp.mpf(S[m, q, i]) * jv
                    mag += abs(wt[i] * mp.mpf(S[m, q, i]) * jv)
                assert abs(delta[m, q, l] - float(d)) <= 1e-14 * float(mag)
                c += 4 * mp.pi * wk[q] * mp.mpf(P[m, q]) * d * d
            assert abs(cl[m, l] - float(c)) <= 1e-13 * float(c)


def test_cosmic_variance_ratio_helper(orc):
    cl = np.array([1.0, 2.0, 4.0])
    r = orc.cosmic_variance_ratio(cl * 1.01, cl, lmin=2)
    l = np.arange(2, 5)
    assert np.allclose(r, 0.01 / np.sqrt(2 / (2 * l + 1)))
