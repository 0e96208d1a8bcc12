"""Pins for the oracle's E-mode polarisation (Eq. 3) and cross spectra (Eq. 1,
X, Y in {T, E}), with eps_l(x) = sqrt((l+2)!/(l-2)!) j_l(x)/x^2.

Each pin fails on a plausible slip: the l = 2 closed form and the mpmath
values catch a wrong prefactor or power of x; the x -> 0 limits catch the
treatment of the x = 0 node; the delta source catches the quadrature; the
scale-invariant closed forms (Weber-Schafheitlin integrals) catch the whole
EE and TE chain; Cauchy-Schwarz and the auto case catch the cross sum."""
import math

import numpy as np
import pytest


def c_l(l):
    return np.sqrt((l + 2.0) * (l + 1.0) * l * (l - 1.0))


def test_eps2_closed_form(orc):
    x = np.linspace(0.5, 2e3, 4001)
    j2 = (3.0 / x ** 2 - 1.0) * np.sin(x) / x - 3.0 * np.cos(x) / x ** 2
    ref = math.sqrt(24.0) * j2 / x ** 2
    got = orc.eps(x, 2)[:, 2]
    env = math.sqrt(24.0) / x ** 3  # |j_2| <= ~1/x: compare on the envelope
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(env).max()
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-12
    assert np.all(orc.eps(x, 6)[:, :2] == 0.0)  # eps_0 = eps_1 = 0


def test_eps_mpmath(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    rng = np.random.default_rng(21)
    for _ in range(40):
        l = int(rng.integers(2, 400))
        x = float(rng.uniform(0.05, 1500.0))
        ref = mp.sqrt(mp.mpf(l + 2) * (l + 1) * l * (l - 1)) * mp.sqrt(mp.pi / (2 * mp.mpf(x))) * \
            mp.besselj(l + mp.mpf(1) / 2, x) / mp.mpf(x) ** 2
        got = orc.eps(np.array([x]), l)[0, l]
        env = float(c_l(l)) / x ** 2 / max(1.0, math.sqrt(max(x * x - l * l, 1.0)))  # scale near the value
        if abs(float(ref)) < 1e-250:
            continue
        assert abs(got - float(ref)) <= 1e-11 * max(abs(float(ref)), 1e-3 * env), (l, x, got, float(ref))


def test_eps_at_and_near_zero(orc):
    e0 = orc.eps(np.array([0.0]), 8)[0]
    assert e0[2] == pytest.approx(math.sqrt(24.0) / 15.0, rel=1e-15)
    assert np.all(e0[3:] == 0.0) and np.all(e0[:2] == 0.0)
    # leading terms of the power series: j_l(x) = x^l/(2l+1)!! (1 - x^2/(2(2l+3)) + ...)
    x = 1e-3
    e = orc.eps(np.array([x]), 8)[0]
    for l in range(2, 9):
        dfact = float(np.prod(np.arange(2 * l + 1, 0, -2)))
        ref = c_l(l) * x ** (l - 2) / dfact * (1.0 - x * x / (2.0 * (2 * l + 3)))
        assert e[l] == pytest.approx(ref, rel=1e-10), l


def test_delta_source_gives_eps(orc):
    tau0 = 14000.0
    tau = np.linspace(200.0, 14000.0, 60)
    k = np.geomspace(1e-4, 0.3, 30)
    w = orc.trapz_weights(tau)
    i = 37
    SP = np.zeros((k.size, tau.size))
    SP[:, i] = 1.0 / w[i]
    d = orc.los_e(k, tau, tau0, 2, 300, SP)
    ref = orc.eps(k * (tau0 - tau[i]), 300)[:, 2:]
    assert np.abs(d - ref).max() <= 1e-14 * np.abs(ref).max()


def _sw_grid(orc, rstar):
    xs_log = np.exp(np.arange(math.log(1e-3), math.log(10.0), 0.004))
    xs_lin = np.arange(10.0, 2e4 + 1e-9, 0.05)
    x = np.concatenate([xs_log, xs_lin[1:] if xs_log[-1] >= 10.0 else xs_lin])
    return x / rstar


def test_scale_invariant_ee_and_te_closed_forms(orc):
    """Delta sources at r* in T and E, P = A:
    C^EE_l = 4 pi A c_l^2 int j_l^2 x^-5 dx = (16 pi A / 15) / ((l+3)(l-2))   (l >= 3),
    C^TE_l = 4 pi A c_l   int j_l^2 x^-3 dx = (4 pi A / 3) / c_l              (l >= 2),
    from int_0^inf J_nu(t)^2 t^-lam dt = Gamma(lam) Gamma(nu + (1-lam)/2) /
    (2^lam Gamma((1+lam)/2)^2 Gamma(nu + (1+lam)/2))."""
    tau0 = 14000.0
    tau = np.array([13000.0, 13500.0, 13900.0])
    istar = 1
    rstar = tau0 - tau[istar]
    w = orc.trapz_weights(tau)
    k = _sw_grid(orc, rstar)
    S = np.zeros((k.size, tau.size))
    S[:, istar] = 1.0 / w[istar]
    A = 2.1e-9
    P = np.full(k.size, A)
    dT, _ = orc.los_cl(k, tau, tau0, 2, 40, S, P, want_cl=False)
    dE = orc.los_e(k, tau, tau0, 2, 40, S)
    ee = orc.cl_cross(k, dE, dE, P)
    te = orc.cl_cross(k, dT, dE, P)
    l = np.arange(2, 41)
    ref_ee = 16.0 * math.pi * A / 15.0 / ((l + 3.0) * (l - 2.0))[1:]
    ref_te = 4.0 * math.pi * A / 3.0 / c_l(l)
    assert np.abs(ee[1:] / ref_ee - 1).max() <= 1e-4
    assert np.abs(te / ref_te - 1).max() <= 1e-4


def test_cross_spectrum_properties(orc):
    rng = np.random.default_rng(4)
    tau0 = 14000.0
    tau = np.linspace(200.0, 13900.0, 80)
    k = np.geomspace(1e-4, 0.2, 50)
    M = 3
    ST = rng.normal(size=(M, k.size, tau.size))
    SP = rng.normal(size=(M, k.size, tau.size))
    P = rng.uniform(1e-9, 3e-9, (M, k.size))
    dT, tt = orc.los_cl(k, tau, tau0, 2, 120, ST, P)
    dE = orc.los_e(k, tau, tau0, 2, 120, SP)
    ee = orc.cl_cross(k, dE, dE, P)
    te = orc.cl_cross(k, dT, dE, P)
    assert np.all(te ** 2 <= tt * ee * (1 + 1e-12))              # Cauchy-Schwarz
    assert np.allclose(orc.cl_cross(k, dT, dT, P), tt, rtol=1e-13, atol=0)  # the auto case is Eq. (1)
    assert np.allclose(orc.cl_cross(k, dE, dT, P), te, rtol=1e-13, atol=0)  # symmetric (to rounding)
    # linearity in S_P (on the scale of the sums: random terms cancel)
    assert np.abs(orc.los_e(k, tau, tau0, 2, 120, 2.5 * SP) - 2.5 * dE).max() <= 1e-13 * np.abs(2.5 * dE).max()


def test_cosmic_variance_te_reduces_to_the_auto_form(orc):
    """Fully correlated fields (TE^2 = TT EE, here TT = EE = TE) give the auto
    spectrum's sigma_CV = sqrt(2/(2l+1)) |C|."""
    rng = np.random.default_rng(5)
    c = rng.uniform(1e-12, 1e-9, 50)
    d = 1e-3 * c
    r_te = orc.cosmic_variance_ratio_te(c + d, c, c, c)
    r_auto = orc.cosmic_variance_ratio(c + d, c)
    assert np.allclose(r_te, r_auto, rtol=1e-12, atol=0)


def test_cosmic_variance_te_monte_carlo(orc):
    """sigma_CV^TE is the standard deviation of the full-sky estimator
    (1/(2l+1)) sum_m a^T_lm a^E_lm of jointly Gaussian (T, E) with covariance
    [[TT, TE], [TE, EE]]: drawn here as real pairs, 2l+1 per estimate."""
    rng = np.random.default_rng(6)
    tt, ee, te = 2.0, 0.5, 0.6
    L = np.linalg.cholesky(np.array([[tt, te], [te, ee]]))
    for l in (2, 7):
        n = 2 * l + 1
        z = rng.normal(size=(200000, n, 2)) @ L.T
        est = (z[..., 0] * z[..., 1]).mean(axis=1)
        sig_mc = est.std()
        # a unit deviation of C^TE measured in sigma_CV^TE units
        ratio = orc.cosmic_variance_ratio_te(np.array([te + 1.0]), np.array([tt]), np.array([ee]), np.array([te]),
                                             lmin=l)[0]
        assert 1.0 / ratio == pytest.approx(sig_mc, rel=0.01)
