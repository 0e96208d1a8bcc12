"""Pins for the oracle's tensor-mode projection: kernels
t_l = sqrt((l+2)!/(l-2)!) j_l/x^2, e_l = -j_l + j_l'' + 2 j_l/x^2 + 4 j_l'/x,
b_l = 2 j_l' + 4 j_l/x (the oracle evaluates e_l, b_l through the Bessel
equation and j_{l-1}; these pins use the derivative forms).

A slip in the rewrite (a sign, the l(l-1) factor, the j_{l-1} index) fails
the mpmath check; the x -> 0 limits catch the x = 0 node; the delta source
catches the quadrature; the scale-invariant closed forms (Weber-Schafheitlin
integrals of J_mu J_nu t^-lam) catch the whole chain of the TT, EE, BB and TE
spectra."""
import math

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")


def _jl(l, x):
    return mp.sqrt(mp.pi / (2 * x)) * mp.besselj(l + mp.mpf(1) / 2, x)


def test_tensor_kernels_mpmath(orc):
    mp.mp.dps = 30
    rng = np.random.default_rng(31)
    for _ in range(30):
        l = int(rng.integers(2, 300))
        x = float(rng.uniform(0.05, 1200.0))
        xm = mp.mpf(x)
        j = _jl(l, xm)
        jp = mp.diff(lambda s: _jl(l, s), xm)
        jpp = mp.diff(lambda s: _jl(l, s), xm, 2)
        e_ref = -j + jpp + 2 * j / xm ** 2 + 4 * jp / xm
        b_ref = 2 * jp + 4 * j / xm
        t, e, b = orc.tensor_kernels(np.array([x]), l)
        scale = max(abs(float(e_ref)), abs(float(b_ref)), 1e-3 / max(1.0, x))
        assert abs(e[0, l] - float(e_ref)) <= 1e-10 * scale, (l, x)
        assert abs(b[0, l] - float(b_ref)) <= 1e-10 * scale, (l, x)
        c = math.sqrt((l + 2.0) * (l + 1.0) * l * (l - 1.0))
        assert t[0, l] == pytest.approx(c * float(j) / x ** 2, rel=1e-10, abs=1e-300)


def test_tensor_kernels_at_and_near_zero(orc):
    t, e, b = orc.tensor_kernels(np.array([0.0, 1e-4]), 6)
    assert e[0, 2] == 0.8 and np.all(e[0, 3:] == 0) and np.all(b[0] == 0)
    assert t[0, 2] == pytest.approx(math.sqrt(24.0) / 15.0, rel=1e-15)
    # leading terms: e_2 = 4/5 - 22 x^2/105, e_3 = 4x/21, b_2 = 8x/15, b_3 = 2x^2/21
    x = 1e-4
    assert e[1, 2] == pytest.approx(0.8 - 22 * x * x / 105, rel=1e-12)
    assert e[1, 3] == pytest.approx(4 * x / 21, rel=1e-7)
    assert b[1, 2] == pytest.approx(8 * x / 15, rel=1e-7)
    assert b[1, 3] == pytest.approx(2 * x * x / 21, rel=1e-7)
    assert np.all(t[:, :2] == 0) and np.all(e[:, :2] == 0) and np.all(b[:, :2] == 0)


def test_delta_source_gives_the_kernels(orc):
    tau0 = 14000.0
    tau = np.linspace(200.0, 14000.0, 50)
    k = np.geomspace(1e-4, 0.3, 20)
    w = orc.trapz_weights(tau)
    i = 31
    S = np.zeros((k.size, tau.size))
    S[:, i] = 1.0 / w[i]
    dt, de, db = orc.los_tensor(k, tau, tau0, 2, 200, S, 2.0 * S)
    t, e, b = orc.tensor_kernels(k * (tau0 - tau[i]), 200)
    for d, ref in ((dt, t[:, 2:]), (de, 2.0 * e[:, 2:]), (db, 2.0 * b[:, 2:])):
        assert np.abs(d - ref).max() <= 1e-14 * np.abs(ref).max()


def _W(mu, nu, lam):
    """int_0^inf J_mu(t) J_nu(t) t^-lam dt (Weber-Schafheitlin)."""
    return mp.gamma(lam) * mp.gamma((mu + nu - lam + 1) / 2) * mp.rgamma((-mu + nu + lam + 1) / 2) * \
        mp.rgamma((mu + nu + lam + 1) / 2) * mp.rgamma((mu - nu + lam + 1) / 2) / mp.mpf(2) ** lam


def _closed_forms(l):
    """4 pi int K_l(x) K'_l(x) dx/x for the scale-invariant delta source, from
    j_a j_b = (pi / 2x) J_(a+1/2) J_(b+1/2); per unit amplitude A."""
    mp.mp.dps = 30
    n, m = mp.mpf(l) + mp.mpf(1) / 2, mp.mpf(l) - mp.mpf(1) / 2
    c2 = mp.mpf(l + 2) * (l + 1) * l * (l - 1)
    L1 = mp.mpf(l) * (l - 1)
    half_pi = mp.pi / 2
    bb = half_pi * (4 * _W(m, m, 2) - 8 * (l - 1) * _W(m, n, 3) + 4 * (l - 1) ** 2 * _W(n, n, 4))
    out = {"BB": 4 * mp.pi * bb}
    if l >= 3:
        tt = c2 * half_pi * _W(n, n, 6)
        ee = half_pi * (L1 ** 2 * _W(n, n, 6) - 4 * L1 * _W(n, n, 4) + 4 * _W(n, n, 2) + 4 * L1 * _W(n, m, 5)
                        - 8 * _W(n, m, 3) + 4 * _W(m, m, 4))
        te = mp.sqrt(c2) * half_pi * (L1 * _W(n, n, 6) - 2 * _W(n, n, 4) + 2 * _W(n, m, 5))
        out.update(TT=4 * mp.pi * tt, EE=4 * mp.pi * ee, TE=4 * mp.pi * te)
    return {key: float(v) for key, v in out.items()}


def test_scale_invariant_tensor_closed_forms(orc):
    tau0 = 14000.0
    tau = np.array([13000.0, 13500.0, 13900.0])
    istar = 1
    rstar = tau0 - tau[istar]
    w = orc.trapz_weights(tau)
    xs_log = np.exp(np.arange(math.log(1e-3), math.log(10.0), 0.004))
    xs_lin = np.arange(10.0, 2e4 + 1e-9, 0.05)
    k = np.concatenate([xs_log, xs_lin[1:]]) / rstar
    S = np.zeros((k.size, tau.size))
    S[:, istar] = 1.0 / w[istar]
    P = np.ones(k.size)
    dt, de, db = orc.los_tensor(k, tau, tau0, 2, 30, S, S)
    spectra = {"TT": orc.cl_cross(k, dt, dt, P), "EE": orc.cl_cross(k, de, de, P),
               "BB": orc.cl_cross(k, db, db, P), "TE": orc.cl_cross(k, dt, de, P)}
    for l in (2, 3, 5, 12, 30):
        ref = _closed_forms(l)
        for key, val in ref.items():
            assert spectra[key][l - 2] == pytest.approx(val, rel=2e-4), (key, l, spectra[key][l - 2], val)
