"""Pins for the oracle's hyperspherical Bessel functions Phi^beta_l(chi) and
curved-space projection (open K < 0 and closed K > 0 space).

The oracle runs the recurrence downwards (Miller) and normalises to the
closed forms of Phi_0, Phi_1; these pins use other routes: the forward
recurrence at 60 digits (mpmath) from the closed forms, the addition theorem
sum_l (2l+1) Phi_l^2 = 1, the flat limit Phi -> j_l(q r) as K -> 0, and, in
closed space, Phi_l = 0 for l >= beta.  A wrong coefficient of the
recurrence, sign or normalisation fails the first two; a wrong argument
(beta, chi) the third."""
import numpy as np
import pytest


def _forward_mp(beta, chi, lmax, closed):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    b, c = mp.mpf(beta), mp.mpf(chi)
    sh = mp.sin(c) if closed else mp.sinh(c)
    ct = mp.cot(c) if closed else mp.coth(c)
    s = (lambda l: mp.sqrt(b * b - l * l)) if closed else (lambda l: mp.sqrt(b * b + l * l))
    out = [mp.sin(b * c) / (b * sh)]
    out.append((mp.sin(b * c) * ct - b * mp.cos(b * c)) / (b * sh * s(1)))
    for l in range(1, lmax):
        if closed and l + 1 >= beta:
            out.append(mp.mpf(0))
            continue
        out.append(((2 * l + 1) * ct * out[l] - s(l) * out[l - 1]) / s(l + 1))
    return np.array([float(v) for v in out[:lmax + 1]])


@pytest.mark.parametrize("beta,chi,closed", [(5.0, 0.5, False), (40.0, 0.9, False), (300.0, 0.05, False),
                                             (12.0, 2.0, False), (60.0, 1.1, True), (25.0, 2.9, True),
                                             (200.0, 0.15, True)])
def test_against_60_digit_forward_recurrence(orc, beta, chi, closed):
    lmax = 40
    ref = _forward_mp(beta, chi, lmax, closed)
    got = orc.hyper_bessel(beta, chi, lmax, closed)[0]
    scale = np.abs(ref).max()
    big = np.abs(ref) > 1e-30 * scale
    assert np.all(np.abs(got - ref)[big] <= 1e-11 * np.maximum(np.abs(ref[big]), 1e-6 * scale))


@pytest.mark.parametrize("beta,chi,closed", [(30.0, 1.2, False), (500.0, 0.3, False), (3.5, 4.0, False),
                                             (80.0, 1.1, True), (400.0, 2.5, True), (7.0, 0.4, True)])
def test_addition_theorem_sum_rule(orc, beta, chi, closed):
    # open space: past the turning order the terms fall by tanh(chi/2) per order
    L = int(beta) - 1 if closed else int(beta * np.sinh(chi) + 200 + 60.0 / -np.log(np.tanh(0.5 * chi)))
    p = orc.hyper_bessel(beta, chi, L, closed)[0]
    l = np.arange(L + 1)
    assert ((2 * l + 1) * p * p).sum() == pytest.approx(1.0, abs=1e-12)


def test_flat_limit(orc):
    R = 1e9  # curvature radius [Mpc]: corrections O((r/R)^2) ~ 1e-10
    for q, r in ((0.003, 13000.0), (0.05, 9000.0), (0.2, 2000.0)):
        ref = orc.sph_bessel(300, q * r)
        for closed in (False, True):
            beta = q * R if not closed else float(np.round(q * R))
            got = orc.hyper_bessel(beta, r / R, 300, closed)[0]
            assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), (q, r, closed)


def test_closed_space_vanishes_beyond_beta_and_at_chi0(orc):
    p = orc.hyper_bessel(17.0, 0.8, 40, True)[0]
    assert np.all(p[17:] == 0.0) and np.any(p[:17] != 0.0)
    p0 = orc.hyper_bessel(50.0, 0.0, 10, False)[0]
    assert p0[0] == 1.0 and np.all(p0[1:] == 0.0)


def test_delta_source_gives_phi(orc):
    K = -1e-8
    tau0 = 14000.0
    tau = np.linspace(200.0, 14000.0, 40)
    q = np.geomspace(1e-3, 0.2, 15)
    w = orc.trapz_weights(tau)
    i = 21
    S = np.zeros((q.size, tau.size))
    S[:, i] = 1.0 / w[i]
    d = orc.los_curved(q, tau, tau0, K, 2, 200, S)
    rk = np.sqrt(-K)
    ref = orc.hyper_bessel(q / rk, rk * (tau0 - tau[i]), 200, False)[:, 2:]
    assert np.abs(d - ref).max() <= 1e-14 * np.abs(ref).max()
