"""Pins for the oracle's spherical Bessel functions j_l(x) (the flat-space
kernel phi_l of Eq. 2).  Each check is tied to mathematics, not to the oracle:
closed forms, power series, the addition sum rule, 50-digit mpmath values,
Watson's inequality, and the x = 0 limit."""
import math

import numpy as np
import pytest

from tests.conftest import jl_mpmath


def _series(l, x):
    """j_l(x) = x^l/(2l+1)!! sum_n (-x^2/2)^n / (n! (2l+3)(2l+5)...(2l+2n+1)), to convergence."""
    df = 1.0
    for q in range(1, 2 * l + 2, 2):
        df *= q
    term, total, n = 1.0, 1.0, 0
    while abs(term) > 1e-19 * abs(total):
        n += 1
        term *= -(x * x / 2) / (n * (2 * l + 2 * n + 1))
        total += term
    return x ** l / df * total


def _j012(x):
    if x < 1.0:
        return tuple(_series(l, x) for l in range(3))
    s, c = math.sin(x), math.cos(x)
    j0 = s / x
    j1 = s / x ** 2 - c / x
    j2 = (3 / x ** 2 - 1) * s / x - 3 * c / x ** 2
    return j0, j1, j2


def test_closed_forms_j0_j1_j2(orc):
    xs = np.concatenate([10 ** np.linspace(-3, 4, 400), [0.5, 1.0, 1.5, 2.0, 3.0, math.pi, 2 * math.pi]])
    for x in xs:
        j = orc.sph_bessel(5, float(x))
        ref = _j012(float(x))
        # closed forms lose relative accuracy near their zeros and through
        # cancellation at small x: compare against the local envelope
        for l in range(3):
            # relative below x = 1; above, the closed forms are compared on the
            # scale of their 1/x envelope (they cross zero there)
            tol = 2e-15 * abs(ref[l]) if x < 1 else 4e-15 * (1.0 / x + abs(ref[l]))
            assert abs(j[l] - ref[l]) <= tol, (l, x, j[l], ref[l])


def test_tiny_arguments(orc):
    """Below x = 1e-3 the leading series terms; compared with 30-digit mpmath."""
    pytest.importorskip("mpmath")
    for x in (1e-200, 1e-40, 1e-7, 9.9e-4):
        j = orc.sph_bessel(12, x)
        for l in (0, 1, 2, 5, 12):
            ref = jl_mpmath(l, x)
            if abs(ref) < 1e-300:
                assert abs(j[l]) < 1e-300
            else:
                assert abs(j[l] - ref) <= 1e-15 * abs(ref), (l, x, j[l], ref)


def test_x_zero(orc):
    j = orc.sph_bessel(7, 0.0)
    assert j[0] == 1.0 and np.all(j[1:] == 0.0)


@pytest.mark.parametrize("x", [1e-3, 0.3, 0.99, 1.0, 2.5, 17.3, 99.5, 500.0, 2499.7, 6000.0, 13800.0])
def test_sum_rule(orc, x):
    """sum_{l>=0} (2l+1) j_l(x)^2 = 1 (addition theorem at zero separation)."""
    L = int(x + 40 + 4 * x ** (1 / 3) + math.sqrt(40 * x))
    j = orc.sph_bessel(L, x)
    l = np.arange(L + 1)
    s = math.fsum((2 * l + 1) * j * j)
    assert abs(s - 1.0) <= 1e-13 * max(1.0, math.sqrt(x) / 10), s


def test_three_term_recurrence(orc):
    rng = np.random.default_rng(3)
    for _ in range(40):
        x = float(10 ** rng.uniform(-2, 4))
        L = int(rng.integers(10, 3000))
        j = orc.sph_bessel(L, x)
        l = np.arange(1, L)
        lhs = j[l - 1] + j[l + 1]
        rhs = (2 * l + 1) / x * j[l]
        scale = np.maximum(np.abs(lhs), np.abs(rhs)) + np.abs(j[l + 1]) + np.abs(j[l - 1])
        assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale + 1e-300)


def test_mpmath_spot_checks(orc):
    """50-digit Bessel J of half-integer order at seeded random (l, x), plus
    points on the turning line l ~ x where forward and backward parts meet."""
    pytest.importorskip("mpmath")
    rng = np.random.default_rng(7)
    cases = []
    for _ in range(40):
        lmax = int(rng.integers(2, 6000))
        x = float(10 ** rng.uniform(-3, math.log10(14000)))
        for l in rng.integers(0, lmax + 1, 2):
            cases.append((lmax, int(l), x))
        cases.append((lmax, min(lmax, int(x)), x))
        cases.append((lmax, min(lmax, int(x) + 1), x))
    for lmax, l, x in cases:
        j = orc.sph_bessel(lmax, x)[l]
        ref = jl_mpmath(l, x)
        if abs(ref) < 1e-280:
            continue
        env = abs(ref) if x < l + 0.5 else max(abs(ref), 1.0 / x)
        assert abs(j - ref) <= 1e-12 * env, (l, x, j, ref)


def test_watson_bound(orc):
    """A&S 9.1.63: |J_nu(nu z)| <= [z exp(sqrt(1-z^2)) / (1+sqrt(1-z^2))]^nu for 0<z<=1,
    so |j_l(x)| <= sqrt(pi/(2x)) exp(-nu (alpha - tanh alpha)), nu = l+1/2, x = nu sech(alpha)."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        l = int(rng.integers(2, 6000))
        nu = l + 0.5
        z = float(rng.uniform(0.05, 0.999))
        x = nu * z
        j = orc.sph_bessel(l, x)[l]
        s = math.sqrt(1 - z * z)
        logb = 0.5 * math.log(math.pi / (2 * x)) + nu * (math.log(z) + s - math.log1p(s))
        if logb < -700:
            assert abs(j) < 1e-300
        else:
            assert abs(j) <= math.exp(logb) * (1 + 1e-12)
