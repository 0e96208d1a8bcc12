"""Pins for the oracle's source interpolation (natural cubic spline in k,
oracle/interp.py): it passes through the nodes, is exact on linear data, its
end second derivatives vanish, it agrees with an independent implementation
(scipy's CubicSpline with natural ends), and its error on a smooth function
falls as h^4 (a dropped term or a wrong coefficient breaks the order)."""
import numpy as np
import pytest

from oracle import interp


def test_nodes_linear_and_ends():
    rng = np.random.default_rng(1)
    x = np.sort(rng.uniform(0.0, 3.0, 40))
    y = rng.normal(size=(3, 40))
    M = interp.natural_second_derivatives(x, y)
    assert np.allclose(interp.natural_spline_eval(x, y, M, x), y, rtol=0, atol=1e-13)
    assert np.all(M[:, 0] == 0) and np.all(M[:, -1] == 0)
    lin = 2.0 * x - 0.7
    xq = np.linspace(x[0], x[-1], 999)
    Ml = interp.natural_second_derivatives(x, lin)
    assert np.allclose(interp.natural_spline_eval(x, lin, Ml, xq), 2.0 * xq - 0.7, rtol=0, atol=1e-13)


def test_against_scipy_natural_spline():
    CubicSpline = pytest.importorskip("scipy.interpolate").CubicSpline
    rng = np.random.default_rng(2)
    x = np.sort(rng.uniform(-1.0, 2.0, 25))
    y = rng.normal(size=(4, 25))
    xq = np.linspace(x[0], x[-1], 777)
    ref = CubicSpline(x, y, axis=1, bc_type="natural")(xq)
    got = interp.natural_spline_eval(x, y, interp.natural_second_derivatives(x, y), xq)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fourth_order_convergence():
    f = lambda x: np.sin(3.0 * x) * np.exp(-0.2 * x)
    errs = []
    for n in (41, 81, 161):
        x = np.linspace(0.0, 4.0, n)
        xq = np.linspace(1.0, 3.0, 1001)  # interior: away from the natural ends
        y = f(x)
        errs.append(np.abs(interp.natural_spline_eval(x, y, interp.natural_second_derivatives(x, y), xq) - f(xq)).max())
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(12.0 < r < 20.0 for r in ratios), ratios


def test_interp_sources_layout():
    rng = np.random.default_rng(3)
    k_in = np.geomspace(1e-4, 0.3, 30)
    S = rng.normal(size=(2, 30, 7))
    k_out = np.geomspace(1e-4, 0.3, 95)
    out = interp.interp_sources(k_in, S, k_out)
    assert out.shape == (2, 95, 7)
    for m in range(2):
        for i in range(7):
            y = S[m, :, i]
            ref = interp.natural_spline_eval(k_in, y, interp.natural_second_derivatives(k_in, y), k_out)
            assert np.allclose(out[m, :, i], ref, rtol=0, atol=1e-13)
