"""Pins for the emulator network's FP64 reference (oracle/mlp.py): GELU's
values and derivative, the backward pass against central finite differences
of the loss, bfloat16 rounding rules, and Adam's first step."""
import math

import numpy as np

from oracle import mlp


def test_gelu_values():
    # GELU(z) = z Phi(z); Phi(1) = 0.8413447460685429, Phi(-1) = 1 - Phi(1)
    assert mlp.gelu(0.0) == 0.0
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(-1.0) + 0.15865525393145707) < 1e-15
    assert abs(mlp.gelu(3.0) - 3.0 * 0.9986501019683699) < 1e-14


def test_gelu_grad_finite_differences():
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(z)).max() < 1e-9


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [9, 6, 5, 7, 11]
    Ws, bs = mlp.init_params(sizes, seed=3)
    x = rng.normal(size=(4, 9))
    y = rng.normal(size=(4, 11))

    def loss(Ws_, bs_):
        out, _ = mlp.forward(Ws_, bs_, x, rounding=False)
        return float(np.mean((out - y) ** 2))
    out, cache = mlp.forward(Ws, bs, x, rounding=False)
    L0, dW, db = mlp.backward(Ws, bs, cache, y, rounding=False)
    assert abs(L0 - loss(Ws, bs)) < 1e-15
    h = 1e-6
    for l in range(len(Ws)):
        for (i, j) in [(0, 0), (Ws[l].shape[0] - 1, Ws[l].shape[1] - 1), (1, 2)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (loss(Wp, bs) - loss(Wm, bs)) / (2 * h)
            assert abs(fd - dW[l][i, j]) <= 1e-7 * max(1.0, abs(fd)), (l, i, j)
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][0] += h
        bm[l][0] -= h
        fd = (loss(Ws, bp) - loss(Ws, bm)) / (2 * h)
        assert abs(fd - db[l][0]) <= 1e-7 * max(1.0, abs(fd))


def test_bf16_rounding_rules():
    e = 2.0 ** -8  # bf16 spacing just above 1 is 2^-7; half of it is 2^-8
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + e) == 1.0                    # tie -> even (1.0)
    assert mlp.bf16(1.0 + 3 * e) == 1.0 + 4 * e        # tie -> even (1 + 2^-6)
    assert mlp.bf16(1.0 + 1.5 * e) == 1.0 + 2 * e      # above the tie -> up
    assert mlp.bf16(-3.0) == -3.0
    x = np.random.default_rng(1).normal(size=1000)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 * 1.0000001)
    assert np.array_equal(mlp.bf16(r), r)


def test_adam_first_step():
    p, g = np.array([1.0, -2.0]), np.array([0.5, -3.0])
    p1, m, v = mlp.adam_step(p, g, np.zeros(2), np.zeros(2), 1, lr=0.01)
    # bias-corrected moments are g and g^2 on the first step
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
