"""FP64 reference of the C_l emulator network (test infrastructure only).

An MLP  x[9] -> 512 -> 512 -> 512 -> y[2499]  with GELU between layers,
trained on the mean squared error of standardised log C_l with Adam.  The
paper builds no emulator; it motivates fast spectra for emulator training sets
(Sec. 1, Sec. 5).  This module is the plain definition the device kernels are
checked against:

  z_l = h_{l-1} W_l^T + b_l,  h_l = GELU(z_l) (hidden layers), out = z_L
  GELU(z) = z Phi(z),  Phi = standard normal CDF  (exact form, with erf)
  loss = mean((out - y)^2)

With rounding=True every matrix-product operand is first rounded to bfloat16
(fp32 first, as the device holds fp32 values): this is where the device's
arithmetic rounds (its tensor-core products take bf16 operands, everything
else is fp32), so the two can be compared at fp32-accumulation accuracy.
"""
from __future__ import annotations

import math

import numpy as np

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def _erf(x):
    try:
        from scipy.special import erf
        return erf(x)
    except Exception:  # pragma: no cover - scipy is present where tests run
        return np.vectorize(math.erf)(x)


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via float32; as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    finite = np.isfinite(a)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    r = np.where(finite, r, u & 0xFFFF0000)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + _erf(z / SQRT2))


def gelu_grad(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * (1.0 + _erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def forward(Ws, bs, x, rounding=True):
    """Returns (out, cache); cache holds the layer inputs h and pre-activations z."""
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    h = np.asarray(x, dtype=np.float64)
    hs, zs = [h], []
    L = len(Ws)
    for l in range(L):
        z = r(h) @ r(Ws[l]).T + bs[l]
        zs.append(z)
        if l < L - 1:
            h = gelu(z)
            hs.append(h)
    return zs[-1], {"h": hs, "z": zs}


def backward(Ws, bs, cache, y, rounding=True):
    """Loss and its gradients (dW_l, db_l) for the mean squared error."""
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    out = cache["z"][-1]
    y = np.asarray(y, dtype=np.float64)
    B, N = y.shape
    diff = out - y
    loss = float(np.mean(diff * diff))
    d = 2.0 * diff / (B * N)
    L = len(Ws)
    dW = [None] * L
    db = [None] * L
    for l in range(L - 1, -1, -1):
        dW[l] = r(d).T @ r(cache["h"][l])
        db[l] = d.sum(axis=0)
        if l > 0:
            dh = r(d) @ r(Ws[l])
            d = dh * gelu_grad(cache["z"][l - 1])
    return loss, dW, db


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; t counts from 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(sizes, seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for a, b in zip(sizes[:-1], sizes[1:]):
        bound = 1.0 / math.sqrt(a)
        Ws.append(rng.uniform(-bound, bound, size=(b, a)))
        bs.append(rng.uniform(-bound, bound, size=b))
    return Ws, bs
