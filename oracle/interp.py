"""FP64 oracle of the source interpolation onto the transfer k grid (the
`InterpolateSources` step that precedes the projection, Sec. 3.3).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baselines).

Reading: the paper names the step but not the interpolant; this oracle takes
the natural cubic spline in k of every (source, tau) column: on nodes
k_0 < ... < k_(n-1) with h_j = k_(j+1) - k_j, the second derivatives M_j
solve
    h_(j-1) M_(j-1) + 2 (h_(j-1) + h_j) M_j + h_j M_(j+1)
        = 6 [(y_(j+1) - y_j) / h_j - (y_j - y_(j-1)) / h_(j-1)],  0 < j < n-1,
with M_0 = M_(n-1) = 0, and on [k_j, k_(j+1)], with t = (k - k_j) / h_j,
    y(k) = (1-t) y_j + t y_(j+1)
           + h_j^2 / 6 [((1-t)^3 - (1-t)) M_j + (t^3 - t) M_(j+1)].
The banded linear solve is a library step (scipy.linalg.solve_banded).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded


def natural_second_derivatives(x, y) -> np.ndarray:
    """M[..., n] of the natural cubic spline through (x, y[..., n]) (y's last
    axis runs over the nodes)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.size
    M = np.zeros_like(y)
    if n < 3:
        return M
    h = np.diff(x)
    ab = np.zeros((3, n - 2))
    ab[0, 1:] = h[1:-1]                    # super-diagonal
    ab[1, :] = 2.0 * (h[:-1] + h[1:])      # diagonal
    ab[2, :-1] = h[1:-1]                   # sub-diagonal
    slope = np.diff(y, axis=-1) / h
    rhs = 6.0 * (slope[..., 1:] - slope[..., :-1])
    flat = rhs.reshape(-1, n - 2).T
    M[..., 1:-1] = solve_banded((1, 1), ab, flat).T.reshape(rhs.shape)
    return M


def natural_spline_eval(x, y, M, xq) -> np.ndarray:
    """Values at xq (inside [x_0, x_(n-1)]) of the spline with second
    derivatives M; y, M [..., n] -> [..., xq.size]."""
    x = np.asarray(x, dtype=np.float64)
    xq = np.asarray(xq, dtype=np.float64)
    n = x.size
    j = np.clip(np.searchsorted(x, xq, side="right") - 1, 0, n - 2)
    h = x[j + 1] - x[j]
    t = (xq - x[j]) / h
    y0, y1 = y[..., j], y[..., j + 1]
    m0, m1 = M[..., j], M[..., j + 1]
    return (1 - t) * y0 + t * y1 + h * h / 6.0 * (((1 - t) ** 3 - (1 - t)) * m0 + (t ** 3 - t) * m1)


def interp_sources(k_in, S_in, k_out) -> np.ndarray:
    """S_in [M][nk_in][ntau] on k_in -> [M][nk_out][ntau] on k_out (natural
    cubic spline in k of every (source, tau) column)."""
    S = np.asarray(S_in, dtype=np.float64)
    cols = np.moveaxis(S, 1, -1)  # [M][ntau][nk_in]
    M = natural_second_derivatives(k_in, cols)
    out = natural_spline_eval(k_in, cols, M, k_out)
    return np.ascontiguousarray(np.moveaxis(out, -1, 1))
