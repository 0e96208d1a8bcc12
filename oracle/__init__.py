"""FP64 CPU oracle for the line-of-sight projection (arXiv 2509.25110, Eqs. 1-3).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the product path.  It shares
no code with the CUDA library; both sides are fed by the seeded input module
`paper_2509_25110_gb300.synth`, which holds none of the method's arithmetic.

The C part (`gcamb_oracle.c`) is compiled with gcc into `liboracle.so` by
`oracle.build.build()`.  The emulator's reference network (`oracle.mlp`) is
plain numpy in float64.

Pins (tests/test_oracle_*.py): closed forms of j_0, j_1, j_2; the addition
sum rule; 50-digit mpmath values; the trapezoid's exactness on linear
integrands and its error bound; a delta-function source; linearity; the
Sachs-Wolfe plateau C_l = 2 pi A / (l (l+1)); brute force on tiny grids.
E-mode and cross spectra: eps_2 in closed form, mpmath eps_l, its x -> 0
limit, a delta source, the scale-invariant C^EE and C^TE closed forms,
Cauchy-Schwarz; the cross-spectrum cosmic variance against its auto form
and a Monte Carlo of the full-sky estimator.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

_dp = ctypes.POINTER(ctypes.c_double)


def lib_path() -> str:
    return os.path.join(_HERE, "liboracle.so")


def _load():
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        from . import build as _b
        _b.build()
    lib = ctypes.CDLL(path)
    lib.orc_trapz_weights.argtypes = [ctypes.c_int, _dp, _dp]
    lib.orc_lnk_weights.argtypes = [ctypes.c_int, _dp, _dp]
    lib.orc_sph_bessel.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
    lib.orc_sph_bessel_many.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp]
    lib.orc_los_cl.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_double,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                               _dp, _dp, _dp, _dp, ctypes.c_int]
    lib.orc_los_cl.restype = ctypes.c_int
    lib.orc_cl.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
    lib.orc_cl.restype = ctypes.c_int
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_eps_many.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp]
    lib.orc_los_e.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, _dp, _dp, _dp, ctypes.c_int]
    lib.orc_los_e.restype = ctypes.c_int
    lib.orc_cl_cross.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
    lib.orc_cl_cross.restype = ctypes.c_int
    lib.orc_hyper_bessel_many.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp]
    lib.orc_los_curved.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int]
    lib.orc_los_curved.restype = ctypes.c_int
    lib.orc_tensor_kernels_many.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp]
    lib.orc_los_tensor.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
    lib.orc_los_tensor.restype = ctypes.c_int
    _LIB = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def trapz_weights(x) -> np.ndarray:
    """Trapezoid weights on increasing nodes."""
    x = _f64(x)
    w = np.empty_like(x)
    _load().orc_trapz_weights(x.size, _ptr(x), _ptr(w))
    return w


def lnk_weights(k) -> np.ndarray:
    """Trapezoid weights in ln k (the dk/k measure of Eq. 1)."""
    k = _f64(k)
    w = np.empty_like(k)
    _load().orc_lnk_weights(k.size, _ptr(k), _ptr(w))
    return w


def sph_bessel(lmax: int, x) -> np.ndarray:
    """j_l(x) for l = 0..lmax; x scalar -> [lmax+1], x array -> [n, lmax+1]."""
    lib = _load()
    if np.ndim(x) == 0:
        out = np.empty(lmax + 1)
        lib.orc_sph_bessel(int(lmax), float(x), _ptr(out))
        return out
    xa = _f64(x).ravel()
    out = np.empty((xa.size, lmax + 1))
    lib.orc_sph_bessel_many(xa.size, _ptr(xa), int(lmax), _ptr(out))
    return out


def los_cl(k, tau, tau0, lmin, lmax, S, Pk=None, want_delta=True, want_cl=True,
           wtau=None, wk=None, nthreads=0):
    """Dense FP64 Delta[M][nk][nl] and C_l[M][nl] (Eqs. 1-2 discretised).

    S has shape [M][nk][ntau] (or [nk][ntau] for one model)."""
    k = _f64(k)
    tau = _f64(tau)
    S = _f64(S)
    single = S.ndim == 2
    if single:
        S = S[None]
    M, nk, ntau = S.shape
    assert nk == k.size and ntau == tau.size
    nl = lmax - lmin + 1
    delta = np.empty((M, nk, nl)) if want_delta else None
    cl = None
    if want_cl:
        assert Pk is not None
        Pk = _f64(Pk).reshape(M, nk)
        cl = np.empty((M, nl))
    rc = _load().orc_los_cl(nk, _ptr(k), ntau, _ptr(tau), float(tau0), int(lmin), int(lmax), M,
                            _ptr(S), _ptr(Pk) if want_cl else None,
                            _ptr(_f64(wtau)) if wtau is not None else None,
                            _ptr(_f64(wk)) if wk is not None else None,
                            _ptr(delta), _ptr(cl), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    if single:
        delta = None if delta is None else delta[0]
        cl = None if cl is None else cl[0]
    return delta, cl


def cl_from_delta(k, delta, Pk, wk=None) -> np.ndarray:
    """C_l[M][nl] from Delta[M][nk][nl] and P[M][nk] (Eq. 1)."""
    k = _f64(k)
    delta = _f64(delta)
    single = delta.ndim == 2
    if single:
        delta = delta[None]
    M, nk, nl = delta.shape
    Pk = _f64(Pk).reshape(M, nk)
    cl = np.empty((M, nl))
    _load().orc_cl(nk, _ptr(k), nl, M, _ptr(delta), _ptr(Pk),
                   _ptr(_f64(wk)) if wk is not None else None, _ptr(cl))
    return cl[0] if single else cl


def eps(x, lmax) -> np.ndarray:
    """eps_l(x) = sqrt((l+2)!/(l-2)!) j_l(x)/x^2 (0 for l < 2; limit at x = 0)
    for l = 0..lmax, shape [x.size][lmax + 1] (the kernel of Eq. 3)."""
    xa = _f64(x).ravel()
    out = np.empty((xa.size, lmax + 1))
    _load().orc_eps_many(xa.size, _ptr(xa), int(lmax), _ptr(out))
    return out


def los_e(k, tau, tau0, lmin, lmax, SP, wtau=None, nthreads=0) -> np.ndarray:
    """Dense FP64 Delta^E[M][nk][nl] of Eq. (3), S_P of shape [M][nk][ntau]."""
    k = _f64(k)
    tau = _f64(tau)
    SP = _f64(SP)
    single = SP.ndim == 2
    if single:
        SP = SP[None]
    M, nk, ntau = SP.shape
    assert nk == k.size and ntau == tau.size
    d = np.empty((M, nk, lmax - lmin + 1))
    rc = _load().orc_los_e(nk, _ptr(k), ntau, _ptr(tau), float(tau0), int(lmin), int(lmax), M, _ptr(SP),
                           _ptr(_f64(wtau)) if wtau is not None else None, _ptr(d), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return d[0] if single else d


def hyper_bessel(beta, chi, lmax, closed) -> np.ndarray:
    """Phi^beta_l(chi), l = 0..lmax, for arrays beta, chi of one shape n ->
    [n][lmax + 1]; closed = True for K > 0 (integer beta)."""
    b = _f64(np.broadcast_to(beta, np.broadcast(beta, chi).shape)).ravel()
    c = _f64(np.broadcast_to(chi, b.shape)).ravel()
    out = np.empty((b.size, lmax + 1))
    _load().orc_hyper_bessel_many(b.size, _ptr(b), _ptr(c), int(lmax), int(bool(closed)), _ptr(out))
    return out


def los_curved(q, tau, tau0, K, lmin, lmax, S, wtau=None, nthreads=0) -> np.ndarray:
    """Dense FP64 curved-space transfer functions [M][nq][nl] (Eq. 2 with
    phi_l the hyperspherical Bessel function of curvature K != 0)."""
    q = _f64(q)
    tau = _f64(tau)
    S = _f64(S)
    single = S.ndim == 2
    if single:
        S = S[None]
    M, nq, ntau = S.shape
    d = np.empty((M, nq, lmax - lmin + 1))
    rc = _load().orc_los_curved(nq, _ptr(q), ntau, _ptr(tau), float(tau0), float(K), int(lmin), int(lmax), M,
                                _ptr(S), _ptr(_f64(wtau)) if wtau is not None else None, _ptr(d), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return d[0] if single else d


def tensor_kernels(x, lmax):
    """Tensor-mode kernels (t_l, e_l, b_l)(x) for l = 0..lmax, each of shape
    [x.size][lmax + 1] (zero below l = 2; limits at x = 0)."""
    xa = _f64(x).ravel()
    t, e, b = (np.empty((xa.size, lmax + 1)) for _ in range(3))
    _load().orc_tensor_kernels_many(xa.size, _ptr(xa), int(lmax), _ptr(t), _ptr(e), _ptr(b))
    return t, e, b


def los_tensor(k, tau, tau0, lmin, lmax, ST, SP, wtau=None, nthreads=0):
    """Dense FP64 tensor transfer functions (DT, DE, DB), each [M][nk][nl],
    from tensor sources ST, SP of shape [M][nk][ntau]."""
    k = _f64(k)
    tau = _f64(tau)
    ST, SP = _f64(ST), _f64(SP)
    single = ST.ndim == 2
    if single:
        ST, SP = ST[None], SP[None]
    M, nk, ntau = ST.shape
    assert SP.shape == ST.shape and nk == k.size and ntau == tau.size
    out = [np.empty((M, nk, lmax - lmin + 1)) for _ in range(3)]
    rc = _load().orc_los_tensor(nk, _ptr(k), ntau, _ptr(tau), float(tau0), int(lmin), int(lmax), M, _ptr(ST),
                                _ptr(SP), _ptr(_f64(wtau)) if wtau is not None else None, _ptr(out[0]),
                                _ptr(out[1]), _ptr(out[2]), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return tuple(o[0] for o in out) if single else tuple(out)


def cl_cross(k, DX, DY, Pk, wk=None) -> np.ndarray:
    """C^XY[M][nl] = 4 pi sum_k w_k P Delta^X Delta^Y (Eq. 1)."""
    k = _f64(k)
    DX = _f64(DX)
    DY = _f64(DY)
    single = DX.ndim == 2
    if single:
        DX, DY = DX[None], DY[None]
    M, nk, nl = DX.shape
    assert DY.shape == DX.shape
    Pk = _f64(Pk).reshape(M, nk)
    cl = np.empty((M, nl))
    _load().orc_cl_cross(nk, _ptr(k), nl, M, _ptr(DX), _ptr(DY), _ptr(Pk),
                         _ptr(_f64(wk)) if wk is not None else None, _ptr(cl))
    return cl[0] if single else cl


def cosmic_variance_ratio(cl_test, cl_ref, lmin=2) -> np.ndarray:
    """|Delta C_l| / sigma_CV with sigma_CV = sqrt(2/(2l+1)) |C_l| (Sec. 4.6),
    the auto spectra TT, EE."""
    cl_ref = np.asarray(cl_ref, dtype=np.float64)
    l = lmin + np.arange(cl_ref.shape[-1])
    sig = np.sqrt(2.0 / (2.0 * l + 1.0)) * np.abs(cl_ref)
    return np.abs(np.asarray(cl_test, dtype=np.float64) - cl_ref) / sig


def cosmic_variance_ratio_te(te_test, tt_ref, ee_ref, te_ref, lmin=2) -> np.ndarray:
    """|Delta C^TE_l| / sigma_CV^TE with the cross-spectrum cosmic variance of
    Sec. 4.6, sigma_CV^TE = sqrt(((C^TE)^2 + C^TT C^EE) / (2l+1))."""
    tt = np.asarray(tt_ref, dtype=np.float64)
    ee = np.asarray(ee_ref, dtype=np.float64)
    te = np.asarray(te_ref, dtype=np.float64)
    l = lmin + np.arange(te.shape[-1])
    sig = np.sqrt((te * te + tt * ee) / (2.0 * l + 1.0))
    return np.abs(np.asarray(te_test, dtype=np.float64) - te) / sig
