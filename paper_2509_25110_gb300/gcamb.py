"""Python binding of libgcamb.so (include/gcamb.h): argument marshalling only.

Every function has the name of the C entry point without the `gcamb_` prefix.
Device arrays are torch CUDA tensors (contiguous, stated dtype); streams
default to torch's current stream.  Every step of the computation runs in the
library's kernels; if the library is missing this module raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgcamb.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, EUNSUPPORTED, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
PLAIN64, PLAIN32, BF16X3, TF32X3, F16X3 = 0, 1, 2, 3, 4
F64, F32 = 0, 1
MODE_NAMES = {PLAIN64: "plain64", PLAIN32: "plain32", BF16X3: "bf16x3", TF32X3: "tf32x3", F16X3: "f16x3"}
INFO_N = 8
K_TABLE, K_LOS_PLAIN, K_CL, K_SPLIT, K_WEIGHTS, K_TC, K_REDUCE, K_INTERP = range(8)
K_NAMES = ("bessel_table", "los_plain", "cl", "split_sources", "weights", "los_cl_tc", "reduce", "interp")

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_lib = None


class GcambError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gcamb error %d: %s" % (code, msg))
        self.code = code


def lib():
    """Loads libgcamb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgcamb.so is not built; run paper_2509_25110_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    L.gcamb_version.restype = ctypes.c_char_p
    L.gcamb_last_error.restype = ctypes.c_char_p
    L.gcamb_grid_create.argtypes = [_dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, ctypes.POINTER(_vp)]
    L.gcamb_grid_destroy.argtypes = [_vp]
    L.gcamb_grid_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    L.gcamb_grid_extents.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
    L.gcamb_grid_weights.argtypes = [_vp, _dp, _dp]
    L.gcamb_bessel_table.argtypes = [_vp, ctypes.c_int, _vp]
    L.gcamb_table_bytes.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.gcamb_table_compressed.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.gcamb_sph_bessel.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp]
    L.gcamb_los_transfer.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]
    L.gcamb_cl.argtypes = [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp]
    L.gcamb_los_transfer_e.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]
    L.gcamb_cl_cross.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp]
    L.gcamb_los_cl_workspace.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.gcamb_los_cl.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_size_t, _vp]
    L.gcamb_grid_set_kernel.argtypes = [_vp, ctypes.c_int]
    L.gcamb_grid_create_curved.argtypes = [_dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_vp)]
    L.gcamb_grid_create_lsampled.argtypes = [_dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double,
                                             ctypes.POINTER(_vp)]
    L.gcamb_l_sampling.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)]
    L.gcamb_cl_interp_workspace.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.gcamb_cl_interp.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_size_t, _vp]
    L.gcamb_interp_sources_workspace.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.gcamb_interp_sources.argtypes = [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                       ctypes.c_size_t, _vp]
    L.gcamb_los_transfer_tensor.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
    L.gcamb_los_cl_pair.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
                                    ctypes.c_size_t, _vp]
    L.gcamb_los_cl_te_workspace.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.gcamb_los_cl_te.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
                                  ctypes.c_size_t, _vp]
    L.gcamb_sync.argtypes = [_vp]
    L.gcamb_plan_create.argtypes = [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]
    L.gcamb_plan_destroy.argtypes = [_vp]
    L.gcamb_plan_workspace.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t)]
    L.gcamb_plan_launch.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
    L.gcamb_plan_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    L.gcamb_emu_create.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                   ctypes.POINTER(_vp)]
    L.gcamb_emu_destroy.argtypes = [_vp]
    L.gcamb_emu_num_params.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t)]
    L.gcamb_emu_params.argtypes = [_vp, _vp, _vp]
    L.gcamb_emu_grads.argtypes = [_vp, _vp]
    L.gcamb_emu_norm.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]
    L.gcamb_emu_fit_norm.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]
    L.gcamb_emu_train_step.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_float, _vp, _vp]
    L.gcamb_emu_forward.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp]
    L.gcamb_emu_check.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _vp, _vp]
    L.gcamb_emulate.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, _vp]
    L.gcamb_emu_info.argtypes = [_vp, _vp]
    L.gcamb_emu_save.argtypes = [_vp, ctypes.c_char_p]
    L.gcamb_emu_load.argtypes = [_vp, ctypes.c_char_p]
    L.gcamb_synth_sources.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, _vp]
    L.gcamb_los_cl_noalloc.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
    L.gcamb_profile_enable.argtypes = [ctypes.c_int]
    L.gcamb_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.gcamb_probe_flops.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.gcamb_probe_mma.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp]
    L.gcamb_selftest_wait.argtypes = [_vp, _vp]
    _lib = L
    return L


def _check(rc):
    if rc != OK:
        raise GcambError(rc, lib().gcamb_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


def _dev(t, dtype, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return _vp(t.data_ptr())


def version() -> str:
    return lib().gcamb_version().decode()


def last_error() -> str:
    return lib().gcamb_last_error().decode()


class Grid:
    """Owning wrapper of a gcamb_grid handle."""

    def __init__(self, handle, k, tau, tau0, lmin, lmax, l=None):
        self.handle = handle
        self.k = k
        self.tau = tau
        self.tau0 = tau0
        self.lmin = lmin
        self.lmax = lmax
        # multipole of each output row: every l, or a sampled list
        self.l = np.arange(lmin, lmax + 1) if l is None else np.asarray(l, dtype=np.int64)

    @property
    def nk(self):
        return self.k.size

    @property
    def ntau(self):
        return self.tau.size

    @property
    def nl(self):
        return self.l.size

    def close(self):
        if self.handle is not None:
            grid_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_create(k, tau, tau0, lmin, lmax, eps_cut=0.0) -> Grid:
    k = np.ascontiguousarray(k, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    h = _vp()
    _check(lib().gcamb_grid_create(k.ctypes.data_as(_dp), k.size, tau.ctypes.data_as(_dp), tau.size, float(tau0),
                                   int(lmin), int(lmax), float(eps_cut), ctypes.byref(h)))
    return Grid(h, k.copy(), tau.copy(), float(tau0), int(lmin), int(lmax))


KERNEL_J, KERNEL_EPS, KERNEL_TENSOR_E, KERNEL_TENSOR_B = 0, 1, 2, 3


def grid_set_kernel(g: Grid, kernel: int):
    """Switch a flat grid's table (before it is built) from j_l to another
    kernel of the projection (KERNEL_EPS, KERNEL_TENSOR_E, KERNEL_TENSOR_B)."""
    _check(lib().gcamb_grid_set_kernel(g.handle, int(kernel)))
    g.kernel = int(kernel)
    return g


def grid_create_curved(q, tau, tau0, lmin, lmax, K, eps_cut=0.0) -> Grid:
    """A curved-space grid (K [Mpc^-2] < 0 open, > 0 closed): the kernel is
    the hyperspherical Bessel function of beta = q / sqrt|K|."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    h = _vp()
    _check(lib().gcamb_grid_create_curved(q.ctypes.data_as(_dp), q.size, tau.ctypes.data_as(_dp), tau.size,
                                          float(tau0), int(lmin), int(lmax), float(K), float(eps_cut), ctypes.byref(h)))
    g = Grid(h, q.copy(), tau.copy(), float(tau0), int(lmin), int(lmax))
    g.K = float(K)
    return g


def grid_create_lsampled(k, tau, tau0, lval, eps_cut=0.0) -> Grid:
    """A grid whose rows are the listed multipoles lval (strictly increasing)."""
    k = np.ascontiguousarray(k, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    lv = np.ascontiguousarray(lval, dtype=np.int32)
    h = _vp()
    _check(lib().gcamb_grid_create_lsampled(k.ctypes.data_as(_dp), k.size, tau.ctypes.data_as(_dp), tau.size,
                                            float(tau0), lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), lv.size,
                                            float(eps_cut), ctypes.byref(h)))
    return Grid(h, k.copy(), tau.copy(), float(tau0), int(lv[0]), int(lv[-1]), l=lv.astype(np.int64))


def l_sampling(lmin, lmax, boost) -> np.ndarray:
    """The sampled multipoles of gcamb_l_sampling (boost >= 50: every l)."""
    n = ctypes.c_int()
    _check(lib().gcamb_l_sampling(int(lmin), int(lmax), float(boost), None, ctypes.byref(n)))
    out = np.empty(n.value, dtype=np.int32)
    _check(lib().gcamb_l_sampling(int(lmin), int(lmax), float(boost), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  ctypes.byref(n)))
    return out


def cl_interp(g: Grid, Cl_s, Cl=None, ws=None, stream=None):
    """C_l[M][lmax-lmin+1] on every multipole from Cl_s[M][nl] on the grid's
    sampled rows (natural cubic spline in l of l (l+1) C_l)."""
    import torch
    M = Cl_s.shape[0]
    if Cl is None:
        Cl = torch.empty((M, g.lmax - g.lmin + 1), dtype=torch.float64, device=Cl_s.device)
    if ws is None:
        b = ctypes.c_size_t()
        _check(lib().gcamb_cl_interp_workspace(g.handle, M, ctypes.byref(b)))
        ws = torch.empty(b.value, dtype=torch.uint8, device=Cl_s.device)
    _check(lib().gcamb_cl_interp(g.handle, _dev(Cl_s, torch.float64, (M, g.nl), "Cl_s"), M,
                                 _dev(Cl, torch.float64, (M, g.lmax - g.lmin + 1), "Cl"),
                                 _dev(ws, torch.uint8, name="ws"), ws.numel(), _stream(stream)))
    return Cl


def grid_destroy(g: Grid):
    if g.handle is not None:
        _check(lib().gcamb_grid_destroy(g.handle))
        g.handle = None


def grid_info(g: Grid) -> dict:
    a = (ctypes.c_int64 * INFO_N)()
    _check(lib().gcamb_grid_info(g.handle, a))
    keys = ("nk", "ntau", "nl", "n_ltile", "active", "stored_plain64", "lmin", "lmax")
    return dict(zip(keys, [int(v) for v in a]))


def grid_extents(g: Grid) -> np.ndarray:
    info = grid_info(g)
    out = np.empty((info["nk"], info["n_ltile"]), dtype=np.int32)
    _check(lib().gcamb_grid_extents(g.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return out


def grid_weights(g: Grid):
    wt = np.empty(g.ntau)
    wk = np.empty(g.nk)
    _check(lib().gcamb_grid_weights(g.handle, wt.ctypes.data_as(_dp), wk.ctypes.data_as(_dp)))
    return wt, wk


def bessel_table(g: Grid, mode: int, stream=None):
    _check(lib().gcamb_bessel_table(g.handle, int(mode), _stream(stream)))


def table_bytes(g: Grid, mode: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().gcamb_table_bytes(g.handle, int(mode), ctypes.byref(b)))
    return int(b.value)


def table_compressed(g: Grid, mode: int) -> bool:
    """True when the built table of `mode` lives in compressible device memory."""
    c = ctypes.c_int()
    _check(lib().gcamb_table_compressed(g.handle, int(mode), ctypes.byref(c)))
    return bool(c.value)


def sph_bessel(x, lmax: int, out=None, stream=None):
    """j_0..j_lmax at device FP64 x[n] -> out[n][lmax+1] (FP64)."""
    import torch
    n = x.numel()
    if out is None:
        out = torch.empty((n, lmax + 1), dtype=torch.float64, device=x.device)
    _check(lib().gcamb_sph_bessel(_dev(x, torch.float64, name="x"), n, int(lmax),
                                  _dev(out, torch.float64, (n, lmax + 1), "out"), _stream(stream)))
    return out


def los_transfer(g: Grid, S, mode: int, Delta=None, stream=None):
    """Eq. (2): S[M][nk][ntau] -> Delta[M][nk][nl] (FP64 for PLAIN64, FP32 for PLAIN32)."""
    import torch
    dt = torch.float64 if mode == PLAIN64 else torch.float32
    M = S.shape[0]
    if Delta is None:
        Delta = torch.empty((M, g.nk, g.nl), dtype=dt, device=S.device)
    _check(lib().gcamb_los_transfer(g.handle, _dev(S, dt, (M, g.nk, g.ntau), "S"), M, int(mode),
                                    _dev(Delta, dt, (M, g.nk, g.nl), "Delta"), _stream(stream)))
    return Delta


def los_transfer_e(g: Grid, SP, mode: int, DeltaE=None, stream=None):
    """Eq. (3), E-mode: S_P[M][nk][ntau] -> Delta_E[M][nk][nl] (FP64 for PLAIN64, FP32 for PLAIN32)."""
    import torch
    dt = torch.float64 if mode == PLAIN64 else torch.float32
    M = SP.shape[0]
    if DeltaE is None:
        DeltaE = torch.empty((M, g.nk, g.nl), dtype=dt, device=SP.device)
    _check(lib().gcamb_los_transfer_e(g.handle, _dev(SP, dt, (M, g.nk, g.ntau), "S_P"), M, int(mode),
                                      _dev(DeltaE, dt, (M, g.nk, g.nl), "Delta_E"), _stream(stream)))
    return DeltaE


def los_transfer_tensor(g: Grid, ST, SP, mode: int, out=None, stream=None):
    """Tensor modes: ST, SP[M][nk][ntau] -> (Delta_T, Delta_E, Delta_B), each
    [M][nk][nl] (FP64 for PLAIN64, FP32 for PLAIN32)."""
    import torch
    dt = torch.float64 if mode == PLAIN64 else torch.float32
    M = ST.shape[0]
    if out is None:
        out = tuple(torch.empty((M, g.nk, g.nl), dtype=dt, device=ST.device) for _ in range(3))
    DT, DE, DB = out
    _check(lib().gcamb_los_transfer_tensor(g.handle, _dev(ST, dt, (M, g.nk, g.ntau), "ST"),
                                           _dev(SP, dt, (M, g.nk, g.ntau), "SP"), M, int(mode),
                                           _dev(DT, dt, (M, g.nk, g.nl), "Delta_T"),
                                           _dev(DE, dt, (M, g.nk, g.nl), "Delta_E"),
                                           _dev(DB, dt, (M, g.nk, g.nl), "Delta_B"), _stream(stream)))
    return DT, DE, DB


def interp_sources(g: Grid, k_in, S_in, S_out=None, ws=None, stream=None):
    """Natural cubic spline in k of S_in[M][nk_in][ntau] (FP64 or FP32) from
    the nodes k_in onto the grid's k: -> S_out[M][nk][ntau], same dtype."""
    import torch
    k_in = np.ascontiguousarray(k_in, dtype=np.float64)
    M = S_in.shape[0]
    dt = S_in.dtype
    if S_out is None:
        S_out = torch.empty((M, g.nk, g.ntau), dtype=dt, device=S_in.device)
    if ws is None:
        b = ctypes.c_size_t()
        _check(lib().gcamb_interp_sources_workspace(g.handle, M, k_in.size, ctypes.byref(b)))
        ws = torch.empty(max(1, b.value), dtype=torch.uint8, device=S_in.device)
    _check(lib().gcamb_interp_sources(g.handle, k_in.ctypes.data_as(_dp), k_in.size,
                                      _dev(S_in, dt, (M, k_in.size, g.ntau), "S_in"), M,
                                      F64 if dt == torch.float64 else F32, _dev(S_out, dt, (M, g.nk, g.ntau), "S_out"),
                                      _dev(ws, torch.uint8, name="ws"), ws.numel(), _stream(stream)))
    return S_out


def cl_cross(g: Grid, DX, DY, Pk, Cl=None, stream=None):
    """Eq. (1) with X, Y in {T, E}: DX, DY [M][nk][nl], Pk [M][nk] -> C^XY [M][nl] (FP64)."""
    import torch
    M = DX.shape[0]
    d_dtype = F64 if DX.dtype == torch.float64 else F32
    if Cl is None:
        Cl = torch.empty((M, g.nl), dtype=torch.float64, device=DX.device)
    _check(lib().gcamb_cl_cross(g.handle, _dev(DX, DX.dtype, (M, g.nk, g.nl), "DX"),
                                _dev(DY, DX.dtype, (M, g.nk, g.nl), "DY"), d_dtype,
                                _dev(Pk, torch.float64, (M, g.nk), "Pk"), M, _dev(Cl, torch.float64, (M, g.nl), "Cl"),
                                _stream(stream)))
    return Cl


def cl(g: Grid, Delta, Pk, Cl=None, stream=None):
    """Eq. (1): Delta[M][nk][nl], Pk[M][nk] -> Cl[M][nl] (FP64)."""
    import torch
    M = Delta.shape[0]
    d_dtype = F64 if Delta.dtype == torch.float64 else F32
    if Cl is None:
        Cl = torch.empty((M, g.nl), dtype=torch.float64, device=Delta.device)
    _check(lib().gcamb_cl(g.handle, _dev(Delta, Delta.dtype, (M, g.nk, g.nl), "Delta"), d_dtype,
                          _dev(Pk, torch.float64, (M, g.nk), "Pk"), M, _dev(Cl, torch.float64, (M, g.nl), "Cl"),
                          _stream(stream)))
    return Cl


def los_cl_workspace(g: Grid, M: int, mode: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().gcamb_los_cl_workspace(g.handle, int(M), int(mode), ctypes.byref(b)))
    return int(b.value)


def los_cl(g: Grid, S, Pk, mode: int, Cl=None, ws=None, stream=None):
    """Fused batched Eqs. (1)-(2) on the tensor cores: S[M][nk][ntau] FP32 -> Cl[M][nl] FP64."""
    import torch
    M = S.shape[0]
    need = los_cl_workspace(g, M, mode) if M > 0 else 0  # M = 0: the call writes nothing
    if ws is None:
        ws = torch.empty(max(1, need), dtype=torch.uint8, device=S.device)
    if Cl is None:
        Cl = torch.empty((M, g.nl), dtype=torch.float64, device=S.device)
    _check(lib().gcamb_los_cl(g.handle, _dev(S, torch.float32, (M, g.nk, g.ntau), "S"),
                              _dev(Pk, torch.float64, (M, g.nk), "Pk"), M, int(mode),
                              _dev(Cl, torch.float64, (M, g.nl), "Cl"), _dev(ws, torch.uint8, name="ws"),
                              ws.numel(), _stream(stream)))
    return Cl


def los_cl_te_workspace(g: Grid, M: int, mode: int = BF16X3) -> int:
    b = ctypes.c_size_t()
    _check(lib().gcamb_los_cl_te_workspace(g.handle, M, int(mode), ctypes.byref(b)))
    return b.value


def los_cl_te(g: Grid, ST, SP, Pk, mode: int = BF16X3, out=None, ws=None, stream=None):
    """Batched temperature + E-mode on the tensor cores (Eqs. 1-3):
    ST, SP[M][nk][ntau] FP32 -> (C^TT, C^EE, C^TE), each [M][nl] FP64."""
    import torch
    M = ST.shape[0]
    if ws is None:
        ws = torch.empty(max(1, los_cl_te_workspace(g, M, mode)), dtype=torch.uint8, device=ST.device)
    if out is None:
        out = tuple(torch.empty((M, g.nl), dtype=torch.float64, device=ST.device) for _ in range(3))
    tt, ee, te = out
    _check(lib().gcamb_los_cl_te(g.handle, _dev(ST, torch.float32, (M, g.nk, g.ntau), "ST"),
                                 _dev(SP, torch.float32, (M, g.nk, g.ntau), "SP"),
                                 _dev(Pk, torch.float64, (M, g.nk), "Pk"), M, int(mode),
                                 _dev(tt, torch.float64, (M, g.nl), "ClTT"), _dev(ee, torch.float64, (M, g.nl), "ClEE"),
                                 _dev(te, torch.float64, (M, g.nl), "ClTE"), _dev(ws, torch.uint8, name="ws"),
                                 ws.numel(), _stream(stream)))
    return tt, ee, te


def los_cl_pair(gx: Grid, gy: Grid, SX, SY, Pk, out=None, ws=None, stream=None):
    """Two fields on kernel grids with the same layout (e.g. tensor T and E),
    batched on the tensor cores: -> (C^XX, C^YY, C^XY), each [M][nl] FP64."""
    import torch
    M = SX.shape[0]
    if ws is None:
        ws = torch.empty(max(1, los_cl_te_workspace(gx, M)), dtype=torch.uint8, device=SX.device)
    if out is None:
        out = tuple(torch.empty((M, gx.nl), dtype=torch.float64, device=SX.device) for _ in range(3))
    xx, yy, xy = out
    _check(lib().gcamb_los_cl_pair(gx.handle, gy.handle, _dev(SX, torch.float32, (M, gx.nk, gx.ntau), "SX"),
                                   _dev(SY, torch.float32, (M, gx.nk, gx.ntau), "SY"),
                                   _dev(Pk, torch.float64, (M, gx.nk), "Pk"), M, BF16X3,
                                   _dev(xx, torch.float64, (M, gx.nl), "ClXX"), _dev(yy, torch.float64, (M, gx.nl), "ClYY"),
                                   _dev(xy, torch.float64, (M, gx.nl), "ClXY"), _dev(ws, torch.uint8, name="ws"),
                                   ws.numel(), _stream(stream)))
    return xx, yy, xy


class Plan:
    """Owning wrapper of a gcamb_plan handle (an uneven batch on one grid)."""

    def __init__(self, handle, grid, M):
        self.handle = handle
        self.grid = grid
        self.M = M

    def close(self):
        if self.handle is not None:
            plan_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_create(g: Grid, M: int, lmax_m=None, nk_m=None, mode: int = F16X3, tune: bool = False) -> Plan:
    """Plan for M sources; lmax_m / nk_m are per-source l_max and k-prefix
    lengths (both None: every source uses the whole grid)."""
    h = _vp()
    if (lmax_m is None) != (nk_m is None):
        raise ValueError("give both lmax_m and nk_m, or neither")
    la = na = None
    if lmax_m is not None:
        la = np.ascontiguousarray(lmax_m, dtype=np.int32)
        na = np.ascontiguousarray(nk_m, dtype=np.int32)
        if la.size != M or na.size != M:
            raise ValueError("lmax_m and nk_m must have M entries")
    _check(lib().gcamb_plan_create(g.handle, int(M), None if la is None else _vp(la.ctypes.data),
                                   None if na is None else _vp(na.ctypes.data), int(mode), 1 if tune else 0,
                                   ctypes.byref(h)))
    return Plan(h, g, int(M))


def plan_destroy(p: Plan):
    if p.handle is not None:
        _check(lib().gcamb_plan_destroy(p.handle))
        p.handle = None


def plan_workspace(p: Plan) -> int:
    b = ctypes.c_size_t()
    _check(lib().gcamb_plan_workspace(p.handle, ctypes.byref(b)))
    return int(b.value)


def plan_info(p: Plan) -> dict:
    a = (ctypes.c_int64 * 13)()
    _check(lib().gcamb_plan_info(p.handle, a))
    keys = ("tile", "items", "ctas", "captures", "replays", "tuned", "M", "workspace", "fused", "lp", "items_per_cta",
            "tail", "kalign")
    return dict(zip(keys, [int(v) for v in a]))


def plan_launch(p: Plan, S, Pk, Cl=None, ws=None, stream=None):
    """Runs the plan (graph replay after the first launch): S[M][nk][ntau]
    FP32, Pk[M][nk] FP64 -> Cl[M][nl] FP64."""
    import torch
    g = p.grid
    M = p.M
    if ws is None:
        ws = torch.empty(plan_workspace(p), dtype=torch.uint8, device=S.device)
    if Cl is None:
        Cl = torch.empty((M, g.nl), dtype=torch.float64, device=S.device)
    _check(lib().gcamb_plan_launch(p.handle, _dev(S, torch.float32, (M, g.nk, g.ntau), "S"),
                                   _dev(Pk, torch.float64, (M, g.nk), "Pk"),
                                   _dev(Cl, torch.float64, (M, g.nl), "Cl"), _dev(ws, torch.uint8, name="ws"),
                                   ws.numel(), _stream(stream)))
    return Cl


def los_cl_noalloc(g: Grid, S, Pk, mode: int, Cl, status=None, stream=None):
    """gcamb_los_cl without a workspace: the library's fixed 64 MiB device
    buffer holds all scratch, and nothing is allocated by the call.  Cl must
    be given (this function allocates nothing either); status, if given, is a
    device int32 tensor of one element."""
    import torch
    M = S.shape[0]
    st = _vp(None) if status is None else _dev(status, torch.int32, (1,), "status")
    _check(lib().gcamb_los_cl_noalloc(g.handle, _dev(S, torch.float32, (M, g.nk, g.ntau), "S"),
                                      _dev(Pk, torch.float64, (M, g.nk), "Pk"), M, int(mode),
                                      _dev(Cl, torch.float64, (M, g.nl), "Cl"), st, _stream(stream)))
    return Cl


def sync(stream=None):
    _check(lib().gcamb_sync(_stream(stream)))


def probe_mma(A, B, C=None, stream=None):
    """C[128][128] = A[128][K] . B[128][K]^T through the library's tcgen05
    GEMM (bf16 operands, FP32 accumulation): the accumulation self-test."""
    import torch
    K = A.shape[1]
    if C is None:
        C = torch.empty((128, 128), dtype=torch.float32, device=A.device)
    _check(lib().gcamb_probe_mma(_dev(A, torch.float32, (128, K), "A"), _dev(B, torch.float32, (128, K), "B"), int(K),
                                 _dev(C, torch.float32, (128, 128), "C"), _stream(stream)))
    return C


def probe_flops(what: int) -> float:
    f = ctypes.c_double()
    _check(lib().gcamb_probe_flops(int(what), ctypes.byref(f)))
    return float(f.value)


def selftest_wait(status=None, stream=None):
    """Device-side failure path self-test: a bounded wait on an mbarrier that
    nothing arrives on gives up after one second and reports GCAMB_ETIMEOUT,
    in `status` (device int32 tensor of one element) or, without it, through
    the next sync()."""
    import torch
    st = _vp(None) if status is None else _dev(status, torch.int32, (1,), "status")
    _check(lib().gcamb_selftest_wait(st, _stream(stream)))


def profile_enable(on: bool = True):
    """Starts (clearing the accumulators) or stops the library's event tracer."""
    _check(lib().gcamb_profile_enable(1 if on else 0))


def profile_read(kernel: int):
    """(total device ms, launches) of one kernel id since profile_enable."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().gcamb_profile_read(int(kernel), ctypes.byref(ms), ctypes.byref(n)))
    return float(ms.value), int(n.value)


# ---------------------------------------------------------------- emulator

class Emu:
    """Owning wrapper of a gcamb_emu handle."""

    def __init__(self, handle, grid, width, depth, max_batch):
        self.handle = handle
        self.grid = grid
        self.width = width
        self.depth = depth
        self.max_batch = max_batch
        self.n_in = 9
        self.n_out = grid.nl

    def close(self):
        if self.handle is not None:
            _check(lib().gcamb_emu_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def emu_create(g: Grid, width: int = 512, depth: int = 3, max_batch: int = 4096, seed: int = 0) -> Emu:
    h = _vp()
    _check(lib().gcamb_emu_create(g.handle, 9, int(width), int(depth), int(max_batch), int(seed), ctypes.byref(h)))
    return Emu(h, g, int(width), int(depth), int(max_batch))


def emu_destroy(e: Emu):
    e.close()


def emu_num_params(e: Emu) -> int:
    n = ctypes.c_size_t()
    _check(lib().gcamb_emu_num_params(e.handle, ctypes.byref(n)))
    return int(n.value)


def emu_layer_shapes(e: Emu):
    sizes = [9] + [e.width] * e.depth + [e.n_out]
    return [(b, a) for a, b in zip(sizes[:-1], sizes[1:])]


def emu_params(e: Emu, new=None) -> np.ndarray:
    """Flat float32 parameters (per layer W [out][in] then b [out]); sets them first if `new` is given."""
    n = emu_num_params(e)
    out = np.empty(n, dtype=np.float32)
    src = None
    if new is not None:
        src = np.ascontiguousarray(new, dtype=np.float32)
        if src.size != n:
            raise ValueError("expected %d parameters" % n)
    _check(lib().gcamb_emu_params(e.handle, _vp(out.ctypes.data), None if src is None else _vp(src.ctypes.data)))
    return out


def emu_grads(e: Emu) -> np.ndarray:
    out = np.empty(emu_num_params(e), dtype=np.float32)
    _check(lib().gcamb_emu_grads(e.handle, _vp(out.ctypes.data)))
    return out


def unflatten(e: Emu, flat):
    """Flat parameter vector -> ([W_l], [b_l]) as float64 arrays."""
    Ws, bs, o = [], [], 0
    for (nout, nin) in emu_layer_shapes(e):
        Ws.append(np.asarray(flat[o:o + nout * nin], dtype=np.float64).reshape(nout, nin))
        o += nout * nin
        bs.append(np.asarray(flat[o:o + nout], dtype=np.float64))
        o += nout
    return Ws, bs


def flatten(Ws, bs) -> np.ndarray:
    parts = []
    for W, b in zip(Ws, bs):
        parts += [np.asarray(W).ravel(), np.asarray(b).ravel()]
    return np.concatenate(parts).astype(np.float32)


def emu_norm(e: Emu, mu_x=None, sd_x=None, mu_y=None, sd_y=None) -> dict:
    """Reads the normalisation, or sets it when all four arrays are given."""
    arrs = [np.zeros(9, np.float32), np.zeros(9, np.float32), np.zeros(e.n_out, np.float32),
            np.zeros(e.n_out, np.float32)]
    setting = mu_x is not None
    if setting:
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (mu_x, sd_x, mu_y, sd_y)]
    _check(lib().gcamb_emu_norm(e.handle, *[_vp(a.ctypes.data) for a in arrs], 1 if setting else 0))
    return dict(zip(("mu_x", "sd_x", "mu_y", "sd_y"), arrs))


def emu_fit_norm(e: Emu, X, Cl, Y=None, per_l=False, stream=None):
    import torch
    N = X.shape[0]
    if Y is None:
        Y = torch.empty((N, e.n_out), dtype=torch.float32, device=X.device)
    _check(lib().gcamb_emu_fit_norm(e.handle, _dev(X, torch.float32, (N, 9), "X"),
                                    _dev(Cl, torch.float64, (N, e.n_out), "Cl"), N, 1 if per_l else 0,
                                    _dev(Y, torch.float32, (N, e.n_out), "Y"), _stream(stream)))
    return Y


def emu_train_step(e: Emu, X, Y, idx, B: int, lr: float, loss=None, stream=None):
    import torch
    ip = _vp(None) if idx is None else _dev(idx, torch.int32, name="idx")
    lp = _vp(None) if loss is None else _dev(loss, torch.float32, (1,), "loss")
    _check(lib().gcamb_emu_train_step(e.handle, _dev(X, torch.float32, name="X"), _dev(Y, torch.float32, name="Y"),
                                      ip, int(B), float(lr), lp, _stream(stream)))
    return loss


def emu_forward(e: Emu, X, Y=None, stream=None):
    import torch
    B = X.shape[0]
    if Y is None:
        Y = torch.empty((B, e.n_out), dtype=torch.float32, device=X.device)
    _check(lib().gcamb_emu_forward(e.handle, _dev(X, torch.float32, (B, 9), "X"), B,
                                   _dev(Y, torch.float32, (B, e.n_out), "Y"), _stream(stream)))
    return Y


def emu_check(e: Emu, X, Cl_ref, tol: float, min_count: int = 4, stream=None) -> dict:
    import torch
    N = X.shape[0]
    rep = np.zeros(6)
    _check(lib().gcamb_emu_check(e.handle, _dev(X, torch.float32, (N, 9), "X"),
                                 _dev(Cl_ref, torch.float64, (N, e.n_out), "Cl_ref"), N, float(tol), int(min_count),
                                 _vp(rep.ctypes.data), _stream(stream)))
    keys = ("max_err", "mean_err", "frac_within_tol", "frac_cells_trusted", "frac_served", "cells")
    return dict(zip(keys, rep.tolist()))


def emulate(e: Emu, X, Cl=None, used_fallback=None, stream=None):
    """C_l[B][n_out] from the emulator (trusted cells) or the projection."""
    import torch
    B = X.shape[0]
    if Cl is None:
        Cl = torch.empty((B, e.n_out), dtype=torch.float64, device=X.device)
    if used_fallback is None:
        used_fallback = torch.empty(B, dtype=torch.int32, device=X.device)
    _check(lib().gcamb_emulate(e.handle, _dev(X, torch.float32, (B, 9), "X"), B,
                               _dev(Cl, torch.float64, (B, e.n_out), "Cl"),
                               _dev(used_fallback, torch.int32, (B,), "used_fallback"), _stream(stream)))
    return Cl, used_fallback


def emu_info(e: Emu) -> dict:
    a = np.zeros(8)
    _check(lib().gcamb_emu_info(e.handle, _vp(a.ctypes.data)))
    keys = ("params", "steps", "check_max_err", "check_tol", "frac_cells_trusted", "n_out", "device_error", "width")
    return dict(zip(keys, a.tolist()))


def emu_save(e: Emu, path: str):
    _check(lib().gcamb_emu_save(e.handle, str(path).encode()))


def emu_load(e: Emu, path: str):
    _check(lib().gcamb_emu_load(e.handle, str(path).encode()))


def synth_sources(g: Grid, X, S=None, Pk=None, stream=None):
    """Synthetic sources S[M][nk][ntau] (float) and P[M][nk] (double) from features X[M][9]."""
    import torch
    M = X.shape[0]
    if S is None:
        S = torch.empty((M, g.nk, g.ntau), dtype=torch.float32, device=X.device)
    if Pk is None:
        Pk = torch.empty((M, g.nk), dtype=torch.float64, device=X.device)
    _check(lib().gcamb_synth_sources(g.handle, _dev(X, torch.float32, (M, 9), "X"), M,
                                     _dev(S, torch.float32, (M, g.nk, g.ntau), "S"),
                                     _dev(Pk, torch.float64, (M, g.nk), "Pk"), _stream(stream)))
    return S, Pk
