"""Seeded synthetic inputs for the line-of-sight projection.

This module only *creates inputs*: wavenumber and conformal-time grids, the
per-model generator parameters, the source functions S(k, tau) and the
primordial spectrum P(k).  It holds none of the projection's arithmetic
(no quadrature weights, no Bessel functions, no transfer or C_l sums), so the
CPU oracle and the CUDA path can both be fed from it without sharing any code
of the method itself.

The paper's workloads are full CAMB runs with Planck parameters (Sec. 3.1);
those source functions come from a Boltzmann ODE that is out of scope here.
The synthetic source below stands in for them: a visibility-like Gaussian peak
near recombination, modulated by acoustic oscillations and Silk-like damping,
plus a broad late-time (ISW-like) term.  With S_T playing the role of the
temperature source of Eq. (2) and P playing P_R of Eq. (1), the sizes and
value distributions follow the five workloads of the build's scope table.

Random numbers: a counter-based generator, the SplitMix64 output function
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) applied to the counter (seed << 40) | (model << 8) | slot, so any
model's parameters can be regenerated independently of batch composition.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

MASK64 = (1 << 64) - 1

# Fixed generator constants of the synthetic source family.
TAU_L = 11000.0   # centre of the late-time term [Mpc]
S_L = 2000.0      # width of the late-time term [Mpc]
K_L = 0.01        # k-scale of the late-time term [1/Mpc]
A_S = 2.1e-9      # primordial amplitude
A_P = 0.3         # polarisation / temperature amplitude at recombination
TAU_RE = 4700.0   # centre of the reionisation term of the polarisation source [Mpc]
S_RE = 600.0      # its width [Mpc]
K_RE = 0.005      # its k-scale [1/Mpc]
B_RE = 0.02       # its amplitude
K_PIVOT = 0.05    # pivot scale [1/Mpc]

# Parameter slots drawn per model, in counter order.
SLOT_TAU_STAR, SLOT_SIGMA, SLOT_RS, SLOT_PHI, SLOT_KD, SLOT_B, SLOT_NS, SLOT_LMAX = range(8)
SLOT_AF, SLOT_OMEGA, SLOT_PHIF = 8, 9, 10   # primordial features
FEATURE_RANGES = {"A_f": (0.0, 0.05), "omega": (10.0, 50.0), "phi_f": (0.0, 2.0 * math.pi)}
PARAM_RANGES = {
    "tau_star": (270.0, 300.0),
    "sigma": (15.0, 25.0),
    "r_s": (140.0, 150.0),
    "phi": (0.0, math.pi),
    "k_D": (0.1, 0.2),
    "b": (0.0, 0.1),
    "n_s": (0.94, 0.99),
}
PARAM_NAMES = ("tau_star", "sigma", "r_s", "phi", "k_D", "b", "n_s")


def splitmix64(counter: int) -> int:
    """SplitMix64 output for one counter value (one step from state=counter)."""
    z = (counter + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def uniform(seed: int, model: int, slot: int) -> float:
    """U[0,1) double from the top 53 bits of the SplitMix64 output."""
    c = ((seed & 0xFFFFFF) << 40) | ((model & 0xFFFFFFFF) << 8) | (slot & 0xFF)
    return (splitmix64(c) >> 11) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class ModelParams:
    """Generator parameters of M models (arrays of length M)."""
    tau_star: np.ndarray
    sigma: np.ndarray
    r_s: np.ndarray
    phi: np.ndarray
    k_D: np.ndarray
    b: np.ndarray
    n_s: np.ndarray
    lmax: Optional[np.ndarray] = None  # only for the uneven-batch workload

    @property
    def M(self) -> int:
        return int(self.tau_star.shape[0])

    def subset(self, idx) -> "ModelParams":
        idx = np.asarray(idx)
        kw = {n: getattr(self, n)[idx] for n in PARAM_NAMES}
        kw["lmax"] = None if self.lmax is None else self.lmax[idx]
        return ModelParams(**kw)

    def as_matrix(self) -> np.ndarray:
        """[M, 7] float64 in PARAM_NAMES order."""
        return np.stack([getattr(self, n) for n in PARAM_NAMES], axis=1)


def model_params(M: int, seed: int = 0, first_model: int = 0,
                 lmax_range: Optional[tuple] = None) -> ModelParams:
    """Draw M models' parameters (models first_model .. first_model+M-1)."""
    out = {n: np.empty(M) for n in PARAM_NAMES}
    slots = dict(zip(PARAM_NAMES, (SLOT_TAU_STAR, SLOT_SIGMA, SLOT_RS, SLOT_PHI,
                                   SLOT_KD, SLOT_B, SLOT_NS)))
    lm = np.empty(M, dtype=np.int64) if lmax_range else None
    for i in range(M):
        m = first_model + i
        for n in PARAM_NAMES:
            lo, hi = PARAM_RANGES[n]
            out[n][i] = lo + (hi - lo) * uniform(seed, m, slots[n])
        if lm is not None:
            lo, hi = lmax_range
            lm[i] = lo + int(math.floor(uniform(seed, m, SLOT_LMAX) * (hi - lo + 1)))
    return ModelParams(lmax=lm, **out)


# ----------------------------------------------------------------------------
# Grids
# ----------------------------------------------------------------------------

def log_grid(lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(np.linspace(math.log(lo), math.log(hi), n))


def uniform_grid(lo: float, hi: float, n: int) -> np.ndarray:
    return np.linspace(lo, hi, n)


def dense_tau_grid(n_peak: int = 1000, n_rest: int = 1000) -> np.ndarray:
    """Grid dense around recombination: n_peak points on [200, 600) then
    n_rest points on [600, 14000]."""
    a = 200.0 + (600.0 - 200.0) * np.arange(n_peak) / n_peak
    b = np.linspace(600.0, 14000.0, n_rest)
    return np.concatenate([a, b])


def master_linear_k(n: int = 3000, kmax: float = 0.5) -> np.ndarray:
    """Shared linear k grid of the uneven batch: k_j = (j+1) * kmax / n."""
    return (np.arange(n) + 1.0) * (kmax / n)


def uneven_nk(lmax: np.ndarray, n_master: int = 3000) -> np.ndarray:
    """k-prefix length of each uneven-batch model, scaled with its l_max."""
    return 1000 + np.rint(2000.0 * (np.asarray(lmax) - 1500) / 4500.0).astype(np.int64)


@dataclasses.dataclass
class Workload:
    name: str
    k: np.ndarray
    tau: np.ndarray
    tau0: float
    lmin: int
    lmax: int
    M: int

    @property
    def nk(self):
        return int(self.k.shape[0])

    @property
    def ntau(self):
        return int(self.tau.shape[0])

    @property
    def nl(self):
        return self.lmax - self.lmin + 1


def workload(name: str, M: Optional[int] = None) -> Workload:
    """The named synthetic workloads.

    plain_lmax500      : 1 model, l 2..500, 300 k log 1e-4..0.3, 400 tau uniform [200,14000]
    plain_lmax5000     : 1 model, l 2..5000, 3000 k log 1e-5..1.0, 2000 tau dense near tau*
    batched_lmax2500   : 256 models, l 2..2500, 2000 k log 1e-4..0.3, 1000 tau uniform
    uneven_lmax6000    : 1000 models on a 3000-point linear k grid, 1000 tau uniform
    features_lmax2500  : 256 models, l 2..2500, 8000 k log 1e-4..0.3 (sources made on
                         1000 k and interpolated), 1000 tau uniform, log-oscillating P(k)
    lsampled_lmax2500  : 256 models, l 2..2500, 400 k log 1e-4..0.01 then 1800 k linear to
                         0.3 (dk = 1.6e-4 < 2 pi / tau0: the projection's oscillations in k
                         are resolved, so C_l is smooth in l), 1000 tau uniform
    tensor_lmax1500    : 1 model, l 2..1500, 1000 k log 1e-4..3000/tau0, 1000 tau uniform
                         (tensor modes: l_max and k tau0 <= 3000 as in the paper's runs)
    """
    tau0 = 14000.0
    if name == "plain_lmax500":
        wl = Workload(name, log_grid(1e-4, 0.3, 300), uniform_grid(200.0, 14000.0, 400), tau0, 2, 500, 1)
    elif name == "plain_lmax5000":
        wl = Workload(name, log_grid(1e-5, 1.0, 3000), dense_tau_grid(), tau0, 2, 5000, 1)
    elif name == "batched_lmax2500":
        wl = Workload(name, log_grid(1e-4, 0.3, 2000), uniform_grid(200.0, 14000.0, 1000), tau0, 2, 2500, 256)
    elif name == "features_lmax2500":
        wl = Workload(name, log_grid(1e-4, 0.3, 8000), uniform_grid(200.0, 14000.0, 1000), tau0, 2, 2500, 256)
    elif name == "lsampled_lmax2500":
        k = np.concatenate([np.geomspace(1e-4, 0.01, 401)[:-1], np.linspace(0.01, 0.3, 1800)])
        wl = Workload(name, k, uniform_grid(200.0, 14000.0, 1000), tau0, 2, 2500, 256)
    elif name == "tensor_lmax1500":
        wl = Workload(name, log_grid(1e-4, 3000.0 / tau0, 1000), uniform_grid(200.0, 14000.0, 1000), tau0, 2, 1500, 1)
    elif name == "uneven_lmax6000":
        wl = Workload(name, master_linear_k(), uniform_grid(200.0, 14000.0, 1000), tau0, 2, 6000, 1000)
    else:
        raise KeyError(name)
    if M is not None:
        wl.M = M
    return wl


# ----------------------------------------------------------------------------
# Sources and primordial spectrum
# ----------------------------------------------------------------------------

def sources(k: np.ndarray, tau: np.ndarray, p: ModelParams, dtype=np.float64) -> np.ndarray:
    """S[M][nk][ntau] evaluated in float64, returned in `dtype`.

    S(k,tau) = g(tau) cos(k r_s + phi) exp(-(k/k_D)^2)
             + b exp(-(tau-tau_L)^2 / (2 s_L^2)) exp(-k/k_L),
    g = unit-area Gaussian of mean tau_star and width sigma.
    """
    k = np.asarray(k, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    out = np.empty((p.M, k.size, tau.size), dtype=dtype)
    late_tau = np.exp(-(tau - TAU_L) ** 2 / (2.0 * S_L ** 2))
    late_k = np.exp(-k / K_L)
    for m in range(p.M):
        g = np.exp(-(tau - p.tau_star[m]) ** 2 / (2.0 * p.sigma[m] ** 2)) / (p.sigma[m] * math.sqrt(2.0 * math.pi))
        ak = np.cos(k * p.r_s[m] + p.phi[m]) * np.exp(-(k / p.k_D[m]) ** 2)
        out[m] = (ak[:, None] * g[None, :] + p.b[m] * late_k[:, None] * late_tau[None, :]).astype(dtype)
    return out


def sources_torch(k, tau, p: ModelParams, device, dtype=None, nk_per_model=None):
    """Same as `sources`, evaluated with torch in float64 on `device` and cast
    to `dtype` (default float32).  For the full-size benchmark inputs.

    If nk_per_model is given, rows k >= nk_per_model[m] are set to zero."""
    import torch
    dtype = dtype or torch.float32
    kt = torch.as_tensor(np.asarray(k, dtype=np.float64), device=device)
    tt = torch.as_tensor(np.asarray(tau, dtype=np.float64), device=device)
    out = torch.empty((p.M, kt.numel(), tt.numel()), dtype=dtype, device=device)
    late_tau = torch.exp(-(tt - TAU_L) ** 2 / (2.0 * S_L ** 2))
    late_k = torch.exp(-kt / K_L)
    for m in range(p.M):
        g = torch.exp(-(tt - float(p.tau_star[m])) ** 2 / (2.0 * float(p.sigma[m]) ** 2)) / (
            float(p.sigma[m]) * math.sqrt(2.0 * math.pi))
        ak = torch.cos(kt * float(p.r_s[m]) + float(p.phi[m])) * torch.exp(-(kt / float(p.k_D[m])) ** 2)
        s = ak[:, None] * g[None, :] + float(p.b[m]) * late_k[:, None] * late_tau[None, :]
        if nk_per_model is not None:
            s[int(nk_per_model[m]):] = 0.0
        out[m] = s.to(dtype)
    return out


def sources_pol(k: np.ndarray, tau: np.ndarray, p: ModelParams, dtype=np.float64) -> np.ndarray:
    """Polarisation source S_P[M][nk][ntau] of the E-mode projection (Eq. 3),
    in float64, returned in `dtype`: the visibility peak of `sources` a quarter
    period out of phase (the quadrupole follows the velocity), plus a broad
    reionisation term at late times and large scales,

    S_P(k,tau) = A_P g(tau) sin(k r_s + phi) exp(-(k/k_D)^2)
               + B_RE exp(-(tau-TAU_RE)^2 / (2 S_RE^2)) exp(-k/K_RE).
    """
    k = np.asarray(k, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    out = np.empty((p.M, k.size, tau.size), dtype=dtype)
    re_tau = np.exp(-(tau - TAU_RE) ** 2 / (2.0 * S_RE ** 2))
    re_k = B_RE * np.exp(-k / K_RE)
    for m in range(p.M):
        g = np.exp(-(tau - p.tau_star[m]) ** 2 / (2.0 * p.sigma[m] ** 2)) / (p.sigma[m] * math.sqrt(2.0 * math.pi))
        ak = A_P * np.sin(k * p.r_s[m] + p.phi[m]) * np.exp(-(k / p.k_D[m]) ** 2)
        out[m] = (ak[:, None] * g[None, :] + re_k[:, None] * re_tau[None, :]).astype(dtype)
    return out


def sources_pol_torch(k, tau, p: ModelParams, device, dtype=None):
    """Same as `sources_pol`, evaluated with torch in float64 on `device` and
    cast to `dtype` (default float32)."""
    import torch
    dtype = dtype or torch.float32
    kt = torch.as_tensor(np.asarray(k, dtype=np.float64), device=device)
    tt = torch.as_tensor(np.asarray(tau, dtype=np.float64), device=device)
    out = torch.empty((p.M, kt.numel(), tt.numel()), dtype=dtype, device=device)
    re_tau = torch.exp(-(tt - TAU_RE) ** 2 / (2.0 * S_RE ** 2))
    re_k = B_RE * torch.exp(-kt / K_RE)
    for m in range(p.M):
        g = torch.exp(-(tt - float(p.tau_star[m])) ** 2 / (2.0 * float(p.sigma[m]) ** 2)) / (
            float(p.sigma[m]) * math.sqrt(2.0 * math.pi))
        ak = A_P * torch.sin(kt * float(p.r_s[m]) + float(p.phi[m])) * torch.exp(-(kt / float(p.k_D[m])) ** 2)
        out[m] = (ak[:, None] * g[None, :] + re_k[:, None] * re_tau[None, :]).to(dtype)
    return out


def sources_tensor(k: np.ndarray, tau: np.ndarray, p: ModelParams, dtype=np.float64):
    """Tensor-mode sources (ST, SP), each [M][nk][ntau] in float64, returned in
    `dtype`: the gravitational-wave amplitude at recombination,
    h(k) = sin(k tau*) / (k tau*), times the visibility peak g(tau), plus a
    late term (temperature) and the reionisation term (polarisation):

    ST(k,tau) = h(k) [g(tau) + b 1e-3 exp(-(tau-TAU_L)^2 / (2 S_L^2))],
    SP(k,tau) = h(k) [A_P g(tau) + B_RE exp(-(tau-TAU_RE)^2 / (2 S_RE^2))].
    """
    k = np.asarray(k, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    ST = np.empty((p.M, k.size, tau.size), dtype=dtype)
    SP = np.empty_like(ST)
    late = np.exp(-(tau - TAU_L) ** 2 / (2.0 * S_L ** 2))
    re = np.exp(-(tau - TAU_RE) ** 2 / (2.0 * S_RE ** 2))
    for m in range(p.M):
        g = np.exp(-(tau - p.tau_star[m]) ** 2 / (2.0 * p.sigma[m] ** 2)) / (p.sigma[m] * math.sqrt(2.0 * math.pi))
        u = k * p.tau_star[m]
        h = np.sin(u) / u
        ST[m] = (h[:, None] * (g + 1e-3 * p.b[m] * late)[None, :]).astype(dtype)
        SP[m] = (h[:, None] * (A_P * g + B_RE * re)[None, :]).astype(dtype)
    return ST, SP


def primordial_tensor(k: np.ndarray, p: ModelParams, r: float = 0.1, A_s: float = A_S) -> np.ndarray:
    """P_t[M][nk] = r A_s (k/0.05)^n_t, n_t = -r/8 (the single-field
    consistency relation), float64."""
    k = np.asarray(k, dtype=np.float64)
    return np.broadcast_to(r * A_s * np.power(k / K_PIVOT, -r / 8.0), (p.M, k.size)).copy()


def feature_params(M: int, seed: int = 0, first_model: int = 0) -> dict:
    """Per-model parameters of a logarithmic primordial oscillation (the
    resonant features of Sec. 5): amplitude A_f, log-frequency omega, phase."""
    out = {n: np.empty(M) for n in FEATURE_RANGES}
    for i in range(M):
        for n, slot in (("A_f", SLOT_AF), ("omega", SLOT_OMEGA), ("phi_f", SLOT_PHIF)):
            lo, hi = FEATURE_RANGES[n]
            out[n][i] = lo + (hi - lo) * uniform(seed, first_model + i, slot)
    return out


def primordial_features(k: np.ndarray, p: ModelParams, f: dict, A_s: float = A_S) -> np.ndarray:
    """P[M][nk] = A_s (k/0.05)^(n_s-1) [1 + A_f sin(omega ln(k/0.05) + phi_f)]."""
    k = np.asarray(k, dtype=np.float64)
    lk = np.log(k / K_PIVOT)[None, :]
    base = A_s * np.exp((p.n_s[:, None] - 1.0) * lk)
    return base * (1.0 + f["A_f"][:, None] * np.sin(f["omega"][:, None] * lk + f["phi_f"][:, None]))


def primordial(k: np.ndarray, p: ModelParams, A_s: float = A_S) -> np.ndarray:
    """P[M][nk] = A_s (k/0.05)^(n_s-1), float64."""
    k = np.asarray(k, dtype=np.float64)
    return A_s * np.power(k[None, :] / K_PIVOT, (p.n_s[:, None] - 1.0))


def emulator_features(p: ModelParams, A_s: float = A_S) -> np.ndarray:
    """[M, 9] float32 features of the emulator: (tau*, sigma, r_s, cos phi,
    sin phi, k_D, b, n_s, ln(1e10 A_s))."""
    M = p.M
    f = np.empty((M, 9), dtype=np.float64)
    f[:, 0] = p.tau_star
    f[:, 1] = p.sigma
    f[:, 2] = p.r_s
    f[:, 3] = np.cos(p.phi)
    f[:, 4] = np.sin(p.phi)
    f[:, 5] = p.k_D
    f[:, 6] = p.b
    f[:, 7] = p.n_s
    f[:, 8] = math.log(1e10 * A_s)
    return f.astype(np.float32)


def params_from_features(f) -> ModelParams:
    """Inverse of emulator_features (phi from atan2), in float64."""
    f = np.asarray(f, dtype=np.float64)
    return ModelParams(tau_star=f[:, 0].copy(), sigma=f[:, 1].copy(), r_s=f[:, 2].copy(),
                       phi=np.arctan2(f[:, 4], f[:, 3]), k_D=f[:, 5].copy(), b=f[:, 6].copy(), n_s=f[:, 7].copy())
