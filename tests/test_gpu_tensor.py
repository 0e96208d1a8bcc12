"""GPU parity of the tensor-mode projection (gcamb_los_transfer_tensor:
kernels t_l, e_l, b_l on the plain FP64 / FP32 kernels) and of its spectra
against the FP64 oracle, through the C ABI.

Tolerances as for the scalar paths: transfer functions on the scale of the
largest |Delta| of their model and field (they cross zero), 1e-11 for
PLAIN64 and 1e-5 for PLAIN32; C^TT, C^EE, C^BB relative per multipole,
1e-10 / 1e-5; C^TE on the Cauchy-Schwarz scale sqrt(C^TT C^EE).

PLAIN32 C^BB and C^TE: b_l = 2 j_(l-1) - 2 (l-1) j_l / x cancels near the
turning point x ~ l, which magnifies the FP32 rounding of the table's j_l
(1.6e-5 relative on C^BB of the 300-node grid).  Their bar is the derived one:
each FP32 tau-sum is within (ntau + 2) 2^-24 of its sum of |terms|, so with
A_X(k, l) = sum_i w_i |S_X| (sum of |components| of the kernel),
  |dC^XY_l| <= (ntau + 2) 2^-24 4 pi sum_k w_k P (|Delta_X| A_Y + |Delta_Y| A_X)."""
import numpy as np
import pytest

from paper_2509_25110_gb300 import build, gcamb, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gcamb.lib()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def workload(lmin, lmax, nk, ntau, M):
    return synth.Workload("small", synth.log_grid(1e-4, 0.3, nk), synth.uniform_grid(200.0, 14000.0, ntau),
                          14000.0, lmin, lmax, M)


def inputs(wl, seed):
    """Tensor sources of the synthetic family plus a random term on the last
    tau nodes (the uniform grid ends at tau0: x = 0 there)."""
    p = synth.model_params(wl.M, seed=seed)
    ST, SP = synth.sources_tensor(wl.k, wl.tau, p)
    rng = np.random.default_rng(seed)
    ST[:, :, -3:] += 0.01 * rng.normal(size=ST[:, :, -3:].shape)
    SP[:, :, -3:] += 0.01 * rng.normal(size=SP[:, :, -3:].shape)
    return ST, SP, synth.primordial_tensor(wl.k, p)


def run(wl, ST, SP, P, mode):
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, mode)
    dt = torch.float64 if mode == gcamb.PLAIN64 else torch.float32
    DT, DE, DB = gcamb.los_transfer_tensor(g, dev(ST, dt), dev(SP, dt), mode)
    Pd = dev(P)
    out = dict(D=[x.cpu().numpy().astype(np.float64) for x in (DT, DE, DB)],
               TT=gcamb.cl(g, DT, Pd).cpu().numpy(), EE=gcamb.cl(g, DE, Pd).cpu().numpy(),
               BB=gcamb.cl(g, DB, Pd).cpu().numpy(), TE=gcamb.cl_cross(g, DT, DE, Pd).cpu().numpy())
    gcamb.sync()
    return out


def reference(orc, wl, ST, SP, P):
    DT, DE, DB = orc.los_tensor(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, ST, SP)
    return dict(D=[DT, DE, DB], TT=orc.cl_cross(wl.k, DT, DT, P), EE=orc.cl_cross(wl.k, DE, DE, P),
                BB=orc.cl_cross(wl.k, DB, DB, P), TE=orc.cl_cross(wl.k, DT, DE, P))


def check(out, ref, M, tol_d, tol_c):
    for d, r in zip(out["D"], ref["D"]):
        scale = np.abs(r).reshape(M, -1).max(axis=1)[:, None, None] + 1e-300
        assert np.all(np.abs(d - r) <= tol_d * scale), np.max(np.abs(d - r) / scale)
    for key in ("TT", "EE", "BB"):
        c, r = out[key], ref[key]
        nz = r > 0
        assert np.all(np.abs(c[nz] - r[nz]) <= tol_c * r[nz]), (key, np.max(np.abs(c[nz] / r[nz] - 1)))
        assert np.all(c[~nz] == 0), key
    cs = np.sqrt(ref["TT"] * ref["EE"])
    assert np.all(np.abs(out["TE"] - ref["TE"]) <= tol_c * cs), np.max(np.abs(out["TE"] - ref["TE"]) / (cs + 1e-300))


@pytest.mark.parametrize("lmin,lmax,nk,ntau,M", [
    (2, 400, 40, 300, 3),     # several l-tiles (row l-1 across a tile boundary), ragged tiles
    (0, 130, 7, 50, 1),       # lmin = 0 (zero below l = 2), tile boundary at 128
    (1, 200, 10, 64, 2),      # lmin = 1: row l-1 of l = 2 stored
    (5, 260, 25, 129, 5),     # lmin > 2: row l-1 of the first multipole from the recurrence
    (2, 3, 3, 20, 1),         # two multipoles only
])
def test_tensor_plain64_matches_oracle(orc, lmin, lmax, nk, ntau, M):
    wl = workload(lmin, lmax, nk, ntau, M)
    ST, SP, P = inputs(wl, seed=41)
    check(run(wl, ST, SP, P, gcamb.PLAIN64), reference(orc, wl, ST, SP, P), M, 1e-11, 1e-10)


def abs_components(orc, wl, ST, SP):
    """A_T, A_E, A_B [M][nk][nl]: sum_i w_i |S| (sum of |components| of t_l, e_l, b_l)."""
    w = orc.trapz_weights(wl.tau)
    x = (wl.k[:, None] * (wl.tau0 - wl.tau[None, :])).ravel()
    j = orc.sph_bessel(wl.lmax, x).reshape(wl.nk, wl.ntau, -1)
    l = np.arange(wl.lmax + 1)[None, None, :]
    small = x.reshape(wl.nk, wl.ntau, 1) < 1e-6
    xx = np.where(small, 1.0, x.reshape(wl.nk, wl.ntau, 1))
    jm = np.concatenate([np.zeros_like(j[:, :, :1]), j[:, :, :-1]], axis=2)  # j_(l-1)
    c = np.sqrt(np.maximum((l + 2.0) * (l + 1.0) * l * (l - 1.0), 0.0))
    kt = c * np.abs(j) / xx ** 2
    ke = l * (l - 1.0) * np.abs(j) / xx ** 2 + 2 * np.abs(j) + 2 * np.abs(jm) / xx
    kb = 2 * np.abs(jm) + 2 * (l - 1.0) * np.abs(j) / xx
    # at tiny x (x = 0 included) the kernels' own size: nothing cancels there
    t0, e0, b0 = (np.abs(a).reshape(wl.nk, wl.ntau, -1) for a in orc.tensor_kernels(x, wl.lmax))
    kt, ke, kb = (np.where(small, a0, a) for a, a0 in ((kt, t0), (ke, e0), (kb, b0)))
    sl = slice(wl.lmin, wl.lmax + 1)
    return [np.einsum("mki,kil->mkl", np.abs(S) * w, K[:, :, sl]) for S, K in ((ST, kt), (SP, ke), (SP, kb))]


def test_tensor_plain32_matches_oracle(orc):
    wl = workload(2, 400, 40, 300, 3)
    ST, SP, P = inputs(wl, seed=42)
    ST, SP = ST.astype(np.float32), SP.astype(np.float32)
    out = run(wl, ST, SP, P, gcamb.PLAIN32)
    ref = reference(orc, wl, ST.astype(np.float64), SP.astype(np.float64), P)
    for d, r in zip(out["D"], ref["D"]):
        scale = np.abs(r).reshape(wl.M, -1).max(axis=1)[:, None, None]
        assert np.all(np.abs(d - r) <= 1e-5 * scale)
    for key in ("TT", "EE"):
        assert np.all(np.abs(out[key] - ref[key]) <= 1e-5 * ref[key]), key
    AT, AE, AB = abs_components(orc, wl, ST.astype(np.float64), SP.astype(np.float64))
    DT, DE, DB = ref["D"]
    f = 4.0 * np.pi * orc.lnk_weights(wl.k)[None, :, None] * P[:, :, None]
    u = (wl.ntau + 2) * 2.0 ** -24
    for key, DX, DY, AX, AY in (("BB", DB, DB, AB, AB), ("TE", DT, DE, AT, AE)):
        bound = u * (f * (np.abs(DX) * AY + np.abs(DY) * AX)).sum(axis=1)
        err = np.abs(out[key] - ref[key])
        assert np.all(err <= bound), (key, np.max(err / bound))


def test_tensor_tiny_x_nodes(orc):
    """Nodes at x = 0 and at x < 1e-12 near tau0 take the series of the kernels."""
    k = synth.log_grid(1e-4, 0.3, 9)
    tau = np.array([200.0, 5000.0, 13999.0, 14000.0 - 1e-4, 14000.0 - 1e-9, 14000.0])
    wl = synth.Workload("x0", k, tau, 14000.0, 2, 40, 2)
    rng = np.random.default_rng(43)
    ST = rng.normal(size=(2, k.size, tau.size))
    SP = rng.normal(size=(2, k.size, tau.size))
    P = np.full((2, k.size), 2e-10)
    check(run(wl, ST, SP, P, gcamb.PLAIN64), reference(orc, wl, ST, SP, P), 2, 1e-11, 1e-10)


def test_delta_source_reproduces_the_kernels(orc):
    wl = workload(2, 300, 12, 64, 1)
    w = orc.trapz_weights(wl.tau)
    istar = 20
    S = np.zeros((1, wl.nk, wl.ntau))
    S[0, :, istar] = 1.0 / w[istar]
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    D = [x.cpu().numpy()[0] for x in gcamb.los_transfer_tensor(g, dev(S), dev(S), gcamb.PLAIN64)]
    gcamb.sync()
    x = wl.k * (wl.tau0 - wl.tau[istar])
    refs = orc.tensor_kernels(x, wl.lmax)
    for d, r in zip(D, refs):
        r = r[:, 2:]
        assert np.abs(d - r).max() <= 1e-12 * np.abs(r).max()


def test_tensor_lmax1500_full_size(orc):
    """The tensor workload of the paper's runs (l <= 1500, k tau0 <= 3000) at
    its full size, FP64: Delta at sampled k against the oracle, spectra
    against the oracle's Eq. (1) sums of those transfer functions."""
    wl = synth.workload("tensor_lmax1500")
    p = synth.model_params(1, seed=0)
    ST, SP = synth.sources_tensor(wl.k, wl.tau, p)
    P = synth.primordial_tensor(wl.k, p)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    D = [x.cpu().numpy() for x in gcamb.los_transfer_tensor(g, dev(ST), dev(SP), gcamb.PLAIN64)]
    gcamb.sync()
    qs = np.array([0, 300, 600, 900, 999])
    wt, _ = gcamb.grid_weights(g)
    R = orc.los_tensor(wl.k[qs], wl.tau, wl.tau0, wl.lmin, wl.lmax, ST[:, qs], SP[:, qs], wtau=wt)
    for d, r in zip(D, R):
        assert np.abs(d[:, qs] - r).max() <= 1e-11 * np.abs(r).max()


def test_tensor_errors():
    wl = workload(2, 100, 10, 64, 1)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    S = torch.zeros((1, wl.nk, wl.ntau), dtype=torch.float64, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_transfer_tensor(g, S, S, gcamb.PLAIN64)
    assert ei.value.code == gcamb.ESTATE
    gcamb.bessel_table(g, gcamb.PLAIN64)
    D = torch.zeros((1, wl.nk, wl.nl), dtype=torch.float64, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_transfer_tensor(g, S, S, gcamb.PLAIN64, out=(D, D, torch.zeros_like(D)))
    assert ei.value.code == gcamb.EINVAL
    g1 = gcamb.grid_create(wl.k, wl.tau, wl.tau0, 2, 2)
    gcamb.bessel_table(g1, gcamb.PLAIN64)
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_transfer_tensor(g1, S, S, gcamb.PLAIN64)
    assert ei.value.code == gcamb.EINVAL
    gcamb.sync()
