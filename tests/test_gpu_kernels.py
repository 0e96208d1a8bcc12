"""GPU parity of kernel grids (gcamb_grid_set_kernel: the table holds
c_l j_l/x^2, the tensor e_l or b_l instead of j_l) against the FP64 oracle,
through the C ABI: the plain FP64 projection and the batched BF16X3
tensor-core path (tensor TT, EE, BB from one kernel grid per field).

Bars: delta sources reproduce the oracle's kernels to 1e-12 of their largest
value; PLAIN64 transfer functions within 1e-11 of their scale; BF16X3 C_l
within the split-product bound: the table holds each kernel value within
2^-16, so with A(k, l) = sum_i w_i |S| |kernel_l| the transfer function is
within (3 2^-16 + ntau 2^-24) A and
  |dC_l| <= (3 2^-16 + ntau 2^-24) 4 pi sum_k w_k P 2 |Delta| A."""
import numpy as np
import pytest

from paper_2509_25110_gb300 import build, gcamb, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KERNELS = {"EPS": gcamb.KERNEL_EPS, "E": gcamb.KERNEL_TENSOR_E, "B": gcamb.KERNEL_TENSOR_B}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gcamb.lib()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def kgrid(k, tau, lmin, lmax, kern):
    g = gcamb.grid_create(k, tau, 14000.0, lmin, lmax)
    return gcamb.grid_set_kernel(g, kern)


@pytest.mark.parametrize("name", ["EPS", "E", "B"])
def test_delta_source_gives_the_kernel(orc, name):
    k = synth.log_grid(1e-4, 0.3, 12)
    tau = synth.uniform_grid(200.0, 14000.0, 64)
    g = kgrid(k, tau, 2, 300, KERNELS[name])
    gcamb.bessel_table(g, gcamb.PLAIN64)
    w = orc.trapz_weights(tau)
    i = 20
    S = np.zeros((1, k.size, tau.size))
    S[0, :, i] = 1.0 / w[i]
    D = gcamb.los_transfer(g, dev(S), gcamb.PLAIN64).cpu().numpy()[0]
    gcamb.sync()
    t, e, b = orc.tensor_kernels(k * (14000.0 - tau[i]), 300)
    ref = {"EPS": t, "E": e, "B": b}[name][:, 2:]
    assert np.abs(D - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("lmin,lmax,nk,ntau", [(2, 400, 40, 300), (0, 130, 7, 50), (5, 260, 25, 129)])
def test_plain64_kernel_grids_match_the_oracle(orc, lmin, lmax, nk, ntau):
    k = synth.log_grid(1e-4, 0.3, nk)
    tau = synth.uniform_grid(200.0, 14000.0, ntau)
    p = synth.model_params(3, seed=71)
    ST, SP = synth.sources_tensor(k, tau, p)
    rng = np.random.default_rng(71)
    SP[:, :, -3:] += 0.01 * rng.normal(size=SP[:, :, -3:].shape)  # weight at x = 0
    DT, DE, DB = orc.los_tensor(k, tau, 14000.0, lmin, lmax, ST, SP)
    for name, S, ref in (("EPS", ST, DT), ("E", SP, DE), ("B", SP, DB)):
        g = kgrid(k, tau, lmin, lmax, KERNELS[name])
        gcamb.bessel_table(g, gcamb.PLAIN64)
        D = gcamb.los_transfer(g, dev(S), gcamb.PLAIN64).cpu().numpy()
        gcamb.sync()
        scale = np.abs(ref).reshape(3, -1).max(axis=1)[:, None, None]
        assert np.all(np.abs(D - ref) <= 1e-11 * scale), name


def test_tiny_x_nodes(orc):
    k = synth.log_grid(1e-4, 0.3, 9)
    tau = np.array([200.0, 5000.0, 13999.0, 14000.0 - 1e-4, 14000.0 - 1e-9, 14000.0])
    rng = np.random.default_rng(72)
    S = rng.normal(size=(2, k.size, tau.size))
    refs = orc.los_tensor(k, tau, 14000.0, 2, 40, S, S)
    for name, ref in zip(("EPS", "E", "B"), refs):
        g = kgrid(k, tau, 2, 40, KERNELS[name])
        gcamb.bessel_table(g, gcamb.PLAIN64)
        D = gcamb.los_transfer(g, dev(S), gcamb.PLAIN64).cpu().numpy()
        gcamb.sync()
        assert np.abs(D - ref).max() <= 1e-11 * np.abs(ref).max(), name


def test_batched_tensor_spectra(orc):
    k = synth.log_grid(1e-4, 3000.0 / 14000.0, 120)
    tau = synth.uniform_grid(200.0, 14000.0, 400)
    M, lmax = 70, 800
    p = synth.model_params(M, seed=73)
    ST, SP = synth.sources_tensor(k, tau, p, np.float32)
    P = synth.primordial_tensor(k, p)
    sub = [0, 35, 69]
    DT, DE, DB = orc.los_tensor(k, tau, 14000.0, 2, lmax, ST[sub].astype(np.float64), SP[sub].astype(np.float64))
    w = orc.trapz_weights(tau)
    x = (k[:, None] * (14000.0 - tau[None, :])).ravel()
    kt, ke, kb = (np.abs(a).reshape(k.size, tau.size, -1)[:, :, 2:] for a in orc.tensor_kernels(x, lmax))
    f = 4.0 * np.pi * orc.lnk_weights(k)[None, :, None] * P[sub][:, :, None]
    u = 3 * 2.0 ** -16 + tau.size * 2.0 ** -24
    for name, S, Dr, K in (("EPS", ST, DT, kt), ("E", SP, DE, ke), ("B", SP, DB, kb)):
        g = kgrid(k, tau, 2, lmax, KERNELS[name])
        gcamb.bessel_table(g, gcamb.BF16X3)
        C = gcamb.los_cl(g, dev(S, torch.float32), dev(P), gcamb.BF16X3).cpu().numpy()[sub]
        gcamb.sync()
        Cr = orc.cl_cross(k, Dr, Dr, P[sub])
        A = np.einsum("mki,kil->mkl", np.abs(S[sub].astype(np.float64)) * w, K)
        bound = u * (f * 2 * np.abs(Dr) * A).sum(axis=1)
        assert np.all(np.abs(C - Cr) <= bound), (name, np.max(np.abs(C - Cr) / bound))


def test_kernel_grid_rules():
    k = synth.log_grid(1e-4, 0.3, 10)
    tau = synth.uniform_grid(200.0, 14000.0, 64)
    g = gcamb.grid_create(k, tau, 14000.0, 2, 100)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    with pytest.raises(gcamb.GcambError) as ei:  # a table already exists
        gcamb.grid_set_kernel(g, gcamb.KERNEL_TENSOR_B)
    assert ei.value.code == gcamb.ESTATE
    g2 = kgrid(k, tau, 2, 100, gcamb.KERNEL_EPS)
    gcamb.bessel_table(g2, gcamb.PLAIN64)
    S = torch.zeros((1, k.size, tau.size), dtype=torch.float64, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_transfer_e(g2, S, gcamb.PLAIN64)
    assert ei.value.code == gcamb.EUNSUPPORTED
    gc = gcamb.grid_create_curved(k, tau, 14000.0, 2, 100, -1e-8)
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.grid_set_kernel(gc, gcamb.KERNEL_EPS)
    assert ei.value.code == gcamb.EUNSUPPORTED
    gcamb.sync()


def test_pair_gives_tensor_te(orc):
    """gcamb_los_cl_pair on the tensor T and E kernel grids: C^TT, C^EE and
    C^TE of the tensor sources from one launch, against the oracle (the split
    bound, C^TE with |Delta_T| A_E + |Delta_E| A_T)."""
    k = synth.log_grid(1e-4, 3000.0 / 14000.0, 120)
    tau = synth.uniform_grid(200.0, 14000.0, 400)
    M, lmax = 70, 800
    p = synth.model_params(M, seed=74)
    ST, SP = synth.sources_tensor(k, tau, p, np.float32)
    P = synth.primordial_tensor(k, p)
    gT = kgrid(k, tau, 2, lmax, gcamb.KERNEL_EPS)
    gE = kgrid(k, tau, 2, lmax, gcamb.KERNEL_TENSOR_E)
    gcamb.bessel_table(gT, gcamb.BF16X3)
    gcamb.bessel_table(gE, gcamb.BF16X3)
    tt, ee, te = (x.cpu().numpy() for x in gcamb.los_cl_pair(gT, gE, dev(ST, torch.float32), dev(SP, torch.float32),
                                                               dev(P)))
    gcamb.sync()
    sub = [0, 35, 69]
    DT, DE, _ = orc.los_tensor(k, tau, 14000.0, 2, lmax, ST[sub].astype(np.float64), SP[sub].astype(np.float64))
    w = orc.trapz_weights(tau)
    x = (k[:, None] * (14000.0 - tau[None, :])).ravel()
    kt, ke, _ = (np.abs(a).reshape(k.size, tau.size, -1)[:, :, 2:] for a in orc.tensor_kernels(x, lmax))
    AT = np.einsum("mki,kil->mkl", np.abs(ST[sub].astype(np.float64)) * w, kt)
    AE = np.einsum("mki,kil->mkl", np.abs(SP[sub].astype(np.float64)) * w, ke)
    f = 4.0 * np.pi * orc.lnk_weights(k)[None, :, None] * P[sub][:, :, None]
    u = 3 * 2.0 ** -16 + tau.size * 2.0 ** -24
    for name, c, DX, DY, AX, AY in (("TT", tt, DT, DT, AT, AT), ("EE", ee, DE, DE, AE, AE), ("TE", te, DT, DE, AT, AE)):
        ref = orc.cl_cross(k, DX, DY, P[sub])
        bound = u * (f * (np.abs(DX) * AY + np.abs(DY) * AX)).sum(axis=1)
        assert np.all(np.abs(c[sub] - ref) <= bound), (name, np.max(np.abs(c[sub] - ref) / bound))
    # grids of another layout are rejected
    gB = kgrid(k, tau, 2, lmax - 1, gcamb.KERNEL_TENSOR_B)
    gcamb.bessel_table(gB, gcamb.BF16X3)
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl_pair(gT, gB, dev(ST, torch.float32), dev(SP, torch.float32), dev(P))
    assert ei.value.code == gcamb.EINVAL
    gcamb.sync()
