"""GPU parity on grids of sampled multipoles (gcamb_grid_create_lsampled):
every path computes the listed rows only, and gcamb_cl_interp fills the rest
by the natural cubic spline in l of l (l+1) C_l.

The sampled rows are compared with the dense FP64 oracle at the same
multipoles, with the bars of the dense grids (PLAIN64 1e-10, BF16X3 the
derived split bound); the interpolation with the oracle's own spline of the
same samples (oracle/interp.py) to 1e-12."""
import numpy as np
import pytest

from oracle import interp as ointerp
from paper_2509_25110_gb300 import build, gcamb, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SPLIT_TOL = 6 * 2.0 ** -16


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gcamb.lib()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def setup(lmax=700, nk=60, ntau=300, M=3, boost=1.0, seed=51):
    k = synth.log_grid(1e-4, 0.3, nk)
    tau = synth.uniform_grid(200.0, 14000.0, ntau)
    lv = gcamb.l_sampling(2, lmax, boost)
    p = synth.model_params(M, seed=seed)
    return k, tau, lv, p


def test_plain64_and_emode_on_sampled_rows(orc):
    k, tau, lv, p = setup()
    S, SP = synth.sources(k, tau, p), synth.sources_pol(k, tau, p)
    P = synth.primordial(k, p)
    g = gcamb.grid_create_lsampled(k, tau, 14000.0, lv)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    D = gcamb.los_transfer(g, dev(S), gcamb.PLAIN64)
    C = gcamb.cl(g, D, dev(P)).cpu().numpy()
    DE = gcamb.los_transfer_e(g, dev(SP), gcamb.PLAIN64)
    EE = gcamb.cl_cross(g, DE, DE, dev(P)).cpu().numpy()
    gcamb.sync()
    Dr, Cr = orc.los_cl(k, tau, 14000.0, 2, int(lv[-1]), S, P)
    DEr = orc.los_e(k, tau, 14000.0, 2, int(lv[-1]), SP)
    EEr = orc.cl_cross(k, DEr, DEr, P)
    rows = lv - 2
    assert np.all(np.abs(C - Cr[:, rows]) <= 1e-10 * Cr[:, rows])
    assert np.all(np.abs(EE - EEr[:, rows]) <= 1e-10 * EEr[:, rows])
    scale = np.abs(Dr).max()
    assert np.abs(D.cpu().numpy() - Dr[:, :, rows]).max() <= 1e-11 * scale


def test_batched_and_te_on_sampled_rows(orc):
    k, tau, lv, p = setup(lmax=900, nk=80, ntau=400, M=40, boost=0.5)
    ST = synth.sources(k, tau, p, np.float32)
    SP = synth.sources_pol(k, tau, p).astype(np.float32)
    P = synth.primordial(k, p)
    g = gcamb.grid_create_lsampled(k, tau, 14000.0, lv)
    gcamb.bessel_table(g, gcamb.BF16X3)
    C = gcamb.los_cl(g, dev(ST, torch.float32), dev(P), gcamb.BF16X3).cpu().numpy()
    tt, ee, te = (x.cpu().numpy() for x in gcamb.los_cl_te(g, dev(ST, torch.float32), dev(SP, torch.float32), dev(P)))
    gcamb.sync()
    lmax = int(lv[-1])
    DT, TT = orc.los_cl(k, tau, 14000.0, 2, lmax, ST.astype(np.float64), P)
    DE = orc.los_e(k, tau, 14000.0, 2, lmax, SP.astype(np.float64))
    EE, TE = orc.cl_cross(k, DE, DE, P), orc.cl_cross(k, DT, DE, P)
    rows = lv - 2
    assert np.abs(C / TT[:, rows] - 1).max() <= SPLIT_TOL
    assert np.abs(tt / TT[:, rows] - 1).max() <= SPLIT_TOL
    # EE and TE: the split-product bound with the sums of |terms| (E-mode
    # terms cancel on coarse grids), as for the dense TE tests
    w = orc.trapz_weights(tau)
    x = (k[:, None] * (14000.0 - tau[None, :])).ravel()
    AT = np.einsum("mki,kil->mkl", np.abs(ST.astype(np.float64)) * w,
                   np.abs(orc.sph_bessel(lmax, x)).reshape(k.size, tau.size, -1)[:, :, lv])
    AE = np.einsum("mki,kil->mkl", np.abs(SP.astype(np.float64)) * w,
                   np.abs(orc.eps(x, lmax)).reshape(k.size, tau.size, -1)[:, :, lv])
    f = 4.0 * np.pi * orc.lnk_weights(k)[None, :, None] * P[:, :, None]
    u = 3 * 2.0 ** -16 + tau.size * 2.0 ** -24
    DTs, DEs = DT[:, :, rows], DE[:, :, rows]
    assert np.all(np.abs(ee - EE[:, rows]) <= u * (f * 2 * np.abs(DEs) * AE).sum(axis=1))
    assert np.all(np.abs(te - TE[:, rows]) <= u * (f * (np.abs(DTs) * AE + np.abs(DEs) * AT)).sum(axis=1))


def test_cl_interp_matches_the_oracle_spline(orc):
    k, tau, lv, p = setup(lmax=1500, nk=60, ntau=300, M=4, boost=1.0)
    S = synth.sources(k, tau, p)
    P = synth.primordial(k, p)
    g = gcamb.grid_create_lsampled(k, tau, 14000.0, lv)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    Cs = gcamb.cl(g, gcamb.los_transfer(g, dev(S), gcamb.PLAIN64), dev(P))
    Cf = gcamb.cl_interp(g, Cs).cpu().numpy()
    Cs = Cs.cpu().numpy()
    gcamb.sync()
    l_all = np.arange(2, int(lv[-1]) + 1, dtype=np.float64)
    x = lv.astype(np.float64)
    y = x * (x + 1.0) * Cs
    ref = ointerp.natural_spline_eval(x, y, ointerp.natural_second_derivatives(x, y), l_all) / (l_all * (l_all + 1.0))
    assert np.abs(Cf / ref - 1).max() <= 1e-12
    assert np.array_equal(Cf[:, lv - 2], Cs)  # samples are copied


def test_tensor_rejects_sampled_grids():
    k, tau, lv, p = setup(lmax=100)
    g = gcamb.grid_create_lsampled(k, tau, 14000.0, lv)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    S = torch.zeros((1, g.nk, g.ntau), dtype=torch.float64, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_transfer_tensor(g, S, S, gcamb.PLAIN64)
    assert ei.value.code == gcamb.EUNSUPPORTED


@pytest.mark.parametrize("nl_keep", [120, 4100])
def test_cl_interp_shared_and_global_paths(nl_keep):
    """Up to 4000 samples the spline runs in shared memory, above that in two
    global-memory kernels; both against the oracle's spline of the same samples."""
    rng = np.random.default_rng(nl_keep)
    lmax = 4600
    keep = np.sort(rng.choice(np.arange(3, lmax), nl_keep - 2, replace=False))
    lv = np.concatenate([[2], keep, [lmax]]).astype(np.int32)
    k = synth.log_grid(1e-4, 0.3, 4)
    g = gcamb.grid_create_lsampled(k, synth.uniform_grid(200.0, 14000.0, 8), 14000.0, lv)
    Cs = np.exp(rng.normal(size=(3, lv.size))) * 1e-10
    Cf = gcamb.cl_interp(g, dev(Cs)).cpu().numpy()
    gcamb.sync()
    l_all = np.arange(2, lmax + 1, dtype=np.float64)
    x = lv.astype(np.float64)
    y = x * (x + 1.0) * Cs
    ref = ointerp.natural_spline_eval(x, y, ointerp.natural_second_derivatives(x, y), l_all) / (l_all * (l_all + 1.0))
    assert np.all(np.abs(Cf - ref) <= 1e-12 * np.abs(y).max(axis=1, keepdims=True) / (l_all * (l_all + 1.0)))
    assert np.array_equal(Cf[:, lv - 2], Cs)
