"""GPU parity of the E-mode polarisation path (Eq. 3 on the plain FP64 / FP32
kernels) and of the cross spectra C^EE, C^TE (Eq. 1 with X, Y in {T, E})
against the FP64 oracle, through the C ABI.

Tolerances as for temperature: Delta_E on the scale of the largest |Delta_E|
of its model (it crosses zero), 1e-11 for PLAIN64 and 1e-5 for PLAIN32;
C^EE relative per multipole, 1e-10 / 1e-5; C^TE crosses zero, so it is
compared on the Cauchy-Schwarz scale sqrt(C^TT C^EE) of its multipole."""
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


def small_workload(lmin=2, lmax=400, nk=40, ntau=300, M=3):
    return synth.Workload("small", synth.log_grid(1e-4, 0.3, nk), synth.uniform_grid(200.0, 14000.0, ntau),
                          14000.0, lmin, lmax, M)


def pol_inputs(wl, seed):
    """Temperature and polarisation sources of the synthetic family, with a
    random polarisation term on the last tau nodes so that the x = 0 node
    (tau = tau0 ends the uniform grid) carries weight."""
    p = synth.model_params(wl.M, seed=seed)
    ST = synth.sources(wl.k, wl.tau, p)
    SP = synth.sources_pol(wl.k, wl.tau, p)
    rng = np.random.default_rng(seed)
    SP[:, :, -3:] += 0.01 * rng.normal(size=SP[:, :, -3:].shape)
    return ST, SP, synth.primordial(wl.k, p)


def run(wl, ST, SP, P, mode):
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, mode)
    dt = torch.float64 if mode == gcamb.PLAIN64 else torch.float32
    DT = gcamb.los_transfer(g, dev(ST, dt), mode)
    DE = gcamb.los_transfer_e(g, dev(SP, dt), mode)
    Pd = dev(P)
    out = dict(DE=DE.cpu().numpy().astype(np.float64),
               EE=gcamb.cl_cross(g, DE, DE, Pd).cpu().numpy(),
               TE=gcamb.cl_cross(g, DT, DE, Pd).cpu().numpy(),
               TT=gcamb.cl(g, DT, Pd).cpu().numpy())
    gcamb.sync()
    return out, g


def reference(orc, wl, ST, SP, P):
    DT, TT = orc.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, ST, P)
    DE = orc.los_e(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, SP)
    return dict(DE=DE, TT=TT, EE=orc.cl_cross(wl.k, DE, DE, P), TE=orc.cl_cross(wl.k, DT, DE, P))


def check(out, ref, M, tol_d, tol_c):
    scale = np.abs(ref["DE"]).reshape(M, -1).max(axis=1)[:, None, None] + 1e-300
    assert np.all(np.abs(out["DE"] - ref["DE"]) <= tol_d * scale)
    ee = ref["EE"]
    nz = ee > 0
    assert np.all(np.abs(out["EE"][nz] - ee[nz]) <= tol_c * ee[nz])
    assert np.all(out["EE"][~nz] == 0)
    cs = np.sqrt(ref["TT"] * ee)
    assert np.all(np.abs(out["TE"] - ref["TE"]) <= tol_c * cs + 1e-300)


@pytest.mark.parametrize("lmin,lmax,nk,ntau,M", [
    (2, 400, 40, 300, 3),     # several l-tiles, ragged last tile and tau-block
    (0, 130, 7, 50, 1),       # lmin = 0 (E vanishes at l < 2), tile boundary at 128
    (2, 2, 1, 1, 2),          # degenerate: one k, one tau node (x = 0, zero weight), one l
    (5, 260, 25, 129, 5),     # lmin > 2, M not a multiple of the source chunk
])
def test_los_e_plain64_matches_oracle(orc, lmin, lmax, nk, ntau, M):
    wl = small_workload(lmin, lmax, nk, ntau, M)
    ST, SP, P = pol_inputs(wl, seed=11)
    out, _ = run(wl, ST, SP, P, gcamb.PLAIN64)
    check(out, reference(orc, wl, ST, SP, P), M, 1e-11, 1e-10)


def test_los_e_plain32_matches_oracle(orc):
    wl = small_workload()
    ST, SP, P = pol_inputs(wl, seed=12)
    ST, SP = ST.astype(np.float32), SP.astype(np.float32)
    out, _ = run(wl, ST, SP, P, gcamb.PLAIN32)
    ref = reference(orc, wl, ST.astype(np.float64), SP.astype(np.float64), P)
    check(out, ref, wl.M, 1e-5, 1e-5)


def test_x0_node_gives_the_l2_limit(orc):
    """A source only at tau = tau0: Delta_E = w S_P eps_l(0) = w S_P sqrt(24)/15 at
    l = 2 and 0 above; nodes at tiny x near tau0 take the same limit."""
    k = synth.log_grid(1e-4, 0.3, 9)
    tau = np.array([200.0, 5000.0, 13999.0, 14000.0 - 1e-4, 14000.0 - 1e-9, 14000.0])
    wl = synth.Workload("x0", k, tau, 14000.0, 2, 40, 1)
    w = orc.trapz_weights(tau)
    g = gcamb.grid_create(k, tau, 14000.0, 2, 40)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    SP = np.zeros((1, k.size, tau.size))
    SP[0, :, -1] = 2.0
    DE = gcamb.los_transfer_e(g, dev(SP), gcamb.PLAIN64).cpu().numpy()[0]
    assert np.allclose(DE[:, 0], w[-1] * 2.0 * np.sqrt(24.0) / 15.0, rtol=1e-14, atol=0)
    assert np.all(DE[:, 1:] == 0.0)
    # every node of the grid, tiny x (< 1e-12) included
    rng = np.random.default_rng(13)
    SP = rng.normal(size=(1, k.size, tau.size))
    DE = gcamb.los_transfer_e(g, dev(SP), gcamb.PLAIN64).cpu().numpy()
    ref = orc.los_e(k, tau, 14000.0, 2, 40, SP)
    scale = np.abs(ref).max()
    assert np.abs(DE - ref).max() <= 1e-11 * scale, np.abs(DE - ref).max() / scale
    gcamb.sync()


def test_delta_source_reproduces_eps(orc):
    wl = small_workload(2, 300, 12, 64, 1)
    w = orc.trapz_weights(wl.tau)
    istar = 20
    SP = np.zeros((1, wl.nk, wl.ntau))
    SP[0, :, istar] = 1.0 / w[istar]
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    DE = gcamb.los_transfer_e(g, dev(SP), gcamb.PLAIN64).cpu().numpy()[0]
    gcamb.sync()
    for q in range(wl.nk):
        x = wl.k[q] * (wl.tau0 - wl.tau[istar])
        ref = orc.eps(np.array([x]), wl.lmax)[0, 2:]
        big = np.abs(ref) > 1e-25 * np.abs(ref).max()
        assert np.allclose(DE[q][big], ref[big], rtol=1e-12, atol=0)
        assert np.all(np.abs(DE[q][~big]) <= 1e-24 * np.abs(ref).max())


def test_plain_lmax500_full_size_ee_te(orc):
    """The 1-model, l_max = 500 workload at its full size: C^EE and C^TE from
    the synthetic polarisation source, FP64 and FP32."""
    wl = synth.workload("plain_lmax500")
    p = synth.model_params(1, seed=0)
    ST = synth.sources(wl.k, wl.tau, p)
    SP = synth.sources_pol(wl.k, wl.tau, p)
    P = synth.primordial(wl.k, p)
    ref = reference(orc, wl, ST, SP, P)
    out, _ = run(wl, ST, SP, P, gcamb.PLAIN64)
    check(out, ref, 1, 1e-11, 1e-10)
    ST32, SP32 = ST.astype(np.float32), SP.astype(np.float32)
    out, _ = run(wl, ST32, SP32, P, gcamb.PLAIN32)
    check(out, reference(orc, wl, ST32.astype(np.float64), SP32.astype(np.float64), P), 1, 1e-5, 1e-5)


def test_cl_cross_auto_is_cl_and_symmetric():
    wl = small_workload()
    ST, SP, P = pol_inputs(wl, seed=14)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    DT = gcamb.los_transfer(g, dev(ST), gcamb.PLAIN64)
    DE = gcamb.los_transfer_e(g, dev(SP), gcamb.PLAIN64)
    Pd = dev(P)
    tt = gcamb.cl(g, DT, Pd).cpu().numpy()
    assert np.array_equal(gcamb.cl_cross(g, DT, DT, Pd).cpu().numpy(), tt)
    assert np.array_equal(gcamb.cl_cross(g, DT, DE, Pd).cpu().numpy(), gcamb.cl_cross(g, DE, DT, Pd).cpu().numpy())
    gcamb.sync()


def test_state_and_argument_errors():
    wl = small_workload()
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    SP = torch.zeros((1, wl.nk, wl.ntau), dtype=torch.float64, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_transfer_e(g, SP, gcamb.PLAIN64)
    assert ei.value.code == gcamb.ESTATE
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_transfer_e(g, SP.float(), gcamb.BF16X3)
    assert ei.value.code == gcamb.EINVAL
    assert gcamb.lib().gcamb_los_transfer_e(g.handle, None, 0, gcamb.PLAIN64, None, None) == gcamb.OK
    D = torch.zeros((1, wl.nk, wl.nl), dtype=torch.float64, device="cuda")
    P = torch.zeros((1, wl.nk), dtype=torch.float64, device="cuda")
    C = torch.zeros((1, wl.nl), dtype=torch.float64, device="cuda")
    assert gcamb.lib().gcamb_cl_cross(g.handle, D.data_ptr(), D.data_ptr(), 7, P.data_ptr(), 1, C.data_ptr(),
                                      None) == gcamb.EINVAL
    assert gcamb.lib().gcamb_cl_cross(g.handle, None, D.data_ptr(), gcamb.F64, P.data_ptr(), 1, C.data_ptr(),
                                      None) == gcamb.EINVAL
    gcamb.sync()
