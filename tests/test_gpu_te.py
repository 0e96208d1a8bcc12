"""GPU parity of the batched temperature + E-mode path (gcamb_los_cl_te:
Eqs. 1-3 on the tensor cores, BF16X3) against the FP64 oracle, through the
C ABI.

The oracle is run on the FP32-rounded sources the kernel reads.

Small grids: the derived BF16X3 bound.  bf16 hi + lo carries each operand
within 2^-16 of itself, so a split product with lo*lo dropped is within
u = 3 * 2^-16 of the exact product; the FP32 tau-sum adds at most
ntau * 2^-24 of the sum of |terms|.  With A_X(k, l) = sum_i w_i |S_X| |kernel_l|
(the oracle's j_l or eps_l) the transfer function is within
(u + ntau 2^-24) A_X, and
  |dC^XY_l| <= (u + ntau 2^-24) 4 pi sum_k w_k P (|Delta_X| A_Y + |Delta_Y| A_X).
This is 6 * 2^-16 relative where the terms of Delta do not cancel, and more
where they do (coarse tau grids, the 1/x^2-weighted E-mode terms).
Full 256-model l_max = 2500 grid: 1e-5 relative (C^TT, C^EE), C^TE on the
Cauchy-Schwarz scale sqrt(C^TT C^EE) of its multipole (it crosses zero)."""
import numpy as np
import pytest

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


def workload(lmin, lmax, nk, ntau, M):
    return synth.Workload("small", synth.log_grid(1e-4, 0.3, nk), synth.uniform_grid(200.0, 14000.0, ntau),
                          14000.0, lmin, lmax, M)


def inputs(wl, seed, models=None):
    """FP32 temperature and polarisation sources of the synthetic family (the
    uniform tau grid ends at tau0: x = 0 there), with a random polarisation
    term on the last tau nodes so that the x = 0 node carries weight."""
    p = synth.model_params(wl.M, seed=seed)
    ST = synth.sources(wl.k, wl.tau, p, np.float32)
    SP = synth.sources_pol(wl.k, wl.tau, p)
    rng = np.random.default_rng(seed)
    SP[:, :, -3:] += 0.01 * rng.normal(size=SP[:, :, -3:].shape)
    return ST, SP.astype(np.float32), synth.primordial(wl.k, p)


def run_te(wl, ST, SP, P):
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, gcamb.BF16X3)
    tt, ee, te = gcamb.los_cl_te(g, dev(ST, torch.float32), dev(SP, torch.float32), dev(P))
    gcamb.sync()
    return tt.cpu().numpy(), ee.cpu().numpy(), te.cpu().numpy(), g


def oracle_te(orc, wl, ST, SP, P, want_delta=False):
    DT, TT = orc.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, ST.astype(np.float64), P)
    DE = orc.los_e(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, SP.astype(np.float64))
    ref = (TT, orc.cl_cross(wl.k, DE, DE, P), orc.cl_cross(wl.k, DT, DE, P))
    return (ref, DT, DE) if want_delta else ref


def abs_terms(orc, wl, S, kernel):
    """A[m][k][l] = sum_i w_i |S[m][k][i]| |kernel_l(k (tau0 - tau_i))|."""
    w = orc.trapz_weights(wl.tau)
    x = (wl.k[:, None] * (wl.tau0 - wl.tau[None, :])).ravel()
    K = np.abs(kernel(x)).reshape(wl.nk, wl.ntau, -1)[:, :, wl.lmin:wl.lmax + 1]
    return np.einsum("mki,kil->mkl", np.abs(S.astype(np.float64)) * w, K)


def check_bound(orc, wl, got, ST, SP, P):
    (TT, EE, TE), DT, DE = oracle_te(orc, wl, ST, SP, P, want_delta=True)
    AT = abs_terms(orc, wl, ST, lambda x: orc.sph_bessel(wl.lmax, x))
    AE = abs_terms(orc, wl, SP, lambda x: orc.eps(x, wl.lmax))
    f = 4.0 * np.pi * orc.lnk_weights(wl.k)[None, :, None] * P[:, :, None]
    u = 3 * 2.0 ** -16 + wl.ntau * 2.0 ** -24
    for name, c, ref, DX, DY, AX, AY in (("TT", got[0], TT, DT, DT, AT, AT), ("EE", got[1], EE, DE, DE, AE, AE),
                                         ("TE", got[2], TE, DT, DE, AT, AE)):
        bound = u * (f * (np.abs(DX) * AY + np.abs(DY) * AX)).sum(axis=1)
        err = np.abs(c - ref)
        assert np.all(err <= bound), (name, np.max(err / np.maximum(bound, 1e-300)))
    assert np.all(got[1][EE == 0] == 0) and np.all(got[2][EE == 0] == 0)


def check(got, ref, tol):
    tt, ee, te = got
    rtt, ree, rte = ref
    assert np.all(np.abs(tt - rtt) <= tol * rtt), np.max(np.abs(tt / rtt - 1))
    nz = ree > 0
    assert np.all(np.abs(ee[nz] - ree[nz]) <= tol * ree[nz]), np.max(np.abs(ee[nz] / ree[nz] - 1))
    assert np.all(ee[~nz] == 0) and np.all(te[~nz] == 0)
    cs = np.sqrt(rtt * ree)
    assert np.all(np.abs(te - rte) <= tol * cs), np.max(np.abs(te - rte)[nz] / cs[nz])


@pytest.mark.parametrize("lmin,lmax,nk,ntau,M", [
    (2, 400, 40, 300, 3),     # several l-tiles, ragged last tile and tau-block, one 32-model tile
    (0, 130, 7, 52, 1),       # lmin = 0 (E vanishes at l < 2), tile boundary at 128
    (2, 300, 30, 200, 40),    # 64-model tiles (128 operand rows), ragged model tile
    (5, 260, 25, 128, 70),    # lmin > 2 (no l = 2 tail), two model tiles
    (2, 2, 1, 4, 2),          # degenerate: one k, one l
])
def test_te_matches_oracle(orc, lmin, lmax, nk, ntau, M):
    wl = workload(lmin, lmax, nk, ntau, M)
    ST, SP, P = inputs(wl, seed=21)
    tt, ee, te, _ = run_te(wl, ST, SP, P)
    check_bound(orc, wl, (tt, ee, te), ST, SP, P)


def test_te_tiny_x_nodes(orc):
    """Nodes at x = 0 and x < 1e-12 (the l = 2 tail), nodes just above the cut."""
    k = synth.log_grid(1e-4, 0.3, 17)
    tau = np.array([200.0, 3000.0, 6000.0, 9000.0, 13999.0, 14000.0 - 1e-4, 14000.0 - 1e-9, 14000.0])
    wl = synth.Workload("x0", k, tau, 14000.0, 2, 60, 5)
    rng = np.random.default_rng(22)
    ST = rng.normal(size=(5, k.size, tau.size)).astype(np.float32)
    SP = rng.normal(size=(5, k.size, tau.size)).astype(np.float32)
    P = np.full((5, k.size), 2.1e-9)
    tt, ee, te, _ = run_te(wl, ST, SP, P)
    check_bound(orc, wl, (tt, ee, te), ST, SP, P)


def test_tt_agrees_with_the_temperature_path():
    wl = workload(2, 400, 40, 300, 50)
    ST, SP, P = inputs(wl, seed=23)
    tt, _, _, g = run_te(wl, ST, SP, P)
    ref = gcamb.los_cl(g, dev(ST, torch.float32), dev(P), gcamb.BF16X3).cpu().numpy()
    gcamb.sync()
    assert np.abs(tt / ref - 1).max() <= SPLIT_TOL


def test_te_deterministic_repeat():
    wl = workload(2, 400, 40, 300, 3)
    ST, SP, P = inputs(wl, seed=24)
    a = run_te(wl, ST, SP, P)
    b = run_te(wl, ST, SP, P)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


def test_te_full_grid_sampled(orc):
    """The 256-model, l_max = 2500 grid at its full size; three models checked
    against the oracle at every l."""
    wl = synth.workload("batched_lmax2500")
    p = synth.model_params(wl.M, seed=0)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, gcamb.BF16X3)
    ST = synth.sources_torch(wl.k, wl.tau, p, "cuda", torch.float32)
    SP = synth.sources_pol_torch(wl.k, wl.tau, p, "cuda", torch.float32)
    P = dev(synth.primordial(wl.k, p))
    tt, ee, te = gcamb.los_cl_te(g, ST, SP, P)
    gcamb.sync()
    ms = [0, 131, 255]
    sub = synth.Workload("sub", wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, len(ms))
    ref = oracle_te(orc, sub, ST[ms].cpu().numpy(), SP[ms].cpu().numpy(), P[ms].cpu().numpy())
    got = (tt[ms].cpu().numpy(), ee[ms].cpu().numpy(), te[ms].cpu().numpy())
    check(got, ref, 1e-5)
    # the paper's validation: |Delta C_l| / sigma_CV (Sec. 4.6), here far below 1
    assert orc.cosmic_variance_ratio(got[0], ref[0]).max() < 1e-3
    assert orc.cosmic_variance_ratio(got[1], ref[1]).max() < 1e-3
    assert orc.cosmic_variance_ratio_te(got[2], ref[0], ref[1], ref[2]).max() < 1e-3


def test_te_errors():
    wl = workload(2, 100, 10, 64, 2)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    S = torch.zeros((2, wl.nk, wl.ntau), dtype=torch.float32, device="cuda")
    P = torch.zeros((2, wl.nk), dtype=torch.float64, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl_te(g, S, S, P)
    assert ei.value.code == gcamb.ESTATE
    gcamb.bessel_table(g, gcamb.BF16X3)
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl_te(g, S, S, P, mode=gcamb.F16X3)
    assert ei.value.code == gcamb.EINVAL
    # a misaligned polarisation source (TMA needs 16-byte alignment)
    big = torch.zeros(2 * wl.nk * wl.ntau + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl_te(g, S, big[1:].view(2, wl.nk, wl.ntau), P)
    assert ei.value.code == gcamb.EINVAL
    # ntau % 4 != 0
    g2 = gcamb.grid_create(wl.k, synth.uniform_grid(200.0, 14000.0, 66), 14000.0, 2, 100)
    gcamb.bessel_table(g2, gcamb.BF16X3)
    S2 = torch.zeros((2, wl.nk, 66), dtype=torch.float32, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl_te(g2, S2, S2, P)
    assert ei.value.code == gcamb.EUNSUPPORTED
    assert gcamb.lib().gcamb_los_cl_te(g.handle, None, None, None, 0, gcamb.BF16X3, None, None, None, None, 0,
                                       None) == gcamb.OK
    gcamb.sync()


def test_te_k_sum_in_chunks_against_every_term_reduce(monkeypatch):
    """Eq. (1)'s k-sums of the TE kernel: FP32 sums of at most 16 k's terms
    (the default) against GCAMB_TC_KSUB=1, where every k's term is its own
    partial and the reduce forms the FP64 sum of the FP32-rounded terms.  The
    TT and EE terms are positive, so each chunk sum is within 15 * 2^-24 of
    their exact sum (one more 2^-24 for the rounding of each term there); the
    TE terms change sign, and Cauchy-Schwarz bounds the sum of their moduli by
    sqrt(TT EE), the scale the TE difference is held to.  With 2000 k nodes
    the first multipole tile has about 2000 partials with KSUB=1, more than the
    1024 indices the reduce stages in shared memory at a time."""
    wl = workload(2, 300, 2000, 128, 40)
    ST, SP, P = inputs(wl, seed=8)
    monkeypatch.setenv("GCAMB_TC_KSUB", "1")
    tt1, ee1, te1, _ = run_te(wl, ST, SP, P)
    monkeypatch.delenv("GCAMB_TC_KSUB", raising=False)
    tt, ee, te, _ = run_te(wl, ST, SP, P)
    assert np.all(tt1 > 0) and np.all(ee1 > 0) and np.all(np.isfinite(te))
    bound = 16 * 2.0 ** -24
    assert (np.abs(tt - tt1) / tt1).max() <= bound
    assert (np.abs(ee - ee1) / ee1).max() <= bound
    assert (np.abs(te - te1) / np.sqrt(tt1 * ee1)).max() <= bound
    assert not np.array_equal(tt, tt1)  # the chunk length reaches the kernel
