"""GPU parity of the plain FP64 / FP32 path (Bessel table, Eq. 2 transfer,
Eq. 1 C_l) against the FP64 oracle, through the C ABI.

Tolerances (relative, per multipole): C_l <= 1e-10 for PLAIN64, <= 1e-5 for
PLAIN32.  Transfer functions are compared on the scale of the largest
|Delta| of their model (they cross zero)."""
import math

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


def run_plain(wl, S, P, mode):
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, mode)
    dt = torch.float64 if mode == gcamb.PLAIN64 else torch.float32
    D = gcamb.los_transfer(g, dev(S, dt), mode)
    C = gcamb.cl(g, D, dev(P))
    gcamb.sync()
    return D.cpu().numpy().astype(np.float64), C.cpu().numpy(), g


def small_workload(lmin=2, lmax=400, nk=40, ntau=300, M=3):
    return synth.Workload("small", synth.log_grid(1e-4, 0.3, nk), synth.uniform_grid(200.0, 14000.0, ntau),
                          14000.0, lmin, lmax, M)


# --------------------------------------------------------------- Bessel routine

def test_sph_bessel_matches_oracle(orc):
    rng = np.random.default_rng(4)
    x = np.concatenate([[0.0, 1e-200, 1e-12, 1e-3, 0.5, 0.999, 1.0, 1.5, 2.0],
                        10 ** rng.uniform(-2, math.log10(9000.0), 120)])
    for lmax in (40, 700, 6000):
        out = gcamb.sph_bessel(dev(x), lmax).cpu().numpy()
        gcamb.sync()
        ref = orc.sph_bessel(lmax, x)
        l = np.arange(lmax + 1)[None, :]
        env = np.where(l > x[:, None], np.abs(ref), np.maximum(np.abs(ref), 1.0 / np.maximum(x[:, None], 1e-300)))
        err = np.abs(out - ref)
        ok = err <= 1e-11 * env + 1e-40
        assert ok.all(), (np.argwhere(~ok)[:5], err[~ok][:5], ref[~ok][:5])


def test_sph_bessel_sum_rule():
    x = np.array([0.3, 3.7, 250.0, 4000.0])
    L = 4800
    out = gcamb.sph_bessel(dev(x), L).cpu().numpy()
    l = np.arange(L + 1)
    s = ((2 * l + 1) * out * out).sum(axis=1)
    assert np.abs(s - 1).max() < 1e-12


# --------------------------------------------------------------- transfer + C_l

@pytest.mark.parametrize("lmin,lmax,nk,ntau,M", [
    (2, 400, 40, 300, 3),     # several l-tiles with a ragged last tile, ragged tau-block
    (0, 130, 7, 50, 1),       # lmin = 0, one partial tau-block, tile boundary at 128
    (2, 2, 1, 1, 2),          # degenerate: one k, one tau node (zero weight), one l
    (5, 260, 25, 129, 5),     # M not a multiple of the source chunk
])
def test_plain64_matches_oracle(orc, lmin, lmax, nk, ntau, M):
    wl = small_workload(lmin, lmax, nk, ntau, M)
    p = synth.model_params(M, seed=3)
    S = synth.sources(wl.k, wl.tau, p)
    P = synth.primordial(wl.k, p)
    D, C, _ = run_plain(wl, S, P, gcamb.PLAIN64)
    Dr, Cr = orc.los_cl(wl.k, wl.tau, wl.tau0, lmin, lmax, S, P)
    scale = np.abs(Dr).reshape(M, -1).max(axis=1)[:, None, None] + 1e-300
    assert np.abs(D - Dr).max() <= 1e-11 * scale.max()
    assert np.all(np.abs(D - Dr) <= 1e-11 * scale)
    nz = Cr > 0
    assert np.all(np.abs(C[nz] - Cr[nz]) <= 1e-10 * Cr[nz])
    assert np.all(C[~nz] == 0)


def test_plain32_matches_oracle(orc):
    wl = small_workload()
    p = synth.model_params(wl.M, seed=5)
    S = synth.sources(wl.k, wl.tau, p)
    P = synth.primordial(wl.k, p)
    D, C, _ = run_plain(wl, S.astype(np.float32), P, gcamb.PLAIN32)
    Dr, Cr = orc.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, S.astype(np.float32).astype(np.float64), P)
    assert np.all(np.abs(C - Cr) <= 1e-5 * Cr)


def test_delta_source_reproduces_bessel(orc):
    wl = small_workload(2, 300, 12, 64, 1)
    w = orc.trapz_weights(wl.tau)
    istar = 20
    S = np.zeros((1, wl.nk, wl.ntau))
    S[0, :, istar] = 1.0 / w[istar]
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    D = gcamb.los_transfer(g, dev(S), gcamb.PLAIN64).cpu().numpy()[0]
    for q in range(wl.nk):
        x = wl.k[q] * (wl.tau0 - wl.tau[istar])
        ref = orc.sph_bessel(wl.lmax, x)[2:]
        big = np.abs(ref) > 1e-25
        assert np.allclose(D[q][big], ref[big], rtol=1e-12, atol=0)
        assert np.all(np.abs(D[q][~big]) < 1e-24)


def test_plain_lmax500_full_size(orc):
    """The 1-model, l_max = 500 workload at its full size, FP64 and FP32."""
    wl = synth.workload("plain_lmax500")
    p = synth.model_params(1, seed=0)
    S = synth.sources(wl.k, wl.tau, p)
    P = synth.primordial(wl.k, p)
    _, Cr = orc.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, S, P, want_delta=False)
    _, C64, _ = run_plain(wl, S, P, gcamb.PLAIN64)
    assert np.abs(C64 / Cr - 1).max() <= 1e-10
    _, C32, _ = run_plain(wl, S.astype(np.float32), P, gcamb.PLAIN32)
    _, Cr32 = orc.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, S.astype(np.float32).astype(np.float64), P,
                         want_delta=False)
    assert np.abs(C32 / Cr32 - 1).max() <= 1e-5


def test_plain_lmax5000_against_oracle(orc):
    """The 1-model, l_max = 5000 workload at full size (3000 k, 2000 tau
    dense around the visibility peak).  C_l for every l = 2..5000 against the
    oracle's own C_l (its weights, its j_l), stored by
    tests/golden/make_plain_lmax5000.py, which calls only the oracle and the
    seeded generator: <= 1e-10 (FP64), <= 1e-5 (FP32 sources).  Delta at
    sampled k against the oracle with its own trapezoid weights."""
    import os
    gold = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "plain_lmax5000_cl.txt"))
    wl = synth.workload("plain_lmax5000")
    assert np.array_equal(gold[:, 0], np.arange(wl.lmin, wl.lmax + 1))
    p = synth.model_params(1, seed=0)
    S = synth.sources(wl.k, wl.tau, p)
    P = synth.primordial(wl.k, p)
    for mode, col, tol in ((gcamb.PLAIN64, 1, 1e-10), (gcamb.PLAIN32, 2, 1e-5)):
        Sm = S if mode == gcamb.PLAIN64 else S.astype(np.float32)
        D, C, g = run_plain(wl, Sm, P, mode)
        err = np.abs(C[0] / gold[:, col] - 1)
        assert err.max() <= tol, (mode, err.max(), int(np.argmax(err)) + wl.lmin)
        qs = np.array([0, 700, 1500, 2100, 2600, 2999])
        Dr, _ = orc.los_cl(wl.k[qs], wl.tau, wl.tau0, wl.lmin, wl.lmax, Sm[:, qs].astype(np.float64),
                           want_cl=False)
        scale = np.abs(Dr).max()
        assert np.abs(D[:, qs] - Dr).max() <= (1e-11 if mode == gcamb.PLAIN64 else 1e-5) * scale


def test_deterministic_repeat():
    wl = small_workload()
    p = synth.model_params(wl.M, seed=8)
    S = synth.sources(wl.k, wl.tau, p)
    P = synth.primordial(wl.k, p)
    _, C1, _ = run_plain(wl, S, P, gcamb.PLAIN64)
    _, C2, _ = run_plain(wl, S, P, gcamb.PLAIN64)
    assert np.array_equal(C1, C2)


def test_state_and_argument_errors():
    wl = small_workload()
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    S = torch.zeros((1, wl.nk, wl.ntau), dtype=torch.float64, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_transfer(g, S, gcamb.PLAIN64)
    assert ei.value.code == gcamb.ESTATE
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.bessel_table(g, 17)
    assert ei.value.code == gcamb.EINVAL


def test_probe_rates_are_sane():
    f64 = gcamb.probe_flops(0)
    f32 = gcamb.probe_flops(1)
    assert 1e11 < f64 < 1e15 and 1e12 < f32 < 1e15
