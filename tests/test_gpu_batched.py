"""GPU parity of the batched tensor-core path (gcamb_los_cl) against the FP64
oracle, through the C ABI.

The oracle is evaluated on the same FP32-rounded sources the device reads.
Tolerance: relative error on every C_l <= 1e-5 (the bound the batched split
precision must meet) for F16X3 and TF32X3, whose hi+lo splits carry 22
significant bits.  BF16X3's split carries 16 bits (unit roundoff 2^-8 per
part), so each product is off by up to ~3 * 2^-16 = 4.6e-5 relative; on
coarse grids, where few k and tau terms average the errors out, C_l errors
reach ~2e-5, and its bound here is 3e-5.  On the full 256-source l_max =
2500 grid all three modes meet 1e-5."""
import numpy as np
import pytest

from paper_2509_25110_gb300 import build, gcamb, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SPLIT_TOL = {gcamb.BF16X3: 3e-5, gcamb.TF32X3: 1e-5, gcamb.F16X3: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gcamb.lib()


def case(nk, ntau, lmin, lmax, M, seed=2):
    k = synth.log_grid(1e-4, 0.3, nk)
    tau = synth.uniform_grid(200.0, 14000.0, ntau)
    p = synth.model_params(M, seed=seed)
    S = synth.sources(k, tau, p).astype(np.float32)
    P = synth.primordial(k, p)
    return k, tau, S, P


def run(k, tau, S, P, lmin, lmax, mode, g=None):
    if g is None:
        g = gcamb.grid_create(k, tau, 14000.0, lmin, lmax)
    gcamb.bessel_table(g, mode)
    C = gcamb.los_cl(g, torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda"), mode)
    gcamb.sync()
    return C.cpu().numpy(), g


@pytest.mark.parametrize("mode", [gcamb.BF16X3, gcamb.F16X3, gcamb.TF32X3])
@pytest.mark.parametrize("nk,ntau,lmin,lmax,M", [
    (96, 1000, 2, 700, 4),     # NT = 64, six l-tiles (ragged), full tau blocks
    (120, 333, 2, 300, 100),   # NT = 128, ragged tau block, ragged source tile
    (64, 200, 0, 129, 300),    # two source tiles of 256, lmin = 0, tile boundary at 128
])
def test_los_cl_matches_oracle(orc, mode, nk, ntau, lmin, lmax, M):
    k, tau, S, P = case(nk, ntau, lmin, lmax, M)
    C, _ = run(k, tau, S, P, lmin, lmax, mode)
    sel = np.unique(np.linspace(0, M - 1, min(M, 6)).astype(int))
    _, Cr = orc.los_cl(k, tau, 14000.0, lmin, lmax, S[sel].astype(np.float64), P[sel], want_delta=False)
    err = np.abs(C[sel] / Cr - 1)
    assert err.max() <= SPLIT_TOL[mode], err.max()


def test_identical_models_and_permutation():
    k, tau, S, P = case(64, 300, 2, 400, 5)
    Srep = np.repeat(S[:1], 70, axis=0)
    Prep = np.repeat(P[:1], 70, axis=0)
    C, g = run(k, tau, Srep, Prep, 2, 400, gcamb.BF16X3)
    assert np.all(C == C[0:1])
    perm = np.array([3, 0, 4, 1, 2])
    C1, _ = run(k, tau, S, P, 2, 400, gcamb.BF16X3, g)
    C2, _ = run(k, tau, S[perm], P[perm], 2, 400, gcamb.BF16X3, g)
    assert np.array_equal(C2, C1[perm])


def test_deterministic_repeat():
    k, tau, S, P = case(80, 400, 2, 500, 40)
    C1, g = run(k, tau, S, P, 2, 500, gcamb.BF16X3)
    C2, _ = run(k, tau, S, P, 2, 500, gcamb.BF16X3, g)
    assert np.array_equal(C1, C2)


def test_workspace_and_state_errors():
    k, tau, S, P = case(16, 64, 2, 40, 3)
    g = gcamb.grid_create(k, tau, 14000.0, 2, 40)
    St = torch.as_tensor(S, device="cuda")
    Pt = torch.as_tensor(P, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl(g, St, Pt, gcamb.BF16X3)
    assert ei.value.code == gcamb.ESTATE
    gcamb.bessel_table(g, gcamb.BF16X3)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl(g, St, Pt, gcamb.BF16X3, ws=small)
    assert ei.value.code == gcamb.EINVAL
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl(g, St, Pt, gcamb.PLAIN64)
    assert ei.value.code == gcamb.EINVAL


@pytest.mark.parametrize("mode", [gcamb.F16X3, gcamb.BF16X3])
def test_batched_lmax2500_full_size_sampled(orc, mode):
    """The 256-model, l_max = 2500 workload at full size in the launch
    configuration the benchmark times; C_l of sampled models against the oracle."""
    wl = synth.workload("batched_lmax2500")
    p = synth.model_params(wl.M, seed=0)
    S = synth.sources_torch(wl.k, wl.tau, p, "cuda", torch.float32)
    P = torch.as_tensor(synth.primordial(wl.k, p), device="cuda")
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, mode)
    C = gcamb.los_cl(g, S, P, mode).cpu().numpy()
    gcamb.sync()
    sel = [0, 97, 255]
    _, Cr = orc.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, S[sel].double().cpu().numpy(),
                       P[sel].cpu().numpy(), want_delta=False)
    err = np.abs(C[sel] / Cr - 1)
    assert err.max() <= 1e-5, err.max()
