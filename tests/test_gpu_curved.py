"""GPU parity of the curved-space projection (gcamb_grid_create_curved:
hyperspherical Bessel kernels, open and closed space) against the FP64
oracle, through the C ABI.

Bars as on flat grids: the table's Phi_l (a delta source) within 1e-11 of
the largest |Phi| per k; PLAIN64 transfer functions within 1e-11 of their
scale and C_l within 1e-10 relative; BF16X3 C_l within the derived split
bound 6 * 2^-16 on these small grids.  The device finds the tau-prefixes from
its own evaluation of Phi (eps_cut), while the oracle sums every node."""
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


def q_grid(K, n=40):
    q = synth.log_grid(1e-3, 0.3, n)
    if K > 0:  # closed: integer beta = q / sqrt(K)
        rk = np.sqrt(K)
        q = np.unique(np.maximum(np.round(q / rk), 3.0)) * rk
    return q


@pytest.mark.parametrize("K", [-1e-8, 1e-8, -5.45e-10])
def test_delta_source_gives_phi(orc, K):
    q = q_grid(K, 15)
    tau = synth.uniform_grid(200.0, 14000.0, 64)
    g = gcamb.grid_create_curved(q, tau, 14000.0, 0, 300, K)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    w = orc.trapz_weights(tau)
    i = 30
    S = np.zeros((1, q.size, tau.size))
    S[0, :, i] = 1.0 / w[i]
    D = gcamb.los_transfer(g, dev(S), gcamb.PLAIN64).cpu().numpy()[0]
    gcamb.sync()
    rk = np.sqrt(abs(K))
    ref = orc.hyper_bessel(q / rk, rk * (14000.0 - tau[i]), 300, K > 0)
    for j in range(q.size):
        assert np.abs(D[j] - ref[j]).max() <= 1e-11 * np.abs(ref[j]).max(), (j, q[j])


@pytest.mark.parametrize("K,lmin,lmax,ntau,M", [(-1e-8, 2, 400, 300, 3), (1e-8, 2, 400, 300, 3),
                                                (-1e-8, 0, 130, 52, 1), (-5.45e-10, 5, 260, 128, 5)])
def test_curved_plain64_matches_oracle(orc, K, lmin, lmax, ntau, M):
    q = q_grid(K)
    tau = synth.uniform_grid(200.0, 14000.0, ntau)
    p = synth.model_params(M, seed=61)
    S = synth.sources(q, tau, p)
    P = synth.primordial(q, p)
    g = gcamb.grid_create_curved(q, tau, 14000.0, lmin, lmax, K)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    D = gcamb.los_transfer(g, dev(S), gcamb.PLAIN64)
    C = gcamb.cl(g, D, dev(P)).cpu().numpy()
    D = D.cpu().numpy()
    gcamb.sync()
    Dr = orc.los_curved(q, tau, 14000.0, K, lmin, lmax, S)
    Cr = orc.cl_from_delta(q, Dr, P)
    scale = np.abs(Dr).reshape(M, -1).max(axis=1)[:, None, None]
    assert np.all(np.abs(D - Dr) <= 1e-11 * scale)
    assert np.all(np.abs(C - Cr) <= 1e-10 * Cr)


@pytest.mark.parametrize("K", [-1e-8, 1e-8])
def test_curved_batched_matches_oracle(orc, K):
    q = q_grid(K, 60)
    tau = synth.uniform_grid(200.0, 14000.0, 400)
    M = 70
    p = synth.model_params(M, seed=62)
    S = synth.sources(q, tau, p, np.float32)
    P = synth.primordial(q, p)
    g = gcamb.grid_create_curved(q, tau, 14000.0, 2, 600, K)
    gcamb.bessel_table(g, gcamb.BF16X3)
    C = gcamb.los_cl(g, dev(S, torch.float32), dev(P), gcamb.BF16X3).cpu().numpy()
    gcamb.sync()
    sub = [0, 33, 69]
    Dr = orc.los_curved(q, tau, 14000.0, K, 2, 600, S[sub].astype(np.float64))
    Cr = orc.cl_from_delta(q, Dr, P[sub])
    assert np.abs(C[sub] / Cr - 1).max() <= SPLIT_TOL


def test_flat_limit_matches_the_flat_grid():
    q = synth.log_grid(1e-3, 0.3, 40)
    tau = synth.uniform_grid(200.0, 14000.0, 200)
    p = synth.model_params(2, seed=63)
    S = dev(synth.sources(q, tau, p))
    P = dev(synth.primordial(q, p))
    gf = gcamb.grid_create(q, tau, 14000.0, 2, 300)
    gc = gcamb.grid_create_curved(q, tau, 14000.0, 2, 300, -1e-20)  # R = 1e10 Mpc: (r/R)^2 ~ 2e-12
    out = []
    for g in (gf, gc):
        gcamb.bessel_table(g, gcamb.PLAIN64)
        out.append(gcamb.cl(g, gcamb.los_transfer(g, S, gcamb.PLAIN64), P).cpu().numpy())
    gcamb.sync()
    assert np.abs(out[1] / out[0] - 1).max() <= 1e-9


def test_curved_rejections():
    q = q_grid(-1e-8, 10)
    tau = synth.uniform_grid(200.0, 14000.0, 64)
    g = gcamb.grid_create_curved(q, tau, 14000.0, 2, 100, -1e-8)
    gcamb.bessel_table(g, gcamb.PLAIN64)
    gcamb.bessel_table(g, gcamb.BF16X3)
    S = torch.zeros((1, q.size, tau.size), dtype=torch.float64, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_transfer_e(g, S, gcamb.PLAIN64)
    assert ei.value.code == gcamb.EUNSUPPORTED
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_transfer_tensor(g, S, S, gcamb.PLAIN64)
    assert ei.value.code == gcamb.EUNSUPPORTED
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl_te(g, S.float(), S.float(), torch.zeros((1, q.size), dtype=torch.float64, device="cuda"))
    assert ei.value.code == gcamb.EUNSUPPORTED
    with pytest.raises(gcamb.GcambError) as ei:  # closed space: beta must be an integer
        gcamb.grid_create_curved(np.array([1.05e-3, 2e-3]), tau, 14000.0, 2, 100, 1e-8)
    assert ei.value.code == gcamb.EINVAL
    gcamb.sync()
