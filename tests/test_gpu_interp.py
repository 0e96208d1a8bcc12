"""GPU parity of the source interpolation onto the transfer k grid
(gcamb_interp_sources: natural cubic spline in k, in the sources precision) against the
oracle's spline (oracle/interp.py), through the C ABI.

Bars: FP64 sources within 1e-12 of the largest |S| (the same arithmetic in a
different order).  FP32 (solved and evaluated in FP32): within 64 * 2^-24 of
the sum of the absolute terms of the spline formula at each point,
|(1-t) y_j| + |t y_(j+1)| + h^2/6 (|(1-t)^3-(1-t)| |M_j| + |t^3-t| |M_(j+1)|),
with the oracle's M (about ten roundings of the formula plus the FP32 sweep's
error in M; an FP32 emulation of the kernel's arithmetic gives at most 29
ulp on these grids).  The second-derivative terms can exceed |y| many times
on uneven nodes, so the bar is not a multiple of the largest |S|.  The
interpolated sources fed to the batched projection: within 1e-5 of the
oracle's projection of its own interpolated sources."""
import numpy as np
import pytest

from oracle import interp as ointerp
from paper_2509_25110_gb300 import build, gcamb, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gcamb.lib()


def grid(nk=95, ntau=64, lmax=100):
    return gcamb.grid_create(synth.log_grid(1e-4, 0.3, nk), synth.uniform_grid(200.0, 14000.0, ntau), 14000.0, 2,
                             lmax)


@pytest.mark.parametrize("nk_in,M,ntau", [(30, 3, 64), (2, 2, 64), (3, 1, 64), (200, 5, 64), (30, 3, 63)])
def test_interp_matches_oracle(nk_in, M, ntau):
    """ntau = 64: the FP32 evaluation takes four tau columns a thread; 63:
    one column a thread."""
    g = grid(ntau=ntau)
    rng = np.random.default_rng(nk_in)
    k_in = np.geomspace(1e-4, 0.3, nk_in)
    k_in[1:-1] *= np.exp(rng.uniform(-0.01, 0.01, max(0, nk_in - 2)))  # uneven spacing
    S = rng.normal(size=(M, nk_in, g.ntau))
    ref = ointerp.interp_sources(k_in, S, g.k)
    out64 = gcamb.interp_sources(g, k_in, torch.as_tensor(S, device="cuda")).cpu().numpy()
    assert np.abs(out64 - ref).max() <= 1e-12 * np.abs(S).max()
    S32 = S.astype(np.float32)
    ref32 = ointerp.interp_sources(k_in, S32.astype(np.float64), g.k)
    out32 = gcamb.interp_sources(g, k_in, torch.as_tensor(S32, device="cuda")).cpu().numpy()
    # the envelope of the formula's terms, from the oracle's second derivatives
    cols = np.moveaxis(S32.astype(np.float64), 1, -1)
    Mo = ointerp.natural_second_derivatives(k_in, cols)
    j = np.clip(np.searchsorted(k_in, g.k, side="right") - 1, 0, nk_in - 2)
    h = k_in[j + 1] - k_in[j]
    t = (g.k - k_in[j]) / h
    u = 1.0 - t
    env = (np.abs(u * cols[..., j]) + np.abs(t * cols[..., j + 1]) +
           h * h / 6.0 * (np.abs(u ** 3 - u) * np.abs(Mo[..., j]) + np.abs(t ** 3 - t) * np.abs(Mo[..., j + 1])))
    env = np.moveaxis(env, -1, 1)
    assert np.all(np.abs(out32 - ref32) <= 64 * 2.0 ** -24 * env + 1e-30)
    gcamb.sync()


def test_interpolated_sources_through_the_batched_projection(orc):
    """Sources of the synthetic family on a 300-node 'solver' k grid,
    interpolated to the 1000-node transfer grid, then projected (BF16X3)."""
    k_ode = np.geomspace(1e-4, 0.3, 300)
    wl = synth.Workload("i", np.geomspace(1.2e-4, 0.29, 1000), synth.uniform_grid(200.0, 14000.0, 400), 14000.0, 2,
                        600, 8)
    p = synth.model_params(wl.M, seed=9)
    S_ode = synth.sources(k_ode, wl.tau, p)
    P = synth.primordial(wl.k, p)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, gcamb.BF16X3)
    S = gcamb.interp_sources(g, k_ode, torch.as_tensor(S_ode.astype(np.float32), device="cuda"))
    C = gcamb.los_cl(g, S, torch.as_tensor(P, device="cuda"), gcamb.BF16X3).cpu().numpy()
    gcamb.sync()
    S_ref = ointerp.interp_sources(k_ode, S_ode.astype(np.float32).astype(np.float64), wl.k)
    _, C_ref = orc.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, S_ref.astype(np.float32).astype(np.float64), P,
                          want_delta=False)
    assert np.abs(C / C_ref - 1).max() <= 1e-5


def test_interp_errors():
    g = grid()
    S = torch.zeros((1, 10, g.ntau), dtype=torch.float64, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:  # grid's k range outside k_in
        gcamb.interp_sources(g, np.geomspace(2e-4, 0.3, 10), S)
    assert ei.value.code == gcamb.EINVAL
    with pytest.raises(gcamb.GcambError) as ei:  # not increasing
        gcamb.interp_sources(g, np.geomspace(0.3, 1e-4, 10), S)
    assert ei.value.code == gcamb.EINVAL
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.interp_sources(g, np.array([1e-4]), S[:, :1])
    assert ei.value.code == gcamb.EINVAL
    gcamb.sync()
