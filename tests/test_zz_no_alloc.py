"""The allocation-free entry point gcamb_los_cl_noalloc, through the C ABI.

Some callers may not allocate device memory -- for instance a likelihood
callback running inside a sampler or host framework that owns the device's
memory budget.  gcamb_los_cl_noalloc serves them from a fixed buffer inside
the library.  Its C_l must match gcamb_los_cl's (the entry point with a caller
workspace) within the batched path's tolerance, 1e-5 relative, on two calls
in a row: the shared buffer keeps the previous call's contents, so the second
call, on different sources, must not see stale scratch.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2509_25110_gb300 import build, gcamb, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gcamb.lib()


def _inputs(k, tau, M, seed):
    p = synth.model_params(M, seed=seed)
    S = torch.as_tensor(synth.sources(k, tau, p).astype(np.float32), device="cuda")
    P = torch.as_tensor(synth.primordial(k, p), device="cuda")
    return S, P


@pytest.mark.parametrize("mode", [gcamb.F16X3, gcamb.BF16X3])
def test_noalloc_matches_workspace_entry_point_twice(mode):
    k = synth.log_grid(1e-4, 0.3, 48)
    tau = synth.uniform_grid(200.0, 14000.0, 300)
    M, lmin, lmax = 40, 2, 400
    g = gcamb.grid_create(k, tau, 14000.0, lmin, lmax)
    gcamb.bessel_table(g, mode)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for seed in (11, 12):  # two calls in a row, different sources
        S, P = _inputs(k, tau, M, seed)
        ref = gcamb.los_cl(g, S, P, mode).cpu().numpy()
        C = torch.full((M, g.nl), float("nan"), dtype=torch.float64, device="cuda")
        gcamb.los_cl_noalloc(g, S, P, mode, C, status)
        gcamb.sync()
        got = C.cpu().numpy()
        assert int(status.item()) == 0
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, ref, rtol=TOL, atol=0)


def test_noalloc_rejects_problems_beyond_its_buffer():
    # 999 tau nodes: the sources are split into the scratch first (~314 MB)
    k = synth.log_grid(1e-4, 0.3, 300)
    tau = synth.uniform_grid(200.0, 14000.0, 999)
    g = gcamb.grid_create(k, tau, 14000.0, 2, 300)
    gcamb.bessel_table(g, gcamb.F16X3)
    S, P = _inputs(k, tau, 256, 13)
    C = torch.empty((256, g.nl), dtype=torch.float64, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl_noalloc(g, S, P, gcamb.F16X3, C)
    assert ei.value.code == gcamb.EINVAL
    assert "scratch" in str(ei.value)


_FRESH = r"""
import numpy as np, torch
from paper_2509_25110_gb300 import gcamb, synth
k = synth.log_grid(1e-4, 0.3, 40)
tau = synth.uniform_grid(200.0, 14000.0, 256)
M = 24
g = gcamb.grid_create(k, tau, 14000.0, 2, 300)
gcamb.bessel_table(g, gcamb.F16X3)
p = synth.model_params(M, seed=21)
S = torch.as_tensor(synth.sources(k, tau, p).astype(np.float32), device="cuda")
P = torch.as_tensor(synth.primordial(k, p), device="cuda")
C = torch.full((M, g.nl), float("nan"), dtype=torch.float64, device="cuda")
gcamb.los_cl_noalloc(g, S, P, gcamb.F16X3, C)   # the first batched call of the process, no status word
gcamb.sync()
ref = gcamb.los_cl(g, S, P, gcamb.F16X3).cpu().numpy()
got = C.cpu().numpy()
assert np.all(np.isfinite(got))
np.testing.assert_allclose(got, ref, rtol=1e-5, atol=0)
print("FRESH_OK")
"""


def test_noalloc_without_status_word_in_a_fresh_process():
    # status = NULL reports a timeout through the library's error word, which
    # the grid's first device call has set up: the entry point itself still
    # allocates nothing, even as the first library launch of a process
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "FRESH_OK" in r.stdout


def test_noalloc_refuses_a_capturing_stream():
    k = synth.log_grid(1e-4, 0.3, 32)
    tau = synth.uniform_grid(200.0, 14000.0, 128)
    g = gcamb.grid_create(k, tau, 14000.0, 2, 200)
    gcamb.bessel_table(g, gcamb.F16X3)
    S, P = _inputs(k, tau, 8, 14)
    C = torch.empty((8, g.nl), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        graph.capture_begin()
        try:
            with pytest.raises(gcamb.GcambError) as ei:
                gcamb.los_cl_noalloc(g, S, P, gcamb.F16X3, C, stream=s)
        finally:
            graph.capture_end()
    assert ei.value.code == gcamb.EUNSUPPORTED
    assert "capture" in str(ei.value)
    # the call still works outside the capture
    gcamb.los_cl_noalloc(g, S, P, gcamb.F16X3, C)
    gcamb.sync()
    np.testing.assert_allclose(C.cpu().numpy(), gcamb.los_cl(g, S, P, gcamb.F16X3).cpu().numpy(), rtol=TOL, atol=0)
