"""Failure detection on the GPU without a GPU fault, through the C ABI.

Every tensor-core kernel of the library waits on mbarriers with a one-second
limit; a wait that runs out reports GCAMB_ETIMEOUT through the library's
error flag (read and cleared by gcamb_sync) or a caller's status word, and
the kernel ends.  gcamb_selftest_wait runs that same wait on a barrier that
nothing arrives on, so the limit is reached for certain.  After it the CUDA
context must still work: the batched path gives its earlier result again.
Nothing here faults, traps or hangs the device."""
import time

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


def _small_batch():
    k = synth.log_grid(1e-4, 0.3, 40)
    tau = synth.uniform_grid(200.0, 14000.0, 200)
    g = gcamb.grid_create(k, tau, 14000.0, 2, 200)
    gcamb.bessel_table(g, gcamb.BF16X3)
    p = synth.model_params(20, seed=41)
    S = torch.as_tensor(synth.sources(k, tau, p).astype(np.float32), device="cuda")
    P = torch.as_tensor(synth.primordial(k, p), device="cuda")
    return g, S, P


def test_expired_wait_is_reported_by_sync_and_the_context_survives():
    g, S, P = _small_batch()
    before = gcamb.los_cl(g, S, P, gcamb.BF16X3).cpu().numpy()
    gcamb.sync()
    t0 = time.perf_counter()
    gcamb.selftest_wait()
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.sync()
    assert ei.value.code == gcamb.ETIMEOUT
    assert 0.9 <= time.perf_counter() - t0 <= 30.0  # the wait ran to its one-second limit, then ended
    gcamb.sync()  # the flag was cleared by the previous sync
    after = gcamb.los_cl(g, S, P, gcamb.BF16X3).cpu().numpy()
    gcamb.sync()
    assert np.array_equal(before, after)


def test_expired_wait_is_reported_in_a_status_word():
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    gcamb.selftest_wait(status)
    gcamb.sync()  # reported in the status word, not the flag
    assert int(status.item()) == gcamb.ETIMEOUT
