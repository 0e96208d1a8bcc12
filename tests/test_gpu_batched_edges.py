"""Edge cases of the batched tensor-core path (gcamb_los_cl) against the FP64
oracle, through the C ABI: few k nodes, one ragged tau block (read in place
and through the split pass), a single multipole, l = 0 alone, a one-source
second source tile with an odd number of l-tiles (the last pair of l-tiles
has one), one k node (trapezoid weight zero: C_l = 0 exactly), and M = 0
(a no-op that writes nothing).

Bound: the split products are within 3 * 2^-16 of the exact ones (BF16X3's
16-bit split; F16X3 and TF32X3 split finer) and the tensor core accumulates
ntau terms in FP32, so with A = sum_i w_i |S_i| |j_l(x_i)| the error of
Delta is at most d = (3 * 2^-16 + ntau 2^-24) A (+ F, F16X3) and
    |C_l - C_l^oracle| <= 4 pi sum_k w_k P (2 |Delta| d + d^2),
which holds where the terms of Delta cancel, as they can on these grids.
F16X3 has an absolute floor besides: its table holds w_i j_l 2^sJ with one
scale (max_i w_i 2^sJ < 2^14), and a hi + lo split in fp16 is exact to
2^-22 of the value plus 2^-25 absolute (the subnormal spacing), i.e. at
most 2^-37 max_i w_i per entry in units of w j; the sources, scaled per row
to a maximum in [2^13, 2^14), at most 2^-38 of the row maximum.  Hence
F = 2^-36 max_i w_i ntau max_i |S_i| per (source, k)."""
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


def inputs(nk, ntau, M, seed=5):
    k = synth.log_grid(1e-4, 0.3, nk) if nk > 1 else np.array([0.01])
    tau = synth.uniform_grid(200.0, 14000.0, ntau)  # ends at tau0: x = 0 on the last node
    p = synth.model_params(M, seed=seed)
    return k, tau, synth.sources(k, tau, p).astype(np.float32), synth.primordial(k, p)


def run(k, tau, S, P, lmin, lmax, mode):
    g = gcamb.grid_create(k, tau, 14000.0, lmin, lmax)
    gcamb.bessel_table(g, mode)
    C = gcamb.los_cl(g, torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda"), mode)
    gcamb.sync()
    return C.cpu().numpy()


@pytest.mark.parametrize("mode", [gcamb.BF16X3, gcamb.F16X3, gcamb.TF32X3])
@pytest.mark.parametrize("nk,ntau,lmin,lmax,M", [
    (2, 40, 2, 50, 3),       # two k nodes
    (30, 8, 2, 40, 2),       # one ragged tau block, read in place
    (30, 7, 2, 40, 2),       # one ragged tau block, split pass (ntau % 4 != 0)
    (30, 100, 10, 10, 5),    # a single multipole
    (25, 96, 0, 0, 3),       # l = 0 alone (every node active, x = 0 included)
    (20, 64, 2, 300, 129),   # second source tile of one source; three l-tiles
])
def test_edges_within_bound(orc, mode, nk, ntau, lmin, lmax, M):
    k, tau, S, P = inputs(nk, ntau, M)
    C = run(k, tau, S, P, lmin, lmax, mode)
    assert C.shape == (M, lmax - lmin + 1) and np.all(np.isfinite(C))
    S64 = S.astype(np.float64)
    D, Cr = orc.los_cl(k, tau, 14000.0, lmin, lmax, S64, P)
    w = orc.trapz_weights(tau)
    x = (k[:, None] * (14000.0 - tau[None, :])).ravel()
    J = np.abs(orc.sph_bessel(lmax, x)).reshape(nk, ntau, -1)[:, :, lmin:lmax + 1]
    A = np.einsum("mki,kil->mkl", np.abs(S64) * w, J)
    f = 4.0 * np.pi * orc.lnk_weights(k)[None, :, None] * P[:, :, None]
    d = (3 * 2.0 ** -16 + ntau * 2.0 ** -24) * A
    if mode == gcamb.F16X3:
        d = d + 2.0 ** -36 * w.max() * ntau * np.abs(S64).max(axis=2)[:, :, None]
    bound = (f * (2.0 * np.abs(D) * d + d * d)).sum(axis=1)
    err = np.abs(C - Cr)
    assert np.all(err <= bound), np.max(err / np.maximum(bound, 1e-300))


@pytest.mark.parametrize("mode", [gcamb.BF16X3, gcamb.F16X3])
def test_one_k_node_gives_zero(orc, mode):
    """One k node: its trapezoid weight in ln k is zero, so C_l = 0 exactly
    (the oracle's too)."""
    k, tau, S, P = inputs(1, 64, 3)
    C = run(k, tau, S, P, 2, 100, mode)
    _, Cr = orc.los_cl(k, tau, 14000.0, 2, 100, S.astype(np.float64), P)
    assert np.all(Cr == 0.0) and np.all(C == 0.0)


def test_zero_sources_is_a_no_op():
    """M = 0: GCAMB_OK and nothing written (the output keeps its sentinel)."""
    k, tau, S, P = inputs(20, 64, 1)
    g = gcamb.grid_create(k, tau, 14000.0, 2, 100)
    gcamb.bessel_table(g, gcamb.BF16X3)
    Cl = torch.full((1, g.nl), -7.0, dtype=torch.float64, device="cuda")
    S0 = torch.empty((0, g.nk, g.ntau), dtype=torch.float32, device="cuda")
    P0 = torch.empty((0, g.nk), dtype=torch.float64, device="cuda")
    gcamb.los_cl(g, S0, P0, gcamb.BF16X3, Cl[:0])
    gcamb.sync()
    assert torch.all(Cl == -7.0)


def test_misaligned_workspace_is_rejected():
    """A workspace pointer that is not 16-byte aligned is refused with
    GCAMB_EINVAL before any launch (bulk copies and vector loads read it);
    the output keeps its sentinel, and an aligned workspace then works."""
    k, tau, S, P = inputs(20, 64, 3)
    g = gcamb.grid_create(k, tau, 14000.0, 2, 100)
    gcamb.bessel_table(g, gcamb.F16X3)
    need = gcamb.los_cl_workspace(g, 3, gcamb.F16X3)
    buf = torch.empty(need + 64, dtype=torch.uint8, device="cuda")
    Cl = torch.full((3, g.nl), -7.0, dtype=torch.float64, device="cuda")
    St, Pt = torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda")
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl(g, St, Pt, gcamb.F16X3, Cl, buf[4:4 + need])
    assert ei.value.code == gcamb.EINVAL and "aligned" in gcamb.last_error()
    gcamb.sync()
    assert torch.all(Cl == -7.0)
    gcamb.los_cl(g, St, Pt, gcamb.F16X3, Cl, buf[:need])
    gcamb.sync()
    assert torch.all(torch.isfinite(Cl)) and torch.all(Cl > 0)


def test_side_stream_gives_the_same_bits():
    """Every launch of the batched path goes on the caller's stream: the same
    batch through gcamb_los_cl, a plan (graph) and the TE kernel on a
    non-default stream (inputs made on the default stream, which the side
    stream waits for) gives the default stream's results bit for bit, and
    the side stream's completion alone makes them visible."""
    k, tau, S, P = inputs(40, 128, 70)
    g = gcamb.grid_create(k, tau, 14000.0, 2, 300)
    gcamb.bessel_table(g, gcamb.F16X3)
    gcamb.bessel_table(g, gcamb.BF16X3)
    St, Pt = torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda")
    SPt = torch.as_tensor(0.5 * S[:, :, ::-1].copy(), device="cuda")
    ref = gcamb.los_cl(g, St, Pt, gcamb.F16X3)
    plan = gcamb.plan_create(g, 70, mode=gcamb.F16X3)
    ref_p = gcamb.plan_launch(plan, St, Pt)
    ref_te = gcamb.los_cl_te(g, St, SPt, Pt)
    gcamb.sync()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        Cl = torch.full_like(ref, -1.0)
        Cp = torch.full_like(ref, -1.0)
        te = tuple(torch.full_like(ref, -1.0) for _ in range(3))
        gcamb.los_cl(g, St, Pt, gcamb.F16X3, Cl, stream=side)
        plan2 = gcamb.plan_create(g, 70, mode=gcamb.F16X3)
        gcamb.plan_launch(plan2, St, Pt, Cp, stream=side)
        gcamb.los_cl_te(g, St, SPt, Pt, out=te, stream=side)
    side.synchronize()
    assert torch.equal(Cl, ref) and torch.equal(Cp, ref_p) and torch.equal(Cp, ref)
    for a, b in zip(te, ref_te):
        assert torch.equal(a, b)


def test_two_host_threads_share_the_library():
    """Two host threads, each with its own grid and stream, call the library
    at the same time (ctypes releases the interpreter lock around each call):
    plan caches, tables and error text are per grid or per thread, so each
    thread gets the C_l a single thread gets, bit for bit, and an error one
    thread provokes is reported to that thread only."""
    import threading
    cases = [inputs(30, 96, 40, seed=11), inputs(36, 128, 90, seed=12)]
    refs = []
    for k, tau, S, P in cases:
        g = gcamb.grid_create(k, tau, 14000.0, 2, 260)
        gcamb.bessel_table(g, gcamb.F16X3)
        refs.append(gcamb.los_cl(g, torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda"),
                                 gcamb.F16X3).cpu())
        gcamb.sync()
        gcamb.grid_destroy(g)
    out, errs = [None, None], []

    def work(i):
        try:
            k, tau, S, P = cases[i]
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                g = gcamb.grid_create(k, tau, 14000.0, 2, 260)
                gcamb.bessel_table(g, gcamb.F16X3, stream=st)
                St, Pt = torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda")
                st.synchronize()
                for _ in range(5):
                    C = gcamb.los_cl(g, St, Pt, gcamb.F16X3, stream=st)
                    if i == 1:  # an argument error on this thread only
                        with pytest.raises(gcamb.GcambError):
                            gcamb.grid_create(k[::-1].copy(), tau, 14000.0, 2, 260)
                        assert "increasing" in gcamb.last_error()
                st.synchronize()
                if i == 0:  # the other thread's errors do not reach this one
                    assert "increasing" not in gcamb.last_error()
                out[i] = C.cpu()
                gcamb.grid_destroy(g)
        except Exception as e:  # reported below, on the main thread
            errs.append(repr(e))

    ts = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs, errs
    for i in range(2):
        assert torch.equal(out[i], refs[i])
