"""GPU parity of the batched tensor-core path (gcamb_los_cl) against the FP64
oracle, through the C ABI.

The oracle is evaluated on the same FP32-rounded sources the device reads.
Tolerance: relative error on every C_l <= 1e-5 (the bound the batched split
precision must meet) for F16X3 and TF32X3, whose hi+lo splits carry 22
significant bits.  BF16X3's split carries 16: with unit roundoff 2^-8 per
part, hi + lo represents each operand within 2^-16 relative, so a split
product (two represented operands, lo*lo dropped) is off by at most
3 * 2^-16 relative, and C_l, quadratic in Delta, by at most 6 * 2^-16 = 9.2e-5
where the terms of Delta do not cancel.  That is its bound on the coarse
grids here (measured up to 3.05e-5).  On the full 256-source l_max = 2500
grid all three modes meet 1e-5.  F16X3 is the library's headline mode (the
benchmark's default): it meets 1e-5 on every grid here and on the full grid
(32 of the 256 sources checked here; the benchmark checks all 256)."""
import numpy as np
import pytest

from paper_2509_25110_gb300 import build, gcamb, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SPLIT_TOL = {gcamb.BF16X3: 6 * 2.0 ** -16, gcamb.TF32X3: 1e-5, gcamb.F16X3: 1e-5}


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
    (96, 1000, 2, 700, 4),     # NT = 64, six l-tiles (ragged), ragged last tau block
    (120, 333, 2, 300, 100),   # NT = 128, ragged tau block, ragged source tile
    (64, 200, 0, 129, 300),    # three source tiles of 128, lmin = 0, tile boundary at 128
    (70, 332, 2, 300, 100),    # sources read in place (ntau % 4 == 0): ragged tau block and source tile
    (63, 200, 2, 300, 5),      # an odd number of (source, k) rows: the row-scale pass's last warp has one
])
def test_los_cl_matches_oracle(orc, mode, nk, ntau, lmin, lmax, M):
    k, tau, S, P = case(nk, ntau, lmin, lmax, M)
    C, _ = run(k, tau, S, P, lmin, lmax, mode)
    sel = np.unique(np.linspace(0, M - 1, min(M, 6)).astype(int))
    _, Cr = orc.los_cl(k, tau, 14000.0, lmin, lmax, S[sel].astype(np.float64), P[sel], want_delta=False)
    err = np.abs(C[sel] / Cr - 1)
    assert err.max() <= SPLIT_TOL[mode], err.max()


@pytest.mark.parametrize("mode", [gcamb.BF16X3, gcamb.F16X3])
@pytest.mark.parametrize("nk,ntau,lmax,M", [(70, 332, 300, 100), (50, 256, 260, 40), (40, 200, 140, 300)])
def test_fused_conversion_matches_split_pass_bitwise(monkeypatch, mode, nk, ntau, lmax, M):
    """The tensor-core kernel that splits the FP32 sources in shared memory
    feeds the MMAs the same operand bits, in the same order, as the separate
    split pass: the C_l agree bit for bit (ragged tau blocks, ragged source
    tiles, 64- and 128-source tiles).  One multipole tile per work item, as
    in the split pass's plan, so that the k-chunks are the same."""
    k, tau, S, P = case(nk, ntau, 2, lmax, M)
    monkeypatch.delenv("GCAMB_TC_FUSED", raising=False)
    monkeypatch.setenv("GCAMB_TC_LP", "1")
    C_f, g = run(k, tau, S, P, 2, lmax, mode)
    ws_f = gcamb.los_cl_workspace(g, M, mode)
    monkeypatch.setenv("GCAMB_TC_FUSED", "0")
    C_s, _ = run(k, tau, S, P, 2, lmax, mode, g)
    ws_s = gcamb.los_cl_workspace(g, M, mode)
    assert ws_f < ws_s  # the in-place path keeps no split sources in its workspace
    assert np.all(np.isfinite(C_f))
    assert np.array_equal(C_f, C_s)


@pytest.mark.parametrize("mode", [gcamb.BF16X3, gcamb.F16X3])
@pytest.mark.parametrize("nk,ntau,lmin,lmax,M", [
    (70, 332, 2, 300, 100),    # three l-tiles: the last pair has one tile; 128-source tile
    (50, 256, 2, 520, 40),     # five l-tiles, 64-source tiles (double-buffered pairs)
    (60, 200, 2, 100, 130),    # one l-tile; two source tiles, the second ragged
    (96, 1000, 0, 1200, 256),  # ten l-tiles, lmin = 0, ragged last tau block
])
def test_paired_l_tiles_match_single_tiles(monkeypatch, mode, nk, ntau, lmin, lmax, M):
    """Two adjacent 128-multipole tiles per work item (each loaded and split
    source block multiplies both tables) against one tile per item, with
    l-tile 0 paired too (GCAMB_TC_CHAIN=0; its chain items are tested
    below).  Each
    (k, l-tile) product D_k is the same sequence of MMAs on the same operand
    bits and each k's term (w (D_hh + D_x))^2 the same FP32 value; only the
    k-chunks over which the epilogue sums the terms in FP32 differ.  A chunk
    sum of at most 16 positive terms is within 15 * 2^-24 of exact (relative),
    and the reduce adds the chunks nearly exactly, so the two C_l agree within
    2 * 16 * 2^-24.  The uniform plan of the same batch runs the paired kernel
    and gives the paired result bit for bit."""
    k, tau, S, P = case(nk, ntau, lmin, lmax, M)
    monkeypatch.setenv("GCAMB_TC_CHAIN", "0")  # l-tile 0 paired as well: the same MMA sequences
    monkeypatch.setenv("GCAMB_TC_LP", "1")
    C1, g = run(k, tau, S, P, lmin, lmax, mode)
    monkeypatch.delenv("GCAMB_TC_LP", raising=False)
    C2, _ = run(k, tau, S, P, lmin, lmax, mode, g)
    assert np.all(np.isfinite(C2)) and np.all(C1 > 0)
    assert (np.abs(C2 - C1) / C1).max() <= 2 * 16 * 2.0 ** -24
    plan = gcamb.plan_create(g, M, mode=mode)
    info = gcamb.plan_info(plan)
    assert info["fused"] == 1 and info["lp"] == 2
    C3 = gcamb.plan_launch(plan, torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda")).cpu().numpy()
    gcamb.sync()
    assert np.array_equal(C3, C2)


@pytest.mark.parametrize("mode", [gcamb.BF16X3, gcamb.F16X3])
@pytest.mark.parametrize("nk,ntau,lmin,lmax,M", [
    (70, 333, 2, 300, 100),   # split pass (ntau % 4 != 0), three l-tiles, 128-source tile
    (50, 256, 2, 520, 40),    # five l-tiles, 64-source tiles
])
def test_split_pass_paired_l_tiles_match_single_tiles(monkeypatch, mode, nk, ntau, lmin, lmax, M):
    """The split-pass kernel (sources split by a separate pass) with two
    l-tiles per item against one tile per item: the bound of the fused test."""
    k, tau, S, P = case(nk, ntau, lmin, lmax, M)
    monkeypatch.setenv("GCAMB_TC_FUSED", "0")
    monkeypatch.setenv("GCAMB_TC_CHAIN", "0")
    monkeypatch.setenv("GCAMB_TC_LP", "1")
    C1, g = run(k, tau, S, P, lmin, lmax, mode)
    monkeypatch.delenv("GCAMB_TC_LP", raising=False)
    C2, _ = run(k, tau, S, P, lmin, lmax, mode, g)
    assert np.all(np.isfinite(C2)) and np.all(C1 > 0)
    assert (np.abs(C2 - C1) / C1).max() <= 2 * 16 * 2.0 ** -24
    info = gcamb.plan_info(gcamb.plan_create(g, M, mode=mode))
    assert info["fused"] == 0 and info["lp"] == 2


@pytest.mark.parametrize("chain", ["1", "2"])
@pytest.mark.parametrize("mode,fused", [(gcamb.F16X3, "1"), (gcamb.BF16X3, "1"), (gcamb.F16X3, "0")])
def test_chain_records_cut_the_accumulation_loss_at_low_l(orc, monkeypatch, mode, fused, chain):
    """The tensor cores add each MMA's products to the FP32 accumulator after
    dropping their bits below a quarter ulp of the largest term, and truncate
    the sum; the loss of every accumulate step is relative to the running sum
    and always towards zero.  On long same-sign tau sums (low l, small k) it
    builds up to a bias of several 1e-6.  Chain records spread a tile's
    hi*hi products over three accumulators, each holding about a third of
    the sum: at every k where an item's second l-tile is idle (chain 1, the
    default), and in addition at every k of l-tile 0 (chain 2).  The error
    at l < 30 must fall (mean over sources and l, to at most 0.6 of the
    single-accumulator error) and stay within 1e-5 on every l; the results
    differ by no more than the single accumulator's error."""
    k, tau, S, P = case(160, 1000, 2, 300, 64, seed=7)
    monkeypatch.setenv("GCAMB_TC_FUSED", fused)
    monkeypatch.setenv("GCAMB_TC_CHAIN", "0")
    C0, g = run(k, tau, S, P, 2, 300, mode)
    monkeypatch.setenv("GCAMB_TC_CHAIN", chain)
    C3, _ = run(k, tau, S, P, 2, 300, mode, g)
    info = gcamb.plan_info(gcamb.plan_create(g, 64, mode=mode))
    assert info["lp"] == 2
    sel = [0, 9, 21, 33, 47, 63]
    _, Cr = orc.los_cl(k, tau, 14000.0, 2, 300, S[sel].astype(np.float64), P[sel], want_delta=False)
    e0 = np.abs(C0[sel] / Cr - 1)
    e3 = np.abs(C3[sel] / Cr - 1)
    low = slice(0, 28)
    assert e3[:, low].mean() <= 0.6 * e0[:, low].mean(), (e3[:, low].mean(), e0[:, low].mean())
    assert e3.max() <= (1e-5 if mode == gcamb.F16X3 else 6 * 2.0 ** -16), e3.max()
    assert (np.abs(C3 - C0) / C0).max() <= 2 * max(e0.max(), 1e-6)


@pytest.mark.parametrize("mode,fused", [(gcamb.F16X3, "1"), (gcamb.BF16X3, "1"), (gcamb.F16X3, "0")])
@pytest.mark.parametrize("nk,ntau,lmin,lmax,M", [
    (2000, 256, 2, 1200, 200),  # items of ~33 k hold several 16-k chunks; two 128-source tiles
    (4000, 128, 2, 1000, 40),   # ~26 k per item, 64-source tile
])
def test_k_sum_in_chunks_of_16_against_exact_sum_of_the_terms(monkeypatch, mode, fused, nk, ntau, lmin, lmax, M):
    """Eq. (1)'s k-sum on the batched path.  The epilogue adds each k's term
    (w_k D_k)^2 to an FP32 sum that it writes out every 16 non-empty k (the
    FP32 accumulation of at most 16 positive terms is within 15 * 2^-24 of
    their exact sum, relative); the reduce adds those chunk sums as TwoSum
    pairs and reads them out in FP64 (within ~n^2 2^-48).  With
    GCAMB_TC_KSUB=1 every k's term is its own partial, so the reduce's result
    is the FP64 sum of the FP32-rounded terms: the default must be within
    (15 + 1) * 2^-24 of it (the one extra 2^-24: the rounding of each term
    there, which the fused multiply-add of the chunk sum does not make).
    GCAMB_TC_KSUB=64, the longest chunk, must be within 64 * 2^-24.  Items of
    equal cost (GCAMB_TC_KALIGN=0), so that an item spans several chunks; the
    default k-aligned items (12 k) hold one chunk each."""
    k, tau, S, P = case(nk, ntau, lmin, lmax, M)
    monkeypatch.setenv("GCAMB_TC_KALIGN", "0")
    monkeypatch.setenv("GCAMB_TC_FUSED", fused)
    monkeypatch.setenv("GCAMB_TC_KSUB", "1")
    C1, g = run(k, tau, S, P, lmin, lmax, mode)
    monkeypatch.delenv("GCAMB_TC_KSUB", raising=False)
    C16, _ = run(k, tau, S, P, lmin, lmax, mode, g)
    monkeypatch.setenv("GCAMB_TC_KSUB", "64")
    C64, _ = run(k, tau, S, P, lmin, lmax, mode, g)
    assert np.all(C1 > 0) and np.all(np.isfinite(C16))
    assert (np.abs(C16 - C1) / C1).max() <= 16 * 2.0 ** -24
    assert (np.abs(C64 - C1) / C1).max() <= 64 * 2.0 ** -24
    assert not np.array_equal(C16, C64)  # the chunk length reaches the kernel


@pytest.mark.parametrize("mode", [gcamb.F16X3, gcamb.BF16X3])
def test_k_aligned_items_match_equal_cost_items(monkeypatch, mode):
    """Work items cut at multiples of 12 k (the default for a uniform batch)
    against items of equal cost (GCAMB_TC_KALIGN=0): every (k, l-tile)
    product is the same MMA sequence and every k's term the same FP32 value;
    only the chunks the epilogue sums in FP32 differ (at most 16 terms each,
    within 15 * 2^-24), so the C_l agree within 2 * 16 * 2^-24."""
    k, tau, S, P = case(300, 200, 2, 500, 200)
    monkeypatch.setenv("GCAMB_TC_KALIGN", "0")
    C0, g = run(k, tau, S, P, 2, 500, mode)
    monkeypatch.delenv("GCAMB_TC_KALIGN", raising=False)
    C12, _ = run(k, tau, S, P, 2, 500, mode, g)
    monkeypatch.setenv("GCAMB_TC_KALIGN", "5")
    C5, _ = run(k, tau, S, P, 2, 500, mode, g)
    assert np.all(C0 > 0) and np.all(np.isfinite(C12)) and np.all(np.isfinite(C5))
    assert (np.abs(C12 - C0) / C0).max() <= 2 * 16 * 2.0 ** -24
    assert (np.abs(C5 - C0) / C0).max() <= 2 * 16 * 2.0 ** -24
    assert not np.array_equal(C12, C0)  # the cut reaches the work list


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
    # sources read in place by TMA must start on a 16-byte boundary: refused on the host
    buf = torch.empty(St.numel() + 1, dtype=torch.float32, device="cuda")
    Smis = buf[1:].view(St.shape)
    Smis.copy_(St)
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.los_cl(g, Smis, Pt, gcamb.BF16X3)
    assert ei.value.code == gcamb.EINVAL and "16-byte" in str(ei.value)


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
    sel = list(range(0, 256, 8)) + [255] if mode == gcamb.F16X3 else [0, 97, 255]
    _, Cr = orc.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, S[sel].double().cpu().numpy(),
                       P[sel].cpu().numpy(), want_delta=False)
    err = np.abs(C[sel] / Cr - 1)
    assert err.max() <= 1e-5, err.max()


@pytest.mark.parametrize("mode", [gcamb.F16X3, gcamb.BF16X3, gcamb.TF32X3, gcamb.PLAIN64])
def test_compressed_table_gives_the_same_bits(monkeypatch, mode):
    """A table in compressible device memory (the library's default where the
    device supports it) and one from cudaMalloc (GCAMB_TABLE_COMPRESS=0) give
    bit-identical results: compression changes only how the memory system
    moves the zero-padded blocks between DRAM and L2."""
    k, tau, S, P = case(160, 1000, 2, 700, 64, seed=5)
    out = {}
    for env in ("1", "0"):
        monkeypatch.setenv("GCAMB_TABLE_COMPRESS", env)
        g = gcamb.grid_create(k, tau, 14000.0, 2, 700)
        gcamb.bessel_table(g, mode)
        comp = gcamb.table_compressed(g, mode)
        if mode == gcamb.PLAIN64:
            D = gcamb.los_transfer(g, torch.as_tensor(S.astype(np.float64), device="cuda"), mode)
            C = gcamb.cl(g, D, torch.as_tensor(P, device="cuda"))
        else:
            C = gcamb.los_cl(g, torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda"), mode)
        gcamb.sync()
        out[env] = (C.cpu().numpy(), comp)
        gcamb.grid_destroy(g)
    assert not out["0"][1], "GCAMB_TABLE_COMPRESS=0 must give a plain allocation"
    print("table compressed by default: %s" % out["1"][1])
    assert np.array_equal(out["1"][0], out["0"][0])
