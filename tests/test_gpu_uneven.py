"""GPU parity of plans (uneven batches: per-source l_max and k prefix on one
shared grid, one persistent kernel replayed from a CUDA graph, autotuned
source tiles) against the FP64 oracle run on each source's own grid.

Each source m is checked against the oracle on k[0..nk_m) (trapezoid in ln k
on that prefix) and l <= lmax_m; C_l above lmax_m must be exactly zero.
Tolerance: 1e-5 relative (F16X3, and the FP32 plans of the plain kernels),
as for the uniform batched path."""
import os

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


def uneven_batch(M, nk, lmax_lo, lmax_hi, seed):
    p = synth.model_params(M, seed=seed, lmax_range=(lmax_lo, lmax_hi))
    lm = p.lmax.astype(np.int32)
    nkm = np.clip(np.rint(nk / 3 + (nk - nk / 3) * (lm - lmax_lo) / max(1, lmax_hi - lmax_lo)), 1, nk).astype(np.int32)
    return p, lm, nkm


def check_against_oracle(orc, k, tau, tau0, lmin, C, S, P, lm, nkm, sel, tol=TOL):
    for m in sel:
        q = int(nkm[m])
        L = int(lm[m])
        _, cr = orc.los_cl(k[:q], tau, tau0, lmin, L, S[m, :q].astype(np.float64), P[m, :q], want_delta=False)
        got = C[m, :L - lmin + 1]
        err = np.abs(got / cr - 1)
        assert err.max() <= tol, (m, L, q, err.max())
        assert np.all(C[m, L - lmin + 1:] == 0.0)


def test_uneven_batch_matches_oracle(orc):
    nk, ntau, lmin, lmax, M = 60, 200, 2, 500, 70
    k = synth.master_linear_k(nk, 0.05)
    tau = synth.uniform_grid(200.0, 14000.0, ntau)
    p, lm, nkm = uneven_batch(M, nk, 100, lmax, seed=21)
    S = synth.sources(k, tau, p).astype(np.float32)
    P = synth.primordial(k, p)
    g = gcamb.grid_create(k, tau, 14000.0, lmin, lmax)
    gcamb.bessel_table(g, gcamb.F16X3)
    plan = gcamb.plan_create(g, M, lm, nkm, gcamb.F16X3)
    C = gcamb.plan_launch(plan, torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda"))
    gcamb.sync()
    C = C.cpu().numpy()
    order = np.argsort(lm)
    sel = sorted({int(order[0]), int(order[-1]), int(order[M // 2]), 3, 17, 44})
    check_against_oracle(orc, k, tau, 14000.0, lmin, C, S, P, lm, nkm, sel)


@pytest.mark.parametrize("mode", [gcamb.BF16X3, gcamb.F16X3])
def test_uneven_paired_l_tiles_match_single_tiles(monkeypatch, orc, mode):
    """An uneven plan with two adjacent l-tiles per work item (the split
    sources loaded once for both tables; a source tile whose largest l_max
    stops before the second tile gets one-tile items) against the same plan
    with one tile per item.  Each (k, l-tile) product is the same MMA
    sequence (l-tile 0 paired too: GCAMB_TC_CHAIN=0); only the k-chunks of
    the FP32 sums differ, so the C_l agree within 2 * 16 * 2^-24 relative,
    and exactly where a source's l_max ends.
    Against the oracle: 1e-5 for F16X3, BF16X3's bound on coarse grids
    6 * 2^-16 (its 16-bit split; see the batched tests)."""
    nk, ntau, lmin, lmax, M = 60, 200, 2, 700, 300
    k = synth.master_linear_k(nk, 0.05)
    tau = synth.uniform_grid(200.0, 14000.0, ntau)
    p, lm, nkm = uneven_batch(M, nk, 100, lmax, seed=24)
    S = torch.as_tensor(synth.sources(k, tau, p).astype(np.float32), device="cuda")
    P = torch.as_tensor(synth.primordial(k, p), device="cuda")
    g = gcamb.grid_create(k, tau, 14000.0, lmin, lmax)
    gcamb.bessel_table(g, mode)
    monkeypatch.setenv("GCAMB_TC_CHAIN", "0")  # l-tile 0 paired as well: the same MMA sequences
    monkeypatch.setenv("GCAMB_TC_LP", "1")
    plan1 = gcamb.plan_create(g, M, lm, nkm, mode)
    assert gcamb.plan_info(plan1)["lp"] == 1
    C1 = gcamb.plan_launch(plan1, S, P).cpu().numpy()
    monkeypatch.delenv("GCAMB_TC_LP", raising=False)
    plan2 = gcamb.plan_create(g, M, lm, nkm, mode)
    info = gcamb.plan_info(plan2)
    assert info["lp"] == 2 and info["fused"] == 0
    C2 = gcamb.plan_launch(plan2, S, P).cpu().numpy()
    gcamb.sync()
    live = C1 != 0
    assert np.array_equal(live, C2 != 0)
    assert (np.abs(C2[live] - C1[live]) / np.abs(C1[live])).max() <= 2 * 16 * 2.0 ** -24
    sel = [int(np.argmin(lm)), int(np.argmax(lm)), 5, 150]
    check_against_oracle(orc, k, tau, 14000.0, lmin, C2, S.cpu().numpy(), P.cpu().numpy(), lm, nkm, sel,
                         tol=TOL if mode == gcamb.F16X3 else 6 * 2.0 ** -16)


def test_uneven_plain32_plan_matches_oracle(orc):
    """The FP32 form of the uneven batch: a plan in GCAMB_PLAIN32 runs the
    plain CUDA-core kernels on chunks of sources, each summed over its own k
    prefix (trapezoid in ln k on the prefix) and zero above its own l_max;
    captured once in a CUDA graph and replayed.  Against the oracle on the
    FP32-rounded sources: 1e-5 relative, every source checked."""
    nk, ntau, lmin, lmax, M = 60, 200, 2, 500, 37
    k = synth.master_linear_k(nk, 0.05)
    tau = synth.uniform_grid(200.0, 14000.0, ntau)
    p, lm, nkm = uneven_batch(M, nk, 100, lmax, seed=25)
    S = synth.sources(k, tau, p).astype(np.float32)
    P = synth.primordial(k, p)
    g = gcamb.grid_create(k, tau, 14000.0, lmin, lmax)
    gcamb.bessel_table(g, gcamb.PLAIN32)
    plan = gcamb.plan_create(g, M, lm, nkm, gcamb.PLAIN32)
    St, Pt = torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda")
    C1 = gcamb.plan_launch(plan, St, Pt)
    C1 = C1.cpu().numpy()
    C2 = gcamb.plan_launch(plan, St, Pt).cpu().numpy()
    gcamb.sync()
    info = gcamb.plan_info(plan)
    assert info["captures"] == 1 and info["replays"] == 2 and info["tile"] == 0
    assert np.array_equal(C1, C2)
    check_against_oracle(orc, k, tau, 14000.0, lmin, C1, S, P, lm, nkm, range(M))


def test_uniform_plain32_plan_equals_plain_path():
    k = synth.log_grid(1e-4, 0.3, 50)
    tau = synth.uniform_grid(200.0, 14000.0, 300)
    M = 20
    p = synth.model_params(M, seed=26)
    S = torch.as_tensor(synth.sources(k, tau, p).astype(np.float32), device="cuda")
    P = torch.as_tensor(synth.primordial(k, p), device="cuda")
    g = gcamb.grid_create(k, tau, 14000.0, 2, 400)
    gcamb.bessel_table(g, gcamb.PLAIN32)
    ref = gcamb.cl(g, gcamb.los_transfer(g, S, gcamb.PLAIN32), P).cpu().numpy()
    got = gcamb.plan_launch(gcamb.plan_create(g, M, mode=gcamb.PLAIN32), S, P).cpu().numpy()
    gcamb.sync()
    assert np.array_equal(got, ref)


def test_uniform_plan_equals_los_cl():
    k = synth.log_grid(1e-4, 0.3, 80)
    tau = synth.uniform_grid(200.0, 14000.0, 300)
    M = 100
    p = synth.model_params(M, seed=22)
    S = torch.as_tensor(synth.sources(k, tau, p).astype(np.float32), device="cuda")
    P = torch.as_tensor(synth.primordial(k, p), device="cuda")
    g = gcamb.grid_create(k, tau, 14000.0, 2, 600)
    gcamb.bessel_table(g, gcamb.F16X3)
    ref = gcamb.los_cl(g, S, P, gcamb.F16X3).cpu().numpy()
    plan = gcamb.plan_create(g, M, mode=gcamb.F16X3)
    got = gcamb.plan_launch(plan, S, P).cpu().numpy()
    gcamb.sync()
    assert np.array_equal(got, ref)


def test_graph_replay_and_tuning(tmp_path, monkeypatch):
    monkeypatch.setenv("GCAMB_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    nk, ntau, lmin, lmax, M = 50, 250, 2, 400, 150
    k = synth.master_linear_k(nk, 0.04)
    tau = synth.uniform_grid(200.0, 14000.0, ntau)
    p, lm, nkm = uneven_batch(M, nk, 80, lmax, seed=23)
    S = torch.as_tensor(synth.sources(k, tau, p).astype(np.float32), device="cuda")
    P = torch.as_tensor(synth.primordial(k, p), device="cuda")
    g = gcamb.grid_create(k, tau, 14000.0, lmin, lmax)
    gcamb.bessel_table(g, gcamb.F16X3)
    plan = gcamb.plan_create(g, M, lm, nkm, gcamb.F16X3, tune=True)
    assert gcamb.plan_info(plan)["tile"] == 0  # not tuned yet
    ws = torch.empty(gcamb.plan_workspace(plan), dtype=torch.uint8, device="cuda")
    C = torch.empty((M, g.nl), dtype=torch.float64, device="cuda")
    gcamb.plan_launch(plan, S, P, C, ws)
    c1 = C.cpu().numpy()
    gcamb.plan_launch(plan, S, P, C, ws)
    gcamb.sync()
    c2 = C.cpu().numpy()
    info = gcamb.plan_info(plan)
    assert info["tuned"] == 1 and info["tile"] in (64, 128, 256)
    assert info["lp"] in (1, 2) and info["kalign"] in (0, 8, 16) and info["tail"] in (1, 10004)
    assert info["captures"] == 1 and info["replays"] == 2
    assert np.array_equal(c1, c2)
    # the cache line records the whole choice (width, tiles per item, tail, items per CTA)
    import json
    lines = [json.loads(x) for x in open(tmp_path / "tune.jsonl").read().splitlines()]
    assert len(lines) == 1
    rec = lines[0]
    assert rec["nt"] == info["tile"] and rec["lp"] == info["lp"] and rec["per_cta"] == info["items_per_cta"]
    assert rec["kalign"] == info["kalign"]
    assert round(rec["tail_frac"] * 1000) * 100 + rec["tail_parts"] == info["tail"]
    # the same batch again: the width comes from the cache, no timing
    plan2 = gcamb.plan_create(g, M, lm, nkm, gcamb.F16X3, tune=True)
    info2 = gcamb.plan_info(plan2)
    assert info2["tuned"] == 1 and info2["tile"] == info["tile"]
    assert (info2["lp"], info2["kalign"], info2["tail"]) == (info["lp"], info["kalign"], info["tail"])
    c3 = gcamb.plan_launch(plan2, S, P).cpu().numpy()
    gcamb.sync()
    assert np.array_equal(c3, c1)
    # and a heuristic plan agrees within the tolerance
    plan3 = gcamb.plan_create(g, M, lm, nkm, gcamb.F16X3)
    c4 = gcamb.plan_launch(plan3, S, P).cpu().numpy()
    gcamb.sync()
    nz = c1 != 0
    assert np.all(np.abs(c4[nz] / c1[nz] - 1) <= 2 * TOL)


def test_plan_argument_errors():
    k = synth.master_linear_k(20, 0.02)
    tau = synth.uniform_grid(200.0, 14000.0, 64)
    g = gcamb.grid_create(k, tau, 14000.0, 2, 100)
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.plan_create(g, 3, mode=gcamb.F16X3)
    assert ei.value.code == gcamb.ESTATE
    gcamb.bessel_table(g, gcamb.F16X3)
    for lm, nk in (([50, 101, 60], [5, 5, 5]), ([50, 60, 70], [0, 5, 5]), ([50, 1, 70], [5, 5, 5])):
        with pytest.raises(gcamb.GcambError) as ei:
            gcamb.plan_create(g, 3, lm, nk, gcamb.F16X3)
        assert ei.value.code == gcamb.EINVAL
    with pytest.raises(gcamb.GcambError) as ei:
        gcamb.plan_create(g, 3, mode=gcamb.PLAIN64)
    assert ei.value.code == gcamb.EINVAL


def test_uneven_lmax6000_full_size_sampled(orc):
    """The 1000-source uneven workload at full size: l_max ~ U{1500..6000}, k
    prefixes of 1000..3000 nodes of the 3000-node linear grid on (0, 0.5], 1000
    tau; tuned plan, graph launch; sampled sources against the oracle."""
    wl = synth.workload("uneven_lmax6000")
    M = wl.M
    p = synth.model_params(M, seed=0, lmax_range=(1500, 6000))
    lm = p.lmax.astype(np.int32)
    nkm = synth.uneven_nk(lm).astype(np.int32)
    S = synth.sources_torch(wl.k, wl.tau, p, "cuda", torch.float32, nk_per_model=nkm)
    P = torch.as_tensor(synth.primordial(wl.k, p), device="cuda")
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(g, gcamb.F16X3)
    plan = gcamb.plan_create(g, M, lm, nkm, gcamb.F16X3, tune=True)
    C = gcamb.plan_launch(plan, S, P)
    C = gcamb.plan_launch(plan, S, P, C).cpu().numpy()
    gcamb.sync()
    order = np.argsort(lm)
    sel = [int(order[0]), int(order[1])]  # the two smallest l_max (the oracle's cheapest)
    Sh = S[sel].cpu().numpy()
    Ph = P[sel].cpu().numpy()
    for j, m in enumerate(sel):
        q, L = int(nkm[m]), int(lm[m])
        _, cr = orc.los_cl(wl.k[:q], wl.tau, wl.tau0, wl.lmin, L, Sh[j, :q].astype(np.float64), Ph[j, :q],
                           want_delta=False)
        err = np.abs(C[m, :L - wl.lmin + 1] / cr - 1)
        assert err.max() <= TOL, (m, L, q, err.max())
        assert np.all(C[m, L - wl.lmin + 1:] == 0.0)



@pytest.mark.parametrize("mode", [gcamb.F16X3, gcamb.PLAIN32, gcamb.TF32X3, gcamb.BF16X3])
def test_uneven_high_multipoles_match_oracle(orc, mode):
    """Multipoles above 2500 in plans: an uneven batch (F16X3 on the tensor
    cores, and the FP32 plan of the plain kernels) with l_max ~
    U{2500..6000} on a coarse linear k grid to 0.5, each source's k prefix
    scaled with its l_max by the uneven workload's law (so
    that k_max (tau0 - tau_0) exceeds l_max: every multipole of a source has
    support), checked against the oracle at 1e-5 on every l of the sources
    of the smallest, the median and the largest l_max and two more, each on
    its own k prefix (BF16X3: its coarse-grid bound 6 * 2^-16)."""
    nk, ntau, lmin, lmax, M = 400, 300, 2, 6000, 40
    k = synth.master_linear_k(nk, 0.5)
    tau = synth.uniform_grid(200.0, 14000.0, ntau)
    p = synth.model_params(M, seed=33, lmax_range=(2500, lmax))
    lm = p.lmax.astype(np.int32)
    nkm = np.rint(synth.uneven_nk(lm) * nk / 3000.0).astype(np.int32)
    assert np.all(k[nkm - 1] * (14000.0 - tau[0]) > lm)
    S = synth.sources(k, tau, p).astype(np.float32)
    P = synth.primordial(k, p)
    g = gcamb.grid_create(k, tau, 14000.0, lmin, lmax)
    gcamb.bessel_table(g, mode)
    plan = gcamb.plan_create(g, M, lm, nkm, mode)
    C = gcamb.plan_launch(plan, torch.as_tensor(S, device="cuda"), torch.as_tensor(P, device="cuda"))
    gcamb.sync()
    C = C.cpu().numpy()
    order = np.argsort(lm, kind="stable")
    sel = sorted({int(order[0]), int(order[M // 2]), int(order[-1]), 5, 29})
    assert lm[order[-1]] > 5000
    check_against_oracle(orc, k, tau, 14000.0, lmin, C, S, P, lm, nkm, sel,
                         tol=6 * 2.0 ** -16 if mode == gcamb.BF16X3 else TOL)
