"""Training recipe for the C_l emulator (library kernels only).

1. Draw parameters of the synthetic source family (paper_2509_25110_gb300.synth),
   regenerate their sources on the device (gcamb_synth_sources) and compute
   their spectra with the batched projection (gcamb_los_cl): the training set
   and a held-out set.
2. Fit the normalisation, then train the MLP with Adam (gcamb_emu_train_step)
   on shuffled mini-batches, the learning rate following a cosine from lr0 to
   lr_min.
3. Check it on the held-out spectra (gcamb_emu_check): cells of parameter
   space where every held-out spectrum is within tol are served by the
   network, the rest by the projection (gcamb_emulate).

The paper builds no emulator; it motivates fast spectra as emulator training
sets (Sec. 1, Sec. 5).  This module only sequences the library's calls.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import gcamb, synth


def make_dataset(g, n, seed, mode=gcamb.F16X3, batch=256, first_model=0):
    """Features X[n][9] (device float32) and spectra C[n][nl] (device float64)."""
    import torch
    p = synth.model_params(n, seed=seed, first_model=first_model)
    X = torch.as_tensor(synth.emulator_features(p), device="cuda")
    C = torch.empty((n, g.nl), dtype=torch.float64, device="cuda")
    gcamb.bessel_table(g, mode)
    ws = None
    S = P = None
    for a in range(0, n, batch):
        b = min(n, a + batch)
        S, P = gcamb.synth_sources(g, X[a:b].contiguous())
        if ws is None or b - a != batch:
            ws = torch.empty(gcamb.los_cl_workspace(g, b - a, mode), dtype=torch.uint8, device="cuda")
        C[a:b] = gcamb.los_cl(g, S, P, mode, ws=ws)
    gcamb.sync()
    return X, C


def train(g, n_train=100_000, n_hold=4096, steps=10000, batch=4096, width=512, depth=3, lr0=2e-3, lr_min=1e-5,
          tol=1e-3, min_count=32, seed=0, per_l=False, log=None, data=None):
    """Trains an emulator on grid g; returns (emu, report)."""
    import torch
    rep = {"n_train": n_train, "n_hold": n_hold, "steps": steps, "batch": batch, "width": width, "depth": depth}
    t0 = time.perf_counter()
    if data is None:
        X, C = make_dataset(g, n_train, seed=seed)
        Xh, Ch = make_dataset(g, n_hold, seed=seed + 1)
    else:
        X, C, Xh, Ch = data
    rep["data_s"] = time.perf_counter() - t0
    e = gcamb.emu_create(g, width=width, depth=depth, max_batch=max(batch, n_hold), seed=seed + 7)
    Y = gcamb.emu_fit_norm(e, X, C, per_l=per_l)
    rng = np.random.default_rng(seed + 11)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    perm = None
    pos = n_train
    hist = []
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for s in range(steps):
        if pos + batch > n_train:
            perm = torch.as_tensor(rng.permutation(n_train).astype(np.int32), device="cuda")
            pos = 0
        idx = perm[pos:pos + batch]
        pos += batch
        lr = lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * s / max(1, steps - 1)))
        gcamb.emu_train_step(e, X, Y, idx, batch, lr, loss)
        if s % max(1, steps // 20) == 0 or s == steps - 1:
            hist.append((s, float(loss.item())))
            if log:
                log("step %d loss %.3e lr %.2e" % (s, hist[-1][1], lr))
    torch.cuda.synchronize()
    rep["train_s"] = time.perf_counter() - t1
    rep["train_step_ms"] = 1e3 * rep["train_s"] / steps
    rep["loss_history"] = hist
    rep["check"] = gcamb.emu_check(e, Xh, Ch, tol=tol, min_count=min_count)
    rep["tol"] = tol
    return e, rep, (Xh, Ch)


def accuracy(e, Xh, Ch, lmin=2):
    """Held-out accuracy of the network alone: |C_net / C_ref - 1| per
    (spectrum, l), summarised (the amplitude term is zero on data of one A_s)."""
    import torch
    Y = gcamb.emu_forward(e, Xh)
    nrm = gcamb.emu_norm(e)
    gcamb.sync()
    x8 = Xh[:, 8].double().cpu().numpy()[:, None] - float(nrm["mu_x"][8])
    logc = Y.cpu().numpy().astype(np.float64) * nrm["sd_y"] + nrm["mu_y"] + x8
    err = np.abs(np.exp(logc) / Ch.cpu().numpy() - 1.0)
    per = err.max(axis=1)
    l = np.arange(lmin, lmin + err.shape[1])
    out = {"median": float(np.median(err)), "p99": float(np.quantile(err, 0.99)),
           "spectrum_max_p50": float(np.median(per)), "spectrum_max_p90": float(np.quantile(per, 0.9)),
           "frac_elements_within_1e-3": float((err <= 1e-3).mean())}
    for a, b in ((2, 30), (30, 500), (500, 1500), (1500, 2501)):
        sel = (l >= a) & (l < b)
        if sel.any():
            out["median_l%d-%d" % (a, b - 1)] = float(np.median(err[:, sel]))
    return out


def served_by_tolerance(e, Xh, Ch, tols=(1e-3, 3e-3, 1e-2, 3e-2, 1e-1), min_count=32):
    """Fraction of held-out requests the network would serve at each tolerance
    (the check is re-run per tolerance; the last one stays in force)."""
    return {"%g" % t: gcamb.emu_check(e, Xh, Ch, tol=t, min_count=min_count)["frac_served"] for t in tols}


def serve_rates(e, g, Xh, reps=5):
    """Spectra per second: the emulator on Xh (trusted and fallback as they
    fall), the network alone (every populated cell trusted), the batched
    projection on 256 of the same sources (inputs ready), and the method
    without the network as the fallback runs it (sources regenerated from
    the features, then projected)."""
    import torch
    B = Xh.shape[0]
    Cl = torch.empty((B, g.nl), dtype=torch.float64, device="cuda")
    fb = torch.empty(B, dtype=torch.int32, device="cuda")
    gcamb.emulate(e, Xh, Cl, fb)
    gcamb.sync()
    t0 = time.perf_counter()
    for _ in range(reps):
        gcamb.emulate(e, Xh, Cl, fb)
    gcamb.sync()
    mixed = reps * B / (time.perf_counter() - t0)
    served = 1.0 - float(fb.float().mean().item())
    S, P = gcamb.synth_sources(g, Xh[:256].contiguous())
    ws = torch.empty(gcamb.los_cl_workspace(g, 256, gcamb.F16X3), dtype=torch.uint8, device="cuda")
    C = gcamb.los_cl(g, S, P, gcamb.F16X3, ws=ws)
    gcamb.sync()
    t0 = time.perf_counter()
    for _ in range(reps):
        gcamb.los_cl(g, S, P, gcamb.F16X3, C, ws)
    gcamb.sync()
    proj = reps * 256 / (time.perf_counter() - t0)
    # the method without the network, as the fallback runs it: the sources
    # regenerated from the request's features, then the projection
    Xs = Xh[:256].contiguous()
    gcamb.sync()
    t0 = time.perf_counter()
    for _ in range(reps):
        S2, P2 = gcamb.synth_sources(g, Xs, S, P)
        gcamb.los_cl(g, S2, P2, gcamb.F16X3, C, ws)
    gcamb.sync()
    proj_src = reps * 256 / (time.perf_counter() - t0)
    Y = gcamb.emu_forward(e, Xh)
    gcamb.sync()
    t0 = time.perf_counter()
    for _ in range(reps):
        gcamb.emu_forward(e, Xh, Y)
    gcamb.sync()
    net = reps * B / (time.perf_counter() - t0)
    return {"emulate_spectra_per_s": mixed, "served_fraction": served, "network_spectra_per_s": net,
            "projection_spectra_per_s": proj, "sources_and_projection_spectra_per_s": proj_src}
