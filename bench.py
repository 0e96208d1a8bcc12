#!/usr/bin/env python
"""Benchmark of the batched split-precision line-of-sight path.

Metric: C_l spectra per second at l_max = 2500 (batched split precision vs
plain FP64, relative error <= 1e-5), on the batched workload: 256 sources
sharing one grid, l = 2..2500, 2000 k log-spaced on [1e-4, 0.3] 1/Mpc, 1000
tau uniform on [200, 14000] Mpc, synthetic sources (paper_2509_25110_gb300.synth).

One step = one pass of the batched path over one batch of 256 sources
(gcamb_los_cl): the epilogue weights (and, for fp16, the sources' row
scales), the tensor-core kernel that splits the FP32 sources into hi/lo
planes in shared memory and does the tau-contraction + square + k-chunk sum,
and the FP64 reduction to C_l.  The grid's Bessel table is
built once per grid before the timed region (its build time is reported in
`config`).  Inputs (2.0 GB of sources, a 3.3 GB table) are larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode bf16x3|f16x3|tf32x3]
  python bench.py --impl reference ...   (the FP64 CPU oracle, timed on the host)

Under torchrun every rank runs its own batch (weak scaling, no collective on
the data path); the timed region is bracketed by a barrier and the maximum
over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "C_l spectra/sec at l_max=2500: batched split-precision vs plain FP64, rel err ≤1e-5"
WORKLOAD = "batched_lmax2500"
ORACLE_GROUP = 16  # sources per oracle call (its per-(k, tau) j_l is shared by them)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="f16x3")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-models", type=int, default=256,
                    help="sources of the timed batch checked against the oracle (default: all 256)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nk", type=int, default=0,
                    help="profiling case: the same k range with this many nodes (default: the workload's 2000)")
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "uneven", "emulator", "te", "tensor", "features", "lsampled", "curved",
                             "plain"],
                    help="batched (the headline), uneven (1000 sources, l_max <= 6000, plan + graph), "
                         "emulator (train on 100k spectra, serve)")
    ap.add_argument("--sources", type=int, default=0,
                    help="uneven workload: the first N of its 1000 sources (profiling case)")
    ap.add_argument("--no-tune", action="store_true", help="uneven workload: the heuristic tile, no timing of candidates")
    ap.add_argument("--kernel-only", action="store_true",
                    help="profiling case: only warm-up + timed steps, one short line, no e2e/plain/CPU legs")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = (bus_id or "").lower()
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.25)

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 10]
        if self.bus_id:
            mine = [r for r in rows if self.bus_id[-12:] in r[1].lower()]
            rows = mine or rows
        if not rows:
            return None
        idx = rows[0][0]
        rows = [r for r in rows if r[0] == idx]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[2]) for r in rows]
        smax = max(num(r[3]) for r in rows)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[j] for r in rows for j in range(4) if r[6 + j].lower().startswith("active")})
        loaded = [s for s in sm if s == s]
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax,
                "power_w_max": max(num(r[4]) for r in rows), "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    """The FP64 CPU oracle as it stands, on host cores, one bounded sample per
    step: 16 sources of the batch on a subset of the k nodes (the oracle's
    cost is linear in the k nodes; 16 sources share each (k, tau) Bessel
    evaluation, as in each oracle call of the GPU arm's accuracy check)."""
    import numpy as np

    import oracle
    from oracle import build as ob
    from paper_2509_25110_gb300 import synth

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ob.build()
    wl = synth.workload(WORKLOAD)
    p = synth.model_params(ORACLE_GROUP, seed=0)

    def inputs(qs):  # FP32-rounded sources and P(k) of the batch's first sources on the k nodes qs
        return (synth.sources(wl.k[qs], wl.tau, p).astype(np.float32).astype(np.float64),
                synth.primordial(wl.k[qs], p))
    # per step: sized so that warm-up + steps finish in about two minutes
    budget = 120.0 / max(1, args.steps + args.warmup)
    nks = 32
    while True:
        qs = np.unique(np.linspace(0, wl.nk - 1, nks).astype(int))
        S, P = inputs(qs)
        t0 = time.perf_counter()
        oracle.los_cl(wl.k[qs], wl.tau, wl.tau0, wl.lmin, wl.lmax, S, P, want_delta=False)
        dt = time.perf_counter() - t0
        if dt <= budget or nks <= 2:
            break
        nks = max(2, int(nks * budget / dt * 0.8))
    spectra = ORACLE_GROUP * qs.size / wl.nk
    for _ in range(args.warmup):
        oracle.los_cl(wl.k[qs], wl.tau, wl.tau0, wl.lmin, wl.lmax, S, P, want_delta=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.los_cl(wl.k[qs], wl.tau, wl.tau0, wl.lmin, wl.lmax, S, P, want_delta=False)
    dt = time.perf_counter() - t0
    value = spectra * args.steps / dt
    cores = oracle.num_threads()
    sample = "%d sources x %d of %d k nodes per step (%.2f spectra), all %d tau, l %d..%d" % (
        ORACLE_GROUP, qs.size, wl.nk, spectra, wl.ntau, wl.lmin, wl.lmax)
    q16 = np.unique(np.linspace(0, wl.nk - 1, 16).astype(int))
    S16, P16 = inputs(q16)
    one = oracle_sample_rates(wl, S16, P16, q16)
    line = {
        "metric": METRIC, "value": value, "unit": "spectra/s", "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "M": wl.M, "lmax": wl.lmax, "nk": wl.nk, "ntau": wl.ntau,
                   "reference": "FP64 CPU oracle (oracle/gcamb_oracle.c), dense tau sums"},
        "cpu_baseline": {"value": value, "unit": "spectra/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "same_sample_1_core_vs_all": one},
        "e2e": {"value": value, "unit": "spectra/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def committed_traffic(name, mode):
    """DRAM bytes per launch of the tensor-core kernel from the committed ncu
    summary `profiles/<name>`, or None once tc.cu has changed since it was
    taken (the summary records tc.cu's SHA-1)."""
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", name)) as f:
            tr = json.load(f)
        src = open(os.path.join(ROOT, "paper_2509_25110_gb300", "csrc", "tc.cu"), "rb").read()
        if tr.get("tc_cu_sha1") == hashlib.sha1(src).hexdigest() and tr.get("mode") == mode:
            return tr["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def host_numa(dev, t):
    """NUMA node of the GPU (its PCI function) and of the pages of a pinned
    host tensor (move_pages with no target: the query form), or None."""
    out = {"gpu_node": None, "buffer_node": None}
    try:
        import torch
        bus = torch.cuda.get_device_properties(dev).pci_bus_id.lower()
        dom, rest = bus.split(":", 1)
        path = "/sys/bus/pci/devices/%04x:%s/numa_node" % (int(dom, 16), rest)
        out["gpu_node"] = int(open(path).read().strip())
    except Exception:
        pass
    try:
        import ctypes
        libc = ctypes.CDLL(None, use_errno=True)
        pages = (ctypes.c_void_p * 1)(t.data_ptr())
        status = (ctypes.c_int * 1)(-1)
        nr = {"aarch64": 239, "x86_64": 279}.get(os.uname().machine)
        if nr is not None and libc.syscall(nr, 0, 1, pages, None, status, 0) == 0:
            out["buffer_node"] = int(status[0])
    except Exception:
        pass
    return out


def l_range_errors(rel, lmin, lmax):
    """Max relative error over [sources] within each multipole range."""
    import numpy as np
    ls = np.arange(lmin, lmax + 1)
    out = {}
    for a, b in ((2, 30), (30, 500), (500, 1500), (1500, lmax + 1)):
        sel = (ls >= a) & (ls < b)
        if sel.any():
            out["[%d,%d]" % (a, b - 1)] = float(rel[:, sel].max())
    return out


def oracle_sample_rates(wl, S, P, qs):
    """The oracle on sources S [M][qs][ntau] and P [M][qs] at the k nodes qs
    of the grid, at one thread and at all threads; rates in spectra/s (the
    fraction of a spectrum the sample covers, per second)."""
    import oracle
    spectra = S.shape[0] * qs.size / wl.nk
    out = {"sample": "%d sources x %d of %d k nodes (%.2f spectra), all %d tau, l %d..%d"
                     % (S.shape[0], qs.size, wl.nk, spectra, wl.ntau, wl.lmin, wl.lmax)}
    for name, nt in (("one_core", 1), ("all_cores", 0)):
        t0 = time.perf_counter()
        oracle.los_cl(wl.k[qs], wl.tau, wl.tau0, wl.lmin, wl.lmax, S, P, want_delta=False, nthreads=nt)
        dt = time.perf_counter() - t0
        out[name] = {"value": spectra / dt, "unit": "spectra/s", "cores": 1 if nt == 1 else oracle.num_threads(),
                     "seconds": dt}
    return out


# ------------------------------------------------------------------ other workloads

def _timed_region(fn, steps, dev):
    import torch
    bus = None
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id
    except Exception:
        pass
    sampler = ClockSampler(bus)
    torch.cuda.synchronize()
    sampler.start()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b), sampler.stop()


def run_uneven(args):
    """1000 sources with l_max ~ U{1500..6000} and k prefixes of 1000..3000
    nodes of a 3000-node linear grid, 1000 tau: one tuned plan, replayed from
    its CUDA graph (one persistent tensor-core kernel per launch)."""
    import numpy as np
    import torch

    from paper_2509_25110_gb300 import build, gcamb, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    mode = {"bf16x3": gcamb.BF16X3, "tf32x3": gcamb.TF32X3, "f16x3": gcamb.F16X3,
            "plain32": gcamb.PLAIN32}[args.mode]
    wl = synth.workload("uneven_lmax6000")
    if args.sources:
        wl.M = min(wl.M, args.sources)
    p = synth.model_params(wl.M, seed=0, lmax_range=(1500, 6000))
    lm = p.lmax.astype(np.int32)
    nkm = synth.uneven_nk(lm).astype(np.int32)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    t0 = time.perf_counter()
    gcamb.bessel_table(g, mode)
    torch.cuda.synchronize()
    table_s = time.perf_counter() - t0
    X = torch.as_tensor(synth.emulator_features(p), device=dev)
    S, P = gcamb.synth_sources(g, X)
    plan = gcamb.plan_create(g, wl.M, lm, nkm, mode, tune=not args.no_tune)
    ws = torch.empty(gcamb.plan_workspace(plan), dtype=torch.uint8, device=dev)
    C = torch.empty((wl.M, g.nl), dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    gcamb.plan_launch(plan, S, P, C, ws)  # tunes, then captures the graph
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    for _ in range(max(3, args.warmup)):
        gcamb.plan_launch(plan, S, P, C, ws)
    steps = max(3, min(args.steps, 20))
    ms, clocks = _timed_region(lambda: gcamb.plan_launch(plan, S, P, C, ws), steps, dev)
    gcamb.sync()
    info = gcamb.plan_info(plan)
    # the CPU baseline and the accuracy: the oracle on the sources of the
    # smallest, the median and the largest l_max, each on its own k prefix
    # and l_max (run on the FP32 sources the plan reads); max relative error
    # per multipole range
    acc = cpu = None
    if not args.no_cpu_baseline:
        import oracle
        Ch = C.cpu().numpy()
        order = np.argsort(lm, kind="stable")
        sel = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
        ranges = ((2, 30), (30, 500), (500, 1500), (1500, 2501), (2501, 6001))
        worst = {}
        per = []
        t0 = time.perf_counter()
        for m in sel:
            q, L = int(nkm[m]), int(lm[m])
            Sm = S[m, :q].double().cpu().numpy()
            Pm = P[m, :q].cpu().numpy()
            _, cr = oracle.los_cl(wl.k[:q], wl.tau, wl.tau0, wl.lmin, L, Sm[None], Pm[None], want_delta=False)
            err = np.abs(Ch[m, :L - wl.lmin + 1] / cr[0] - 1)
            ls = np.arange(wl.lmin, L + 1)
            for a, b in ranges:
                w = (ls >= a) & (ls < b)
                if w.any():
                    key = "[%d,%d]" % (a, b - 1)
                    worst[key] = max(worst.get(key, 0.0), float(err[w].max()))
            per.append({"source": m, "lmax": L, "nk": q, "max_rel_err": float(err.max()),
                        "zero_above_lmax": bool(np.all(Ch[m, L - wl.lmin + 1:] == 0.0))})
        dt = time.perf_counter() - t0
        acc = {"max_rel_err_vs_oracle": max(r["max_rel_err"] for r in per), "max_rel_err_by_l": worst,
               "sources": per, "oracle_s": dt, "oracle_threads": oracle.num_threads()}
        cpu = {"value": len(sel) / dt, "unit": "spectra/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "the sources of the smallest, the median and the largest l_max (%s), each on its own "
                         "k prefix, 1000 tau, %.1f s; the same run checks their C_l"
                         % (", ".join(str(r["lmax"]) for r in per), dt)}
    # whole-step roofline (the graph's three launches are not timed apart):
    # the table's active entries once (4 B hi+lo; tf32 8 B) and every
    # source's own k prefix once (FP32)
    peaks, peak_src = load_peaks()
    pair = 8 if mode == gcamb.TF32X3 else 4
    alg = gcamb.grid_info(g)["active"] * pair + int(nkm.astype(np.int64).sum()) * wl.ntau * 4
    scope = "whole step: split pass + tensor-core kernel + reduce"
    if mode == gcamb.PLAIN32:
        # plain kernels: the table once per 8 sources (one CTA's source chunk),
        # the sources once, the FP32 transfer functions written and read once
        alg = (gcamb.grid_info(g)["active"] * 4 * ((wl.M + 7) // 8) + int(nkm.astype(np.int64).sum()) * wl.ntau * 4
               + 2 * 4 * int(nkm.astype(np.int64).sum()) * g.nl)
        scope = "whole step: plain FP32 transfer kernel + prefix C_l kernel per chunk of 16 sources"
    achieved = alg / (ms / steps * 1e-3) / 1e9
    line = {"metric": "C_l spectra/sec, uneven batch (%d sources, l_max U{1500..6000})" % wl.M,
            "value": wl.M * steps / (ms * 1e-3), "unit": "spectra/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {gcamb.BF16X3: "bf16", gcamb.F16X3: "f16", gcamb.TF32X3: "tf32", gcamb.PLAIN32: "f32"}[mode],
            "data": "synthetic",
            "config": {"workload": "uneven_lmax6000", "M": wl.M, "nk_master": wl.nk, "ntau": wl.ntau,
                       "lmax": wl.lmax, "mode": args.mode, "tile": info["tile"], "items": info["items"],
                       "sources_read_in_place": bool(info["fused"]),
                       "ctas": info["ctas"], "graph_captures": info["captures"], "graph_replays": info["replays"],
                       "table_build_s": table_s, "first_launch_s_incl_tuning": first_s,
                       "table_gb": gcamb.table_bytes(g, mode) / 1e9, "accuracy": acc},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": peak_src,
                         "scope": scope, "algorithmic_bytes": alg},
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": (2 * info["items"] if mode == gcamb.PLAIN32 else 3) * steps}
    print(json.dumps(line), flush=True)


def run_plain(args):
    """The plain path on the two single-model grids: l_max = 500 (300 k log
    1e-4..0.3, 400 tau) and the high-accuracy l_max = 5000 (3000 k log
    1e-5..1, 2000 tau dense near tau*), one model a step: Eq. (2) on the CUDA
    cores (gcamb_los_transfer) and Eq. (1) (gcamb_cl), FP64 and FP32.  The
    oracle on the same model over the whole grid gives the accuracy and the
    CPU baseline (l_max = 500 also at one thread)."""
    import numpy as np
    import torch

    from paper_2509_25110_gb300 import build, gcamb, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    peaks, peak_src = load_peaks()
    fp64_peak = gcamb.probe_flops(0)
    grids = {}
    for wname in ("plain_lmax500", "plain_lmax5000"):
        wl = synth.workload(wname)
        p = synth.model_params(1, seed=0)
        S = synth.sources(wl.k, wl.tau, p)
        P = synth.primordial(wl.k, p)
        g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
        info = gcamb.grid_info(g)
        Pt = torch.as_tensor(P, device=dev)
        res = {}
        for name, mode, dt, eb in (("plain64", gcamb.PLAIN64, torch.float64, 8),
                                   ("plain32", gcamb.PLAIN32, torch.float32, 4)):
            gcamb.bessel_table(g, mode)
            Sd = torch.as_tensor(S, dtype=dt, device=dev)
            D = torch.empty((1, wl.nk, wl.nl), dtype=dt, device=dev)
            C = torch.empty((1, wl.nl), dtype=torch.float64, device=dev)

            def step():
                gcamb.los_transfer(g, Sd, mode, D)
                gcamb.cl(g, D, Pt, C)
            for _ in range(max(3, args.warmup)):
                step()
            gcamb.sync()
            steps = max(3, min(args.steps, 50))
            gcamb.profile_enable(True)
            ms, clocks = _timed_region(step, steps, dev)
            gcamb.sync()
            kms, kn = gcamb.profile_read(gcamb.K_LOS_PLAIN)
            gcamb.profile_enable(False)
            pms = kms / max(1, kn)
            # one model streams the table: its active entries once (8 B FP64,
            # 4 B FP32), the sources once and the transfer functions written
            # once; 2 flop per active (l, k, tau)
            alg = info["active"] * eb + wl.nk * wl.ntau * eb + wl.nk * wl.nl * eb
            flops = 2.0 * info["active"]
            res[name] = {"spectra_per_s": steps / (ms * 1e-3), "ms_per_step": ms / steps, "projection_ms": pms,
                         "hbm_frac": alg / (pms * 1e-3) / 1e9 / peaks["hbm_gbs"], "algorithmic_bytes": alg,
                         "clocks": clocks, "C": C.cpu().numpy()[0]}
            if mode == gcamb.PLAIN64:
                res[name]["fp64_frac"] = flops / (pms * 1e-3) / fp64_peak
        grids[wname] = (wl, S, P, res, info)
    # the oracle on the same model, whole grids
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        from oracle import build as ob
        ob.build()
        for wname, (wl, S, P, res, info) in grids.items():
            t0 = time.perf_counter()
            _, cr = oracle.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, S, P, want_delta=False)
            dt = time.perf_counter() - t0
            cr = cr[0]
            for name in res:
                res[name]["max_rel_err_vs_oracle"] = float(np.max(np.abs(res[name]["C"] / cr - 1)))
            res["oracle"] = {"seconds": dt, "cores": oracle.num_threads()}
            if wname == "plain_lmax500":
                t0 = time.perf_counter()
                oracle.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, S, P, want_delta=False, nthreads=1)
                res["oracle_one_core"] = {"seconds": time.perf_counter() - t0, "cores": 1}
        o = grids["plain_lmax5000"][3]["oracle"]
        cpu = {"value": 1.0 / o["seconds"], "unit": "spectra/s", "cores": o["cores"], "kind": "oracle",
               "sample": "the whole l_max = 5000 grid, one model, %.1f s (l_max = 500: %.2f s at %d threads, "
                         "%.2f s at one)" % (o["seconds"], grids["plain_lmax500"][3]["oracle"]["seconds"],
                                             o["cores"], grids["plain_lmax500"][3]["oracle_one_core"]["seconds"])}
    for _, (_, _, _, res, _) in grids.items():
        for name in ("plain64", "plain32"):
            res[name].pop("C")
    wl5, _, _, r5, info5 = grids["plain_lmax5000"]
    main = r5["plain64"]
    line = {"metric": "C_l spectra/sec, plain FP64 path, l_max=5000 high-accuracy grid (1 model)",
            "value": main["spectra_per_s"], "unit": "spectra/s", "n_gpus": 1, "steps": max(3, min(args.steps, 50)),
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "plain_lmax5000", "M": 1, "lmax": wl5.lmax, "nk": wl5.nk, "ntau": wl5.ntau,
                       "active_entries": info5["active"],
                       "lmax5000": r5, "lmax500": grids["plain_lmax500"][3]},
            "roofline": {"bound": "fp64 alu", "achieved": 2.0 * info5["active"] / (main["projection_ms"] * 1e-3) / 1e12,
                         "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": main["fp64_frac"], "traffic": None,
                         "peak_source": "measured (gcamb_probe_flops, FP64 FMA)",
                         "hbm_view": {"frac": main["hbm_frac"], "peak_gbs": peaks["hbm_gbs"], "peak_source": peak_src}},
            "cpu_baseline": cpu, "clocks": main["clocks"], "gpu_launches": 2 * max(3, min(args.steps, 50))}
    print(json.dumps(line), flush=True)


def run_emulator(args):
    """Trains the emulator on 100k spectra of the batched grid (l 2..2500) and
    serves a held-out set; reports spectra/s and the held-out accuracy."""
    import torch

    from paper_2509_25110_gb300 import build, emulator, gcamb, synth
    torch.cuda.set_device(0)
    build.build()
    wl = synth.workload(WORKLOAD)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    steps = args.steps if args.steps != 600 else 80000
    e, rep, (Xh, Ch) = emulator.train(g, steps=steps, log=lambda m: print(m, file=sys.stderr, flush=True))
    acc = emulator.accuracy(e, Xh, Ch)
    served = emulator.served_by_tolerance(e, Xh, Ch)
    rep["check"] = gcamb.emu_check(e, Xh, Ch, tol=rep["tol"], min_count=32)  # the 1e-3 check serves below
    rates = emulator.serve_rates(e, g, Xh)
    line = {"metric": "emulator C_l spectra/sec at l_max=2500 (trusted cells, projection fallback)",
            "value": rates["emulate_spectra_per_s"], "unit": "spectra/s", "n_gpus": 1, "steps": steps,
            "warmup": 0, "ms_per_step": rep["train_step_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "emulator_lmax2500", "arch": "9-512-512-512-2499 GELU", "batch": rep["batch"],
                       "n_train": rep["n_train"], "n_hold": rep["n_hold"], "train_steps": steps,
                       "data_gen_s": rep["data_s"], "train_s": rep["train_s"], "check": rep["check"],
                       "tol": rep["tol"], "network_accuracy": acc, "served_fraction_by_tol": served, **rates,
                       "gain_network_vs_projection": rates["network_spectra_per_s"] / rates["projection_spectra_per_s"],
                       "gain_emulate_vs_sources_and_projection":
                           rates["emulate_spectra_per_s"] / rates["sources_and_projection_spectra_per_s"],
                       "final_loss": rep["loss_history"][-1][1]}}
    print(json.dumps(line), flush=True)


def run_te(args):
    """Temperature + E-mode on the 256-model, l_max = 2500 grid: C^TT, C^EE and
    C^TE per model from one tensor-core kernel (gcamb_los_cl_te), against the
    temperature-only batch on the same grid and the plain FP64 path."""
    import numpy as np
    import torch

    from paper_2509_25110_gb300 import build, gcamb, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    peaks, peak_src = load_peaks()
    wl = synth.workload(WORKLOAD)
    if args.nk:
        wl.k = synth.log_grid(float(wl.k[0]), float(wl.k[-1]), args.nk)
    M = wl.M
    p = synth.model_params(M, seed=0)
    ST = synth.sources_torch(wl.k, wl.tau, p, dev, torch.float32)
    SP = synth.sources_pol_torch(wl.k, wl.tau, p, dev, torch.float32)
    P = torch.as_tensor(synth.primordial(wl.k, p), device=dev)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    info = gcamb.grid_info(g)
    gcamb.bessel_table(g, gcamb.BF16X3)
    ws = torch.empty(gcamb.los_cl_te_workspace(g, M), dtype=torch.uint8, device=dev)
    out = tuple(torch.empty((M, wl.nl), dtype=torch.float64, device=dev) for _ in range(3))
    for _ in range(max(3, args.warmup)):
        gcamb.los_cl_te(g, ST, SP, P, out=out, ws=ws)
    gcamb.sync()
    steps = args.steps
    gcamb.profile_enable(True)
    ms, clocks = _timed_region(lambda: gcamb.los_cl_te(g, ST, SP, P, out=out, ws=ws), steps, dev)
    gcamb.sync()
    kern = {gcamb.K_NAMES[i]: gcamb.profile_read(i) for i in (gcamb.K_SPLIT, gcamb.K_WEIGHTS, gcamb.K_TC, gcamb.K_REDUCE)}
    gcamb.profile_enable(False)
    tc_ms, tc_n = kern["los_cl_tc"]
    tc_avg_s = tc_ms / max(1, tc_n) * 1e-3
    # the table (hi + lo, 4 bytes an active entry) once, both FP32 sources once
    alg_bytes = info["active"] * 4 + 2 * M * wl.nk * wl.ntau * 4
    alg_flops = 3 * 2 * info["active"] * 2 * M
    achieved = alg_bytes / tc_avg_s / 1e9
    # the temperature-only batch on the same grid and sources
    wsT = torch.empty(gcamb.los_cl_workspace(g, M, gcamb.BF16X3), dtype=torch.uint8, device=dev)
    CT = torch.empty((M, wl.nl), dtype=torch.float64, device=dev)
    for _ in range(3):
        gcamb.los_cl(g, ST, P, gcamb.BF16X3, CT, wsT)
    t_ms, _ = _timed_region(lambda: gcamb.los_cl(g, ST, P, gcamb.BF16X3, CT, wsT), steps, dev)
    gcamb.sync()
    # plain FP64 TT, EE, TE of 4 models on the same grid
    gcamb.bessel_table(g, gcamb.PLAIN64)
    S64, P64 = ST[:4].double().contiguous(), P[:4].contiguous()
    E64 = SP[:4].double().contiguous()

    def plain_step():
        DT = gcamb.los_transfer(g, S64, gcamb.PLAIN64)
        DE = gcamb.los_transfer_e(g, E64, gcamb.PLAIN64)
        gcamb.cl(g, DT, P64)
        gcamb.cl_cross(g, DE, DE, P64)
        gcamb.cl_cross(g, DT, DE, P64)
    plain_step()
    plain_ms, _ = _timed_region(plain_step, 2, dev)
    plain_rate = 4 / (plain_ms / 2 * 1e-3)
    gcamb.sync()
    # the oracle on one model: accuracy and the CPU baseline
    cpu = None
    err = None
    if not args.no_cpu_baseline:
        import oracle
        from oracle import build as ob
        ob.build()
        Sc, Ec, Pc = ST[:1].double().cpu().numpy(), SP[:1].double().cpu().numpy(), P[:1].cpu().numpy()
        t0 = time.perf_counter()
        DT, TT = oracle.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, Sc, Pc)
        DE = oracle.los_e(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, Ec)
        EE = oracle.cl_cross(wl.k, DE, DE, Pc)
        TE = oracle.cl_cross(wl.k, DT, DE, Pc)
        dt = time.perf_counter() - t0
        cpu = {"value": 1 / dt, "unit": "models/s (TT, EE, TE)", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "1 of the 256 models, full grid, %.1f s" % dt}
        tt, ee, te = (x[:1].cpu().numpy() for x in out)
        nz = EE > 0
        err = {"TT": float(np.max(np.abs(tt / TT - 1))), "EE": float(np.max(np.abs(ee[nz] / EE[nz] - 1))),
               "TE_on_sqrt_TT_EE": float(np.max(np.abs(te - TE)[nz] / np.sqrt(TT * EE)[nz])),
               "max_dcl_over_sigma_cv": {"TT": float(oracle.cosmic_variance_ratio(tt, TT).max()),
                                         "EE": float(oracle.cosmic_variance_ratio(ee, EE).max()),
                                         "TE": float(oracle.cosmic_variance_ratio_te(te, TT, EE, TE).max())}}
    line = {"metric": "TT+EE+TE spectrum sets/sec at l_max=2500, batched split precision (bf16x3)",
            "value": M * steps / (ms * 1e-3), "unit": "models/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "batched_te_lmax2500", "M": M, "lmax": wl.lmax, "nk": wl.nk, "ntau": wl.ntau,
                       "l2": "inputs larger than L2 (two 2.05 GB fp32 sources)",
                       "tt_only_ms_per_step": t_ms / steps, "te_over_tt_only_time": ms / t_ms,
                       "plain64_models_per_s": plain_rate, "speedup_vs_plain64": M * steps / (ms * 1e-3) / plain_rate,
                       "max_err_vs_oracle": err,
                       "kernel_ms": {k: (v[0] / max(1, v[1])) for k, v in kern.items()}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"],
                         "traffic": committed_traffic("los_cl_tc_te_traffic.txt", "te_bf16x3"), "peak_source": peak_src,
                         "kernel": "los_cl_tc_kernel (TE)", "kernel_ms": tc_avg_s * 1e3, "algorithmic_bytes": alg_bytes,
                         "tensor_view": {"achieved_tflops": alg_flops / tc_avg_s / 1e12,
                                         "frac": alg_flops / tc_avg_s / 1e12 / peaks.get("bf16_tflops", 1900.0)}},
            "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": 3 * steps}
    print(json.dumps(line), flush=True)


def run_tensor(args):
    """Tensor modes on the plain path: the l_max = 1500, k tau0 <= 3000 tensor
    grid of the paper's runs, 4 models a step, Delta_T, Delta_E, Delta_B
    (gcamb_los_transfer_tensor) and C^TT, C^EE, C^BB, C^TE, in FP64 and FP32."""
    import numpy as np
    import torch

    from paper_2509_25110_gb300 import build, gcamb, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    wl = synth.workload("tensor_lmax1500")
    M = 4
    p = synth.model_params(M, seed=0)
    ST, SP = synth.sources_tensor(wl.k, wl.tau, p)
    Pt = torch.as_tensor(synth.primordial_tensor(wl.k, p), device=dev)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    info = gcamb.grid_info(g)
    res = {}
    for name, mode, dt in (("plain64", gcamb.PLAIN64, torch.float64), ("plain32", gcamb.PLAIN32, torch.float32)):
        gcamb.bessel_table(g, mode)
        STd, SPd = (torch.as_tensor(a, dtype=dt, device=dev) for a in (ST, SP))
        out = tuple(torch.empty((M, wl.nk, wl.nl), dtype=dt, device=dev) for _ in range(3))
        cls = tuple(torch.empty((M, wl.nl), dtype=torch.float64, device=dev) for _ in range(4))

        def step():
            DT, DE, DB = gcamb.los_transfer_tensor(g, STd, SPd, mode, out=out)
            gcamb.cl(g, DT, Pt, cls[0])
            gcamb.cl(g, DE, Pt, cls[1])
            gcamb.cl(g, DB, Pt, cls[2])
            gcamb.cl_cross(g, DT, DE, Pt, cls[3])
        for _ in range(max(3, args.warmup)):
            step()
        gcamb.sync()
        steps = max(3, min(args.steps, 20))
        gcamb.profile_enable(True)
        ms, clocks = _timed_region(step, steps, dev)
        gcamb.sync()
        kms, kn = gcamb.profile_read(gcamb.K_LOS_PLAIN)
        gcamb.profile_enable(False)
        # four plain launches a step (D0, D1, D2 of S_P; the temperature), each
        # 2 flop per stored (l, k, tau) table entry per model
        flops = 4 * 2.0 * info["stored_plain64"] * M
        peak = gcamb.probe_flops(0 if mode == gcamb.PLAIN64 else 1)
        res[name] = {"models_per_s": M * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                     "projection_ms": kms / steps, "achieved_tflops": flops / (kms / steps * 1e-3) / 1e12,
                     "peak_tflops": peak / 1e12, "clocks": clocks,
                     "cls": [c.cpu().numpy() for c in cls]}
    # the oracle on one model: accuracy and the CPU baseline
    cpu = None
    err = None
    if not args.no_cpu_baseline:
        import oracle
        from oracle import build as ob
        ob.build()
        t0 = time.perf_counter()
        R = oracle.los_tensor(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, ST[:1], SP[:1])
        P1 = Pt[:1].cpu().numpy()
        ref = [oracle.cl_cross(wl.k, R[0], R[0], P1), oracle.cl_cross(wl.k, R[1], R[1], P1),
               oracle.cl_cross(wl.k, R[2], R[2], P1), oracle.cl_cross(wl.k, R[0], R[1], P1)]
        dt = time.perf_counter() - t0
        cpu = {"value": 1 / dt, "unit": "models/s (tensor TT, EE, BB, TE)", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "1 of the 4 models, full tensor grid, %.1f s" % dt}
        err = {}
        for name in res:
            c = [x[:1] for x in res[name]["cls"]]
            err[name] = {key: float(np.max(np.abs(c[i] / ref[i] - 1)[ref[i] > 0])) for i, key in
                         enumerate(("TT", "EE", "BB"))}
            err[name]["TE_on_sqrt_TT_EE"] = float(np.max(np.abs(c[3] - ref[3])[ref[0] > 0] /
                                                         np.sqrt(ref[0] * ref[1])[ref[0] > 0]))
    # batched tensor-core path: one kernel grid per field (c_l j_l/x^2 for T,
    # e_l for E, b_l for B), 256 models, C^TT, C^EE, C^BB
    Mb = 256
    pb = synth.model_params(Mb, seed=0)
    STb, SPb = (torch.as_tensor(a, dtype=torch.float32, device=dev)
                for a in synth.sources_tensor(wl.k, wl.tau, pb))
    Pb = torch.as_tensor(synth.primordial_tensor(wl.k, pb), device=dev)
    refb = None
    if not args.no_cpu_baseline:
        R1 = oracle.los_tensor(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, STb[:1].double().cpu().numpy(),
                               SPb[:1].double().cpu().numpy())
        P1b = Pb[:1].cpu().numpy()
        refb = {"TT": oracle.cl_cross(wl.k, R1[0], R1[0], P1b), "EE": oracle.cl_cross(wl.k, R1[1], R1[1], P1b),
                "BB": oracle.cl_cross(wl.k, R1[2], R1[2], P1b)}
    batched = {}
    for mname, bmode in (("bf16x3", gcamb.BF16X3), ("f16x3", gcamb.F16X3)):
        grids = {}
        for name, kern in (("TT", gcamb.KERNEL_EPS), ("EE", gcamb.KERNEL_TENSOR_E), ("BB", gcamb.KERNEL_TENSOR_B)):
            gk = gcamb.grid_set_kernel(gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax), kern)
            gcamb.bessel_table(gk, bmode)
            grids[name] = (gk, torch.empty(gcamb.los_cl_workspace(gk, Mb, bmode), dtype=torch.uint8, device=dev),
                           torch.empty((Mb, wl.nl), dtype=torch.float64, device=dev), STb if name == "TT" else SPb)

        def bstep():
            for gk, wsk, Ck, Sk in grids.values():
                gcamb.los_cl(gk, Sk, Pb, bmode, Ck, wsk)
        for _ in range(3):
            bstep()
        gcamb.sync()
        bsteps = max(3, min(args.steps, 50))
        bms, _ = _timed_region(bstep, bsteps, dev)
        gcamb.sync()
        b = {"models_per_s": Mb * bsteps / (bms * 1e-3), "ms_per_step": bms / bsteps, "M": Mb}
        if refb is not None:
            b["max_rel_err_vs_oracle"] = {k: float(np.max(np.abs(grids[k][2][:1].cpu().numpy() / v - 1)))
                                          for k, v in refb.items()}
            b["max_dcl_over_sigma_cv"] = {k: float(oracle.cosmic_variance_ratio(grids[k][2][:1].cpu().numpy(),
                                                                                v).max())
                                          for k, v in refb.items()}
        batched[mname] = b
        if bmode == gcamb.BF16X3:
            # TT, EE and TE from one launch on the T and E kernel grids, BB from the B grid
            gT, gE, gB = grids["TT"][0], grids["EE"][0], grids["BB"][0]
            wsp = torch.empty(gcamb.los_cl_te_workspace(gT, Mb), dtype=torch.uint8, device=dev)
            outp = tuple(torch.empty((Mb, wl.nl), dtype=torch.float64, device=dev) for _ in range(3))

            def pstep():
                gcamb.los_cl_pair(gT, gE, STb, SPb, Pb, out=outp, ws=wsp)
                gcamb.los_cl(gB, SPb, Pb, bmode, grids["BB"][2], grids["BB"][1])
            for _ in range(3):
                pstep()
            gcamb.sync()
            pms, _ = _timed_region(pstep, bsteps, dev)
            gcamb.sync()
            pb_ = {"models_per_s": Mb * bsteps / (pms * 1e-3), "ms_per_step": pms / bsteps,
                   "spectra": "TT, EE, TE (pair) + BB"}
            if refb is not None:
                te_ref = oracle.cl_cross(wl.k, R1[0], R1[1], P1b)
                tt1, ee1, te1 = (x[:1].cpu().numpy() for x in outp)
                pb_["max_rel_err_vs_oracle"] = {"TT": float(np.max(np.abs(tt1 / refb["TT"] - 1))),
                                                "EE": float(np.max(np.abs(ee1 / refb["EE"] - 1))),
                                                "TE_on_sqrt_TT_EE": float(np.max(np.abs(te1 - te_ref) /
                                                                                 np.sqrt(refb["TT"] * refb["EE"])))}
                pb_["max_dcl_over_sigma_cv_TE"] = float(oracle.cosmic_variance_ratio_te(te1, refb["TT"], refb["EE"],
                                                                                        te_ref).max())
            batched["bf16x3_pair_tt_ee_te_plus_bb"] = pb_
        for gk, *_ in grids.values():
            gk.close()
    r64 = res["plain64"]
    line = {"metric": "tensor TT+EE+BB+TE spectrum sets/sec at l_max=1500 (plain FP64)",
            "value": r64["models_per_s"], "unit": "models/s", "n_gpus": 1, "steps": max(3, min(args.steps, 20)),
            "warmup": args.warmup, "ms_per_step": r64["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "tensor_lmax1500", "M": M, "lmax": wl.lmax, "nk": wl.nk, "ntau": wl.ntau,
                       "stored_entries": info["stored_plain64"],
                       "plain32": {k: v for k, v in res["plain32"].items() if k not in ("cls", "clocks")},
                       "batched_tt_ee_bb": batched,
                       "max_err_vs_oracle": err},
            "roofline": {"bound": "alu", "achieved": r64["achieved_tflops"], "peak": r64["peak_tflops"],
                         "unit": "TFLOP/s", "frac": r64["achieved_tflops"] / r64["peak_tflops"], "traffic": None,
                         "peak_source": "FP64 FMA probe (gcamb_probe_flops)", "kernel": "los_plain_kernel<double>",
                         "kernel_ms": r64["projection_ms"]},
            "cpu_baseline": cpu, "clocks": r64["clocks"], "gpu_launches": 9 * max(3, min(args.steps, 20))}
    print(json.dumps(line), flush=True)


def run_features(args):
    """Primordial features (Sec. 5): 256 models with log-oscillating P(k) on a
    dense transfer grid of 8000 k nodes, every l to 2500.  A step interpolates
    the sources from the 1000-node solver grid onto the transfer grid
    (gcamb_interp_sources) and projects them (gcamb_los_cl, BF16X3)."""
    import numpy as np
    import torch

    from paper_2509_25110_gb300 import build, gcamb, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    peaks, peak_src = load_peaks()
    wl = synth.workload("features_lmax2500")
    if args.nk:  # profiling case: the transfer grid's k range with this many nodes
        wl.k = synth.log_grid(float(wl.k[0]), float(wl.k[-1]), args.nk)
    k_ode = synth.log_grid(float(wl.k[0]), float(wl.k[-1]), 1000)
    M = wl.M
    p = synth.model_params(M, seed=0)
    f = synth.feature_params(M, seed=0)
    S_ode = synth.sources_torch(k_ode, wl.tau, p, dev, torch.float32)
    P = torch.as_tensor(synth.primordial_features(wl.k, p, f), device=dev)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    info = gcamb.grid_info(g)
    gcamb.bessel_table(g, gcamb.BF16X3)
    S = torch.empty((M, wl.nk, wl.ntau), dtype=torch.float32, device=dev)
    ws = torch.empty(gcamb.los_cl_workspace(g, M, gcamb.BF16X3), dtype=torch.uint8, device=dev)
    C = torch.empty((M, wl.nl), dtype=torch.float64, device=dev)

    def step():
        gcamb.interp_sources(g, k_ode, S_ode, S)
        gcamb.los_cl(g, S, P, gcamb.BF16X3, C, ws)
    for _ in range(max(3, args.warmup)):
        step()
    gcamb.sync()
    steps = max(3, min(args.steps, 50))
    gcamb.profile_enable(True)
    ms, clocks = _timed_region(step, steps, dev)
    gcamb.sync()
    kern = {gcamb.K_NAMES[i]: gcamb.profile_read(i) for i in (gcamb.K_INTERP, gcamb.K_SPLIT, gcamb.K_WEIGHTS,
                                                               gcamb.K_TC, gcamb.K_REDUCE)}
    gcamb.profile_enable(False)
    tc_ms, tc_n = kern["los_cl_tc"]
    tc_s = tc_ms / max(1, tc_n) * 1e-3
    alg_bytes = info["active"] * 4 + M * wl.nk * wl.ntau * 4
    achieved = alg_bytes / tc_s / 1e9
    cpu = None
    err = None
    if not args.no_cpu_baseline:
        import oracle
        from oracle import build as ob
        from oracle import interp as ointerp
        ob.build()
        mc = 2
        t0 = time.perf_counter()
        Sref = ointerp.interp_sources(k_ode, S_ode[:mc].double().cpu().numpy(), wl.k)
        _, Cr = oracle.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, Sref.astype(np.float32).astype(np.float64),
                              P[:mc].cpu().numpy(), want_delta=False)
        dt = time.perf_counter() - t0
        cpu = {"value": mc / dt, "unit": "spectra/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "%d of the 256 models, full grid (interpolation + projection), %.1f s" % (mc, dt)}
        err = float(np.max(np.abs(C[:mc].cpu().numpy() / Cr - 1)))
    line = {"metric": "C_l spectra/sec at l_max=2500 with primordial features (8000 k, sources interpolated)",
            "value": M * steps / (ms * 1e-3), "unit": "spectra/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "features_lmax2500", "M": M, "lmax": wl.lmax, "nk": wl.nk, "nk_sources": 1000,
                       "ntau": wl.ntau, "l2": "inputs larger than L2 (8.2 GB of interpolated sources)",
                       "table_gb": gcamb.table_bytes(g, gcamb.BF16X3) / 1e9,
                       "kernel_ms": {k: v[0] / max(1, v[1]) for k, v in kern.items()},
                       "max_rel_err_vs_oracle": err},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": peak_src,
                         "kernel": "los_cl_tc_kernel", "kernel_ms": tc_s * 1e3, "algorithmic_bytes": alg_bytes},
            "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": 5 * steps}
    print(json.dumps(line), flush=True)


def run_lsampled(args):
    """l-sampling (the accuracy settings of Sec. 3.1, Table 1): the 256-model
    l_max = 2500 batch computed on sampled multipoles (l_sample_boost 1, 3
    and 20) and splined to every l (gcamb_cl_interp), against every l
    computed (boost 50).  Reports the throughput and the spline's deviation
    from the every-l result, also in units of the cosmic variance (Sec. 4.6).
    The k grid resolves the projection's oscillations in k (linear above
    0.01), so that C_l is smooth in l."""
    import numpy as np
    import torch

    from paper_2509_25110_gb300 import build, gcamb, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    wl = synth.workload("lsampled_lmax2500")
    M = wl.M
    p = synth.model_params(M, seed=0)
    S = synth.sources_torch(wl.k, wl.tau, p, dev, torch.float32)
    P = torch.as_tensor(synth.primordial(wl.k, p), device=dev)
    gd = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    gcamb.bessel_table(gd, gcamb.BF16X3)
    Cd = gcamb.los_cl(gd, S, P, gcamb.BF16X3)
    for _ in range(3):
        gcamb.los_cl(gd, S, P, gcamb.BF16X3, Cd)
    steps = max(3, min(args.steps, 100))
    ms_dense, _ = _timed_region(lambda: gcamb.los_cl(gd, S, P, gcamb.BF16X3, Cd), steps, dev)
    gcamb.sync()
    Cd_h = Cd.cpu().numpy()
    l = np.arange(wl.lmin, wl.lmax + 1, dtype=np.float64)
    out = {}
    clocks = None
    for boost in (1.0, 3.0, 20.0):
        lv = gcamb.l_sampling(wl.lmin, wl.lmax, boost)
        g = gcamb.grid_create_lsampled(wl.k, wl.tau, wl.tau0, lv)
        gcamb.bessel_table(g, gcamb.BF16X3)
        ws = torch.empty(gcamb.los_cl_workspace(g, M, gcamb.BF16X3), dtype=torch.uint8, device=dev)
        Cs = torch.empty((M, g.nl), dtype=torch.float64, device=dev)
        Cf = torch.empty((M, wl.nl), dtype=torch.float64, device=dev)

        def step():
            gcamb.los_cl(g, S, P, gcamb.BF16X3, Cs, ws)
            gcamb.cl_interp(g, Cs, Cf)
        for _ in range(max(3, args.warmup)):
            step()
        gcamb.sync()
        gcamb.profile_enable(True)
        ms, clocks = _timed_region(step, steps, dev)
        gcamb.sync()
        kern = {gcamb.K_NAMES[i]: gcamb.profile_read(i) for i in (gcamb.K_TC, gcamb.K_REDUCE, gcamb.K_INTERP)}
        gcamb.profile_enable(False)
        Cf_h = Cf.cpu().numpy()
        rel = np.abs(Cf_h / Cd_h - 1)
        cv = np.abs(Cf_h - Cd_h) / (np.sqrt(2.0 / (2.0 * l + 1.0)) * np.abs(Cd_h))
        out["boost_%g" % boost] = {"n_l": int(lv.size), "spectra_per_s": M * steps / (ms * 1e-3),
                                   "ms_per_step": ms / steps, "speedup_vs_every_l": ms_dense / ms,
                                   "max_rel_dev_from_every_l": float(rel.max()),
                                   "median_rel_dev": float(np.median(rel)),
                                   "max_dcl_over_sigma_cv": float(cv.max()),
                                   "kernel_ms": {k: v[0] / max(1, v[1]) for k, v in kern.items()}}
        g.close()
    b1 = out["boost_1"]
    line = {"metric": "C_l spectra/sec at l_max=2500, l_sample_boost=1 (sampled l + spline), BF16X3",
            "value": b1["spectra_per_s"], "unit": "spectra/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": b1["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "lsampled_lmax2500", "M": M, "lmax": wl.lmax, "nk": wl.nk,
                       "ntau": wl.ntau, "every_l_spectra_per_s": M * steps / (ms_dense * 1e-3), **out},
            "clocks": clocks, "gpu_launches": 5 * steps}
    print(json.dumps(line), flush=True)


def run_curved(args):
    """Curved space (Sec. 5): the 256-model l_max = 2500 batch in an open
    universe with Omega_K = 0.01 (K = -Omega_K (H0/c)^2, h = 0.7: -5.45e-10
    Mpc^-2), hyperspherical Bessel table, BF16X3; also the flat batch on the
    same grid, and the table builds."""
    import numpy as np
    import torch

    from paper_2509_25110_gb300 import build, gcamb, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    peaks, peak_src = load_peaks()
    K = -0.01 * (0.7 / 2997.92458) ** 2
    wl = synth.workload(WORKLOAD)
    M = wl.M
    p = synth.model_params(M, seed=0)
    S = synth.sources_torch(wl.k, wl.tau, p, dev, torch.float32)
    P = torch.as_tensor(synth.primordial(wl.k, p), device=dev)
    out = {}
    clocks = None
    for name, mk in (("flat", lambda: gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)),
                     ("open", lambda: gcamb.grid_create_curved(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, K))):
        g = mk()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gcamb.bessel_table(g, gcamb.BF16X3)
        torch.cuda.synchronize()
        table_s = time.perf_counter() - t0
        info = gcamb.grid_info(g)
        ws = torch.empty(gcamb.los_cl_workspace(g, M, gcamb.BF16X3), dtype=torch.uint8, device=dev)
        C = torch.empty((M, wl.nl), dtype=torch.float64, device=dev)
        for _ in range(max(3, args.warmup)):
            gcamb.los_cl(g, S, P, gcamb.BF16X3, C, ws)
        gcamb.sync()
        steps = max(3, min(args.steps, 200))
        gcamb.profile_enable(True)
        ms, clocks = _timed_region(lambda: gcamb.los_cl(g, S, P, gcamb.BF16X3, C, ws), steps, dev)
        gcamb.sync()
        tc_ms, tc_n = gcamb.profile_read(gcamb.K_TC)
        gcamb.profile_enable(False)
        tc_s = tc_ms / max(1, tc_n) * 1e-3
        alg = info["active"] * 4 + M * wl.nk * wl.ntau * 4
        out[name] = {"spectra_per_s": M * steps / (ms * 1e-3), "ms_per_step": ms / steps, "kernel_ms": tc_s * 1e3,
                     "table_build_s": table_s, "table_gb": gcamb.table_bytes(g, gcamb.BF16X3) / 1e9,
                     "stored_entries": info["active"], "hbm_frac": alg / tc_s / 1e9 / peaks["hbm_gbs"],
                     "C": C[:2].cpu().numpy()}
        g.close()
    cpu = None
    err = None
    if not args.no_cpu_baseline:
        import oracle
        from oracle import build as ob
        ob.build()
        t0 = time.perf_counter()
        Dr = oracle.los_curved(wl.k, wl.tau, wl.tau0, K, wl.lmin, wl.lmax, S[:1].double().cpu().numpy())
        Cr = oracle.cl_from_delta(wl.k, Dr, P[:1].cpu().numpy())
        dt = time.perf_counter() - t0
        cpu = {"value": 1 / dt, "unit": "spectra/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "1 of the 256 models, full curved grid, %.1f s" % dt}
        err = float(np.max(np.abs(out["open"]["C"][:1] / Cr - 1)))
    o = out["open"]
    line = {"metric": "C_l spectra/sec at l_max=2500 in an open universe (Omega_K = 0.01), BF16X3",
            "value": o["spectra_per_s"], "unit": "spectra/s", "n_gpus": 1, "steps": max(3, min(args.steps, 200)),
            "warmup": args.warmup, "ms_per_step": o["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "batched_lmax2500, open space", "K_per_Mpc2": K, "M": M, "lmax": wl.lmax,
                       "nk": wl.nk, "ntau": wl.ntau, "max_rel_err_vs_oracle": err,
                       "open": {k: v for k, v in o.items() if k != "C"},
                       "flat": {k: v for k, v in out["flat"].items() if k != "C"}},
            "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": 3 * max(3, min(args.steps, 200))}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "plain":
        run_plain(args)
        return
    if args.workload == "uneven":
        run_uneven(args)
        return
    if args.workload == "emulator":
        run_emulator(args)
        return
    if args.workload == "te":
        run_te(args)
        return
    if args.workload == "tensor":
        run_tensor(args)
        return
    if args.workload == "features":
        run_features(args)
        return
    if args.workload == "lsampled":
        run_lsampled(args)
        return
    if args.workload == "curved":
        run_curved(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2509_25110_gb300 import build, gcamb, shard, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    build.build()
    mode = {"bf16x3": gcamb.BF16X3, "tf32x3": gcamb.TF32X3, "f16x3": gcamb.F16X3}[args.mode]
    peaks, peak_src = load_peaks()

    wl = synth.workload(WORKLOAD)
    if args.nk:
        wl.k = synth.log_grid(float(wl.k[0]), float(wl.k[-1]), args.nk)
    M = wl.M
    p = shard.rank_params(M, rank)
    S = synth.sources_torch(wl.k, wl.tau, p, dev, torch.float32)
    P = torch.as_tensor(synth.primordial(wl.k, p), device=dev)
    g = gcamb.grid_create(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax)
    info = gcamb.grid_info(g)

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b)

    first_table_ms = timed(lambda: gcamb.bessel_table(g, mode))
    table_ms = timed(lambda: gcamb.bessel_table(g, mode))
    ws = torch.empty(gcamb.los_cl_workspace(g, M, mode), dtype=torch.uint8, device=dev)
    C = torch.empty((M, wl.nl), dtype=torch.float64, device=dev)
    first_call_ms = timed(lambda: gcamb.los_cl(g, S, P, mode, C, ws))
    gcamb.sync()
    for _ in range(max(3, args.warmup)):
        gcamb.los_cl(g, S, P, mode, C, ws)
    gcamb.sync()

    # ---------------- timed region
    bus = None
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id
    except Exception:
        pass
    sampler = ClockSampler(bus)
    shard.barrier()
    torch.cuda.synchronize()
    gcamb.profile_enable(True)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        gcamb.los_cl(g, S, P, mode, C, ws)
    e1.record()
    e1.synchronize()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    shard.barrier()
    gcamb.sync()
    ms = e0.elapsed_time(e1)
    kern = {gcamb.K_NAMES[i]: gcamb.profile_read(i) for i in (gcamb.K_SPLIT, gcamb.K_WEIGHTS, gcamb.K_TC,
                                                               gcamb.K_REDUCE)}
    gcamb.profile_enable(False)
    if args.kernel_only:
        print(json.dumps({"workload": WORKLOAD, "nk": wl.nk, "mode": args.mode, "steps": args.steps,
                          "ms_per_step": ms / args.steps, "table_compressed": gcamb.table_compressed(g, mode),
                          "kernel_ms": {k: (v[0] / max(1, v[1])) for k, v in kern.items()}}), flush=True)
        return
    ms = shard.max_over_ranks(ms, dev)
    value = shard.job_rate(world, M, args.steps, ms)
    launches = sum(n for _, n in kern.values())

    # ---------------- roofline of the dominant kernel (tensor-core contraction)
    tc_ms, tc_n = kern["los_cl_tc"]
    tc_avg_s = tc_ms / max(1, tc_n) * 1e-3
    pair = 8 if mode == gcamb.TF32X3 else 4            # bytes of one hi+lo table entry
    # active table entries (hi + lo) and the sources once (FP32, read by the
    # fused kernel; the split pass's hi + lo planes for tf32x3: 8 bytes)
    alg_bytes = info["active"] * pair + M * wl.nk * wl.ntau * pair
    alg_flops = 3 * 2 * info["active"] * M                             # three split products
    achieved_gbs = alg_bytes / tc_avg_s / 1e9
    traffic = committed_traffic("los_cl_tc_traffic.txt", args.mode)
    roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved_gbs / peaks["hbm_gbs"], "traffic": traffic,
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                "kernel": "los_cl_tc_kernel", "kernel_ms": tc_avg_s * 1e3,
                "algorithmic_bytes": alg_bytes,
                "tensor_view": {"achieved_tflops": alg_flops / tc_avg_s / 1e12,
                                "peak_tflops": peaks.get("bf16_tflops"),
                                "frac": alg_flops / tc_avg_s / 1e12 / peaks.get("bf16_tflops", 1900.0)}}

    # ---------------- end to end through the C ABI with host buffers: every
    # step copies its sources and P(k) from pinned host memory and reads its
    # C_l back; two buffer sets let the copy of one batch overlap the compute
    # of the previous one (copy stream + the compute stream)
    S_h = S.cpu().pin_memory()
    P_h = P.cpu().pin_memory()
    C_h = [torch.empty((M, wl.nl), dtype=torch.float64).pin_memory() for _ in range(2)]
    S_d = [torch.empty_like(S) for _ in range(2)]
    P_d = [torch.empty_like(P) for _ in range(2)]
    C_d = [torch.empty_like(C) for _ in range(2)]
    ks = torch.cuda.current_stream()
    cs = torch.cuda.Stream()
    free = [torch.cuda.Event() for _ in range(2)]
    ready = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(n):
        for i in range(n):
            b = i % 2
            with torch.cuda.stream(cs):
                cs.wait_event(free[b])
                S_d[b].copy_(S_h, non_blocking=True)
                P_d[b].copy_(P_h, non_blocking=True)
                ready[b].record(cs)
            ks.wait_event(ready[b])
            gcamb.los_cl(g, S_d[b], P_d[b], mode, C_d[b], ws, stream=ks)
            C_h[b].copy_(C_d[b], non_blocking=True)
            free[b].record(ks)
    for b in range(2):
        free[b].record(ks)
    e2e_run(2)
    torch.cuda.synchronize()
    # three timed runs, the median reported: the host link is shared with
    # the other jobs on the machine, so single runs scatter
    e2e_runs = []
    for _ in range(3):
        e2e_runs.append(timed(lambda: e2e_run(args.e2e_steps)))
        torch.cuda.synchronize()
    e2e_ms = sorted(e2e_runs)[1]
    gcamb.sync()
    # the host link: one pinned copy of the sources alone, and where the
    # memory sits (NUMA node of the GPU's PCI function, of the buffer's pages)
    h2d_ms = timed(lambda: S_d[0].copy_(S_h, non_blocking=True))
    e2e = {"value": world * M * args.e2e_steps / (e2e_ms * 1e-3), "unit": "spectra/s",
           "h2d_bytes_per_step": S_h.numel() * 4 + P_h.numel() * 8, "d2h_bytes_per_step": C_h[0].numel() * 8,
           "overlap": "double-buffered: H2D of batch i+1 on a copy stream during the compute of batch i",
           "runs": "median of three timed runs of %d steps (ms: %s)" % (args.e2e_steps,
                                                                    ", ".join("%.1f" % v for v in e2e_runs)),
           "h2d_gbs": S_h.numel() * 4 / (h2d_ms * 1e-3) / 1e9, "numa": host_numa(dev, S_h)}

    # ---------------- plain FP64 on the same grid (the metric's comparison), 4 sources
    gcamb.bessel_table(g, gcamb.PLAIN64)
    S64 = S[:4].double().contiguous()
    D64 = torch.empty((4, wl.nk, wl.nl), dtype=torch.float64, device=dev)
    C64 = torch.empty((4, wl.nl), dtype=torch.float64, device=dev)

    def plain_step():
        gcamb.los_transfer(g, S64, gcamb.PLAIN64, D64)
        gcamb.cl(g, D64, P[:4].contiguous(), C64)
    plain_step()
    plain_ms = timed(lambda: [plain_step() for _ in range(3)]) / 3
    gcamb.sync()
    plain64_rate = 4 / (plain_ms * 1e-3)

    # ---------------- CPU baseline and accuracy: the oracle on the host cores
    # (rank 0, N = 1).  One all-core run over the timed batch's sources on
    # the full grid gives the error of every checked spectrum (per l range)
    # and the all-core rate; the same sources on 16 of the k nodes give the
    # one-core and all-core rates of one sample (the oracle's cost is linear
    # in the k nodes, so the rates are comparable).
    cpu = None
    err = None
    err_by_l = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        from oracle import build as ob
        ob.build()
        mc = min(args.cpu_models, M)
        Cr = np.empty((mc, wl.nl))
        dt = 0.0
        for m0 in range(0, mc, ORACLE_GROUP):
            m1 = min(mc, m0 + ORACLE_GROUP)
            Sc = S[m0:m1].double().cpu().numpy()
            Pc = P[m0:m1].cpu().numpy()
            t0 = time.perf_counter()
            _, Cr[m0:m1] = oracle.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, Sc, Pc, want_delta=False)
            dt += time.perf_counter() - t0
        rel = np.abs(C[:mc].cpu().numpy() / Cr - 1)
        err = float(rel.max())
        err_by_l = l_range_errors(rel, wl.lmin, wl.lmax)
        cores = oracle.num_threads()
        q16 = np.unique(np.linspace(0, wl.nk - 1, 16).astype(int))
        Sg = S[:ORACLE_GROUP].double().cpu().numpy()
        Pg = P[:ORACLE_GROUP].cpu().numpy()
        one = oracle_sample_rates(wl, np.ascontiguousarray(Sg[:, q16, :]), np.ascontiguousarray(Pg[:, q16]), q16)
        cpu = {"value": mc / dt, "unit": "spectra/s", "cores": cores, "kind": "oracle",
               "sample": "%d of the %d sources of the timed batch in calls of %d, full grid (%d k x %d tau, "
                         "l %d..%d), %.1f s; the same run checks their C_l"
                         % (mc, M, ORACLE_GROUP, wl.nk, wl.ntau, wl.lmin, wl.lmax, dt),
               "same_sample_1_core_vs_all": one}

    props = torch.cuda.get_device_properties(dev)
    # the work plan of the timed launches (a uniform plan of the same batch:
    # the same plan builder, items and tiles)
    pinfo = gcamb.plan_info(gcamb.plan_create(g, M, mode=mode))
    line = {
        "metric": METRIC, "value": value, "unit": "spectra/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {gcamb.BF16X3: "bf16", gcamb.F16X3: "f16", gcamb.TF32X3: "tf32"}[mode], "data": "synthetic",
        "config": {"workload": WORKLOAD, "M": M, "lmax": wl.lmax, "nk": wl.nk, "ntau": wl.ntau,
                   "mode": args.mode, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (sources 2.05 GB fp32, table %.2f GB)" % (gcamb.table_bytes(g, mode) / 1e9),
                   "table": "resident, built once per grid: %.2f ms (first build %.2f ms), not in the step" % (
                       table_ms, first_table_ms),
                   "table_compressed": gcamb.table_compressed(g, mode),
                   "first_call_ms": first_call_ms, "max_rel_err_vs_oracle": err,
                   "max_rel_err_by_l": err_by_l,
                   "max_rel_err_sample": ("%d of %d sources, every l" % (min(args.cpu_models, M), M)
                                          if err is not None else None),
                   "plain64_spectra_per_s": plain64_rate, "speedup_vs_plain64": value / world / plain64_rate,
                   "active_entries": info["active"], "kernel_ms": {k: (v[0] / max(1, v[1])) for k, v in kern.items()},
                   "work_items": pinfo["items"], "l_tiles_per_item": pinfo["lp"], "ctas": pinfo["ctas"],
                   "device": props.name},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
