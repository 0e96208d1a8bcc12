"""Writes the expected C_l of the 1-source, l_max = 5000 workload.

The values come from the FP64 CPU oracle alone (oracle/, the dense discrete
sums of Eqs. (1)-(2)), on inputs from the seeded generator
paper_2509_25110_gb300.synth: 3000 k log-spaced on [1e-5, 1] 1/Mpc, 2000 tau
nodes (1000 uniform on [200, 600) Mpc around the visibility peak, 1000
uniform on [600, 14000]), tau0 = 14000 Mpc, l = 2..5000, source parameters of
seed 0, model 0.  Two columns: C_l of the FP64 sources, and C_l of the same
sources rounded to FP32 (the input of the FP32 path).  Nothing here calls
the CUDA library.

    python tests/golden/make_plain_lmax5000.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "plain_lmax5000_cl.txt")


def main():
    import oracle
    from paper_2509_25110_gb300 import synth

    wl = synth.workload("plain_lmax5000")
    p = synth.model_params(1, seed=0)
    S = synth.sources(wl.k, wl.tau, p)
    P = synth.primordial(wl.k, p)
    # both source precisions in one oracle call (they share each j_l evaluation)
    S2 = np.concatenate([S, S.astype(np.float32).astype(np.float64)])
    P2 = np.concatenate([P, P])
    _, c = oracle.los_cl(wl.k, wl.tau, wl.tau0, wl.lmin, wl.lmax, S2, P2, want_delta=False)
    c64, c32 = c[0:1], c[1:2]
    ls = np.arange(wl.lmin, wl.lmax + 1)
    with open(OUT, "w") as f:
        f.write("# C_l of the plain_lmax5000 workload (1 source, seed 0): FP64 CPU oracle, Eqs. (1)-(2)\n")
        f.write("# written by tests/golden/make_plain_lmax5000.py (oracle + seeded inputs only)\n")
        f.write("# columns: l, C_l (FP64 sources), C_l (sources rounded to FP32)\n")
        for l, a, b in zip(ls, c64[0], c32[0]):
            f.write("%d %.17e %.17e\n" % (l, a, b))


if __name__ == "__main__":
    main()
