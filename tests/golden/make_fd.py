"""Central finite differences of the FP64 ANKH energy (the oracle's literal
ANKH-FFT) on 32 seeded atoms of the 96,000-atom workload.

The approximate energy is only piecewise smooth (an atom crossing a leaf face
switches pairs between near and far field), so the 32 atoms are drawn among
those at least 10 h_FD from every leaf face.  Parameters: the library's
default leaf count for this box with L_u = L_c = 5, xi = 0.01.

Usage:  python tests/golden/make_fd.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ankh_ref as ar                  # noqa: E402
from paper_2212_08284_gb300 import synth           # noqa: E402

H_FD = 1e-4
N_ATOMS = 32
N_CELLS = 25      # default leaf count of the library for this box (4.0 A target, n (L_u-1) = 100)
LU = 5


def main():
    b = synth.config_box(3)
    p = ar.Params(b.box, N_CELLS, LU, LU)
    x = b.x.astype(np.float64)
    h = b.box / N_CELLS
    frac = (x + b.box / 2) / h
    dist = np.min(np.abs(frac - np.round(frac)), axis=1) * h
    rng = np.random.default_rng(4242)
    cand = np.where(dist > 10 * H_FD)[0]
    atoms = np.sort(rng.choice(cand, N_ATOMS, replace=False))
    out = {"workload": b.name, "n_cells": N_CELLS, "Lu": LU, "Lc": LU, "xi": 0.01, "h_fd": H_FD,
           "atoms": atoms.tolist(), "fd_dEdx": []}
    t0 = time.time()
    for i in atoms:
        g = []
        for c in range(3):
            xp = x.copy(); xp[i, c] += H_FD
            xm = x.copy(); xm[i, c] -= H_FD
            ep = ar.ankh_energy(xp, b.q, b.mu, b.theta, p, grad=False)["E"]
            em = ar.ankh_energy(xm, b.q, b.mu, b.theta, p, grad=False)["E"]
            g.append((ep - em) / (2 * H_FD))
        out["fd_dEdx"].append(g)
        print(f"atom {i}: {g} ({time.time() - t0:.0f} s)", flush=True)
    with open(os.path.join(HERE, f"fd_{b.name}.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
