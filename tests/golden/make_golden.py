"""Write the FP64 Ewald reference values of the water workloads.

Calls only the oracle (oracle/ewald.py) on the seeded inputs of
paper_2212_08284_gb300/synth.py and stores, per workload:
  * the total energy and its Ewald parts (tin-foil, e^2/A);
  * the gradient rows (dE/dx, dE/dq, dE/dmu, dE/dTheta) of a seeded sample
    of atoms, and the RMS over ALL atoms of each gradient group.

Usage:  python tests/golden/make_golden.py 0 1 2 3 4   (0: the 3,000-atom test box)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import ewald as ew                      # noqa: E402
from paper_2212_08284_gb300 import synth            # noqa: E402


def workload(c: int):
    """Config c of the benchmark (1-4), or 0: the 3,000-atom water box with
    q, mu, Theta in a 31.1 A box that the GPU tests use (seed 31)."""
    return synth.small_box(1000, 31, box=31.1) if c == 0 else synth.config_box(c)

N_SAMPLE = 2048


def main(cfgs):
    for c in cfgs:
        b = workload(c)
        mp = ew.pack_multipoles(b.q, b.mu, b.theta)
        t0 = time.time()
        r = ew.ewald(b.x.astype(np.float64), mp, b.box, tol=1e-11, grad=True)
        dt = time.time() - t0
        g = r["grad"]
        rng = np.random.default_rng(1000 + c)
        n = b.n
        idx = np.sort(rng.choice(n, size=min(N_SAMPLE, n), replace=False))
        rms = lambda a: float(np.sqrt(np.mean(a * a)))
        out = {
            "workload": b.name, "n_atoms": n, "box": b.box,
            "E": r["E"], "E_real": r["E_real"], "E_rec": r["E_rec"], "E_self": r["E_self"],
            "E_neut": r["E_neut"], "alpha": r["alpha"], "rc": r["rc"], "kc": r["kc"],
            "tol": 1e-11, "seconds": dt, "threads": ew.nthreads_default(),
            "rms_all": {"dEdx": rms(g[:, 0:3]), "dEdq": rms(g[:, 3]), "dEdmu": rms(g[:, 4:7]),
                        "dEdtheta": rms(g[:, 7:13])},
            "sample_idx": idx.tolist(),
            "sample_grad": g[idx].tolist(),
            "input_checksum": float(np.sum(b.x.astype(np.float64) * np.arange(1, n + 1)[:, None] % 7.0)),
        }
        with open(os.path.join(HERE, f"ewald_{b.name}.json"), "w") as f:
            json.dump(out, f)
        print(f"config {c}: N={n} E={r['E']:.12f} ({dt:.1f} s)", flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [1, 2, 3])
