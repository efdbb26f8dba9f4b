"""Write the method-error map of ANKH-FFT on the water workloads.

For each water box, equispaced order L_u (L_c = L_u) and leaf count n, the
oracle's literal FP64 ANKH-FFT (oracle/ankh_ref.py) is compared with the
FP64 Ewald reference of the same box (tests/golden/ewald_*.json, written by
make_golden.py from the oracle): relative energy error and relative RMS
force error over the golden's sampled atoms (of the RMS force over all
atoms).  This is the error of the method itself at matched parameters, with
no GPU arithmetic in it; the library's accuracy table (the smallest leaf
edge allowed for each L_u) is read off this map.  Calls only the oracle.

Usage:  python tests/golden/make_error_map.py [config ...] [--Lu 4,5,6,7] [--h 3.0,6.5]
Results are merged into tests/golden/error_map.json (keyed by box, L_u, n).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import ankh_ref as ar                   # noqa: E402
from paper_2212_08284_gb300 import synth            # noqa: E402


def workload(c: int):
    """Config c of the benchmark (1-4), or 0: the 3,000-atom water box with
    q, mu, Theta in a 31.1 A box that the GPU tests use (seed 31)."""
    return synth.small_box(1000, 31, box=31.1) if c == 0 else synth.config_box(c)

OUT = os.path.join(HERE, "error_map.json")


def load():
    if os.path.exists(OUT):
        return json.load(open(OUT))
    return {"description": __doc__.split("\n\n")[1].replace("\n", " "), "entries": []}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("configs", nargs="*", type=int, default=[1, 2, 3])
    ap.add_argument("--Lu", default="4,5,6,7")
    ap.add_argument("--h", default="3.0,6.5", help="leaf-edge range in Angstrom")
    ap.add_argument("--n", default="", help="explicit leaf counts (overrides --h)")
    a = ap.parse_args()
    Lus = [int(v) for v in a.Lu.split(",")]
    hlo, hhi = (float(v) for v in a.h.split(","))
    data = load()
    have = {(e["box"], e["Lu"], e["n"]) for e in data["entries"]}
    for c in a.configs:
        b = workload(c)
        gd = json.load(open(os.path.join(HERE, f"ewald_{b.name}.json")))
        idx = np.array(gd["sample_idx"])
        ref = np.array(gd["sample_grad"])
        ns = ([int(v) for v in a.n.split(",")] if a.n else
              [n for n in range(3, 200) if hlo <= b.box / n <= hhi])
        for Lu in Lus:
            for n in ns:
                if (b.name, Lu, n) in have:
                    continue
                t0 = time.time()
                grad = c != 1                                   # config 1 is charges only, energy only
                o = ar.ankh_energy(b.x, b.q, b.mu, b.theta, ar.Params(b.box, n, Lu, Lu), grad=grad)
                e = {"box": b.name, "n_atoms": b.n, "box_A": b.box, "Lu": Lu, "n": n, "h_A": b.box / n,
                     "rel_energy_error": abs(o["E"] - gd["E"]) / abs(gd["E"]),
                     "rel_rms_force_error": (float(np.sqrt(np.mean((o["grad"][idx, :3] - ref[:, :3]) ** 2))
                                                   / gd["rms_all"]["dEdx"]) if grad else None),
                     "seconds": round(time.time() - t0, 2)}
                data["entries"].append(e)
                have.add((b.name, Lu, n))
                data["entries"].sort(key=lambda r: (r["n_atoms"], r["Lu"], r["n"]))
                json.dump(data, open(OUT, "w"), indent=1)
                print(json.dumps(e), flush=True)


if __name__ == "__main__":
    main()
