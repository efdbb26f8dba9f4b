"""Central finite differences of the FP64 ANKH energy (the oracle's literal
ANKH-FFT) on 32 seeded atoms of the 96,000-atom workload.

fd_dEdx: dE/dx by moving one atom by +-h_FD along each axis.  The
approximate energy is only piecewise smooth (an atom crossing a leaf face
switches pairs between near and far field), so the 32 atoms are drawn among
those at least 10 h_FD from every leaf face.

fd_torque: for the first 8 of those atoms, tau . n = -dE/d(eps) where the
atom's dipole and quadrupole are rotated rigidly by the angle eps about the
axis n = x, y, z (mu -> R mu, Theta -> R Theta R^T, R by Rodrigues' formula;
the position does not move, so no leaf face is crossed).

Parameters: the library's default leaf count for this box with
L_u = L_c = 5, xi = 0.01.

Usage:  python tests/golden/make_fd.py [--torque-only]
   (--torque-only keeps fd_dEdx of an existing output file)
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
EPS_ROT = 1e-4
N_ATOMS = 32
N_TORQUE = 8
N_CELLS = 25      # default leaf count of the library for this box (4.0 A target, n (L_u-1) = 100)
LU = 5


def rotation(axis: int, eps: float) -> np.ndarray:
    """Rodrigues: rotation by eps about the unit vector e_axis."""
    k = np.zeros((3, 3))
    a, b = [(1, 2), (2, 0), (0, 1)][axis]
    k[b, a], k[a, b] = 1.0, -1.0           # k v = e_axis x v
    return np.eye(3) + np.sin(eps) * k + (1.0 - np.cos(eps)) * (k @ k)


def rotated(mu, theta, i, axis, eps):
    r = rotation(axis, eps)
    mu2, th2 = mu.copy(), theta.copy()
    mu2[i] = r @ mu[i]
    t = theta[i]
    T = np.array([[t[0], t[1], t[2]], [t[1], t[3], t[4]], [t[2], t[4], t[5]]])
    T2 = r @ T @ r.T
    th2[i] = [T2[0, 0], T2[0, 1], T2[0, 2], T2[1, 1], T2[1, 2], T2[2, 2]]
    return mu2, th2


def main():
    torque_only = "--torque-only" in sys.argv
    b = synth.config_box(3)
    p = ar.Params(b.box, N_CELLS, LU, LU)
    x = b.x.astype(np.float64)
    mu = b.mu.astype(np.float64)
    theta = b.theta.astype(np.float64)
    path = os.path.join(HERE, f"fd_{b.name}.json")
    h = b.box / N_CELLS
    frac = (x + b.box / 2) / h
    dist = np.min(np.abs(frac - np.round(frac)), axis=1) * h
    rng = np.random.default_rng(4242)
    cand = np.where(dist > 10 * H_FD)[0]
    atoms = np.sort(rng.choice(cand, N_ATOMS, replace=False))
    out = {"workload": b.name, "n_cells": N_CELLS, "Lu": LU, "Lc": LU, "xi": 0.01, "h_fd": H_FD,
           "atoms": atoms.tolist(), "fd_dEdx": []}
    t0 = time.time()
    if torque_only:
        old = json.load(open(path))
        assert old["atoms"] == out["atoms"]
        out["fd_dEdx"] = old["fd_dEdx"]
    else:
        for i in atoms:
            g = []
            for c in range(3):
                xp = x.copy(); xp[i, c] += H_FD
                xm = x.copy(); xm[i, c] -= H_FD
                ep = ar.ankh_energy(xp, b.q, mu, theta, p, grad=False)["E"]
                em = ar.ankh_energy(xm, b.q, mu, theta, p, grad=False)["E"]
                g.append((ep - em) / (2 * H_FD))
            out["fd_dEdx"].append(g)
            print(f"atom {i}: {g} ({time.time() - t0:.0f} s)", flush=True)
    out["eps_rot"] = EPS_ROT
    out["torque_atoms"] = atoms[:N_TORQUE].tolist()
    out["fd_torque"] = []
    for i in atoms[:N_TORQUE]:
        tq = []
        for c in range(3):
            mp, tp = rotated(mu, theta, i, c, EPS_ROT)
            mm, tm = rotated(mu, theta, i, c, -EPS_ROT)
            ep = ar.ankh_energy(x, b.q, mp, tp, p, grad=False)["E"]
            em = ar.ankh_energy(x, b.q, mm, tm, p, grad=False)["E"]
            tq.append(-(ep - em) / (2 * EPS_ROT))
        out["fd_torque"].append(tq)
        print(f"torque atom {i}: {tq} ({time.time() - t0:.0f} s)", flush=True)
    with open(path, "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
