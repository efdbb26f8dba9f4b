"""Seeded synthetic water-like multipole boxes.

This module only draws inputs; it holds none of the method's arithmetic, and
both the CUDA path's tests/benchmark and the CPU oracle consume its output.

Recipe (stand-in for the paper's water boxes of Sec. 5.4: 648 atoms in
18.643 A, 96,000 / 288,000 / 864,000 atoms at liquid density):
  * rigid 3-site water: O -0.834 e, H +0.417 e, OH 0.9572 A, HOH 104.52 deg;
  * O atoms on a cubic lattice of m = ceil(Nw^(1/3)) sites per axis, spacing
    L/m; the first Nw sites of a seeded permutation are used, each jittered
    by U[-0.15, 0.15] * spacing per axis;
  * orientation: uniform random rotation (Shoemake's quaternion method);
  * box edge L = (Nw / 0.0334)^(1/3) A unless given;
  * dipoles: direction uniform on the sphere, magnitude U[0, 0.5] e A;
  * quadrupoles: six entries iid N(0, 0.3) e A^2, then tr/3 removed from the
    diagonal (traceless symmetric).
Positions are returned in float32 (what the GPU receives); the oracle reads
the same float32 values promoted to float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

WATER_DENSITY = 0.0334  # molecules per cubic Angstrom
SEED_BASE = 221208284


@dataclass
class Box:
    x: np.ndarray        # (N,3) float32, inside [-L/2, L/2)
    q: np.ndarray        # (N,) float32
    mu: np.ndarray       # (N,3) float32 (zeros when absent)
    theta: np.ndarray    # (N,6) float32 xx,xy,xz,yy,yz,zz (zeros when absent)
    box: float           # edge length L = 2 r_B (Angstrom)
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def _quat_rotations(rng, n):
    """Uniform random rotation matrices (Shoemake 1992)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    qw = a * np.sin(2 * np.pi * u2)
    qx = a * np.cos(2 * np.pi * u2)
    qy = b * np.sin(2 * np.pi * u3)
    qz = b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz)
    R[:, 0, 1] = 2 * (qx * qy - qz * qw)
    R[:, 0, 2] = 2 * (qx * qz + qy * qw)
    R[:, 1, 0] = 2 * (qx * qy + qz * qw)
    R[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz)
    R[:, 1, 2] = 2 * (qy * qz - qx * qw)
    R[:, 2, 0] = 2 * (qx * qz - qy * qw)
    R[:, 2, 1] = 2 * (qy * qz + qx * qw)
    R[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    return R


def water_box(n_waters: int, seed: int, box: float | None = None, multipoles: bool = True,
              name: str = "") -> Box:
    rng = np.random.default_rng(seed)
    if box is None:
        box = (n_waters / WATER_DENSITY) ** (1.0 / 3.0)
    m = int(math.ceil(n_waters ** (1.0 / 3.0) - 1e-9))
    spacing = box / m
    sites = rng.permutation(m ** 3)[:n_waters]
    ijk = np.stack([sites // (m * m), (sites // m) % m, sites % m], axis=1).astype(np.float64)
    O = -box / 2 + (ijk + 0.5) * spacing
    O += rng.uniform(-0.15, 0.15, size=O.shape) * spacing
    # body frame: O at origin, H in the xy plane symmetric about x
    half = math.radians(104.52) / 2.0
    d = 0.9572
    h1 = np.array([d * math.cos(half), d * math.sin(half), 0.0])
    h2 = np.array([d * math.cos(half), -d * math.sin(half), 0.0])
    R = _quat_rotations(rng, n_waters)
    H1 = O + R @ h1
    H2 = O + R @ h2
    x = np.stack([O, H1, H2], axis=1).reshape(-1, 3)
    # wrap into [-L/2, L/2)
    x = x - box * np.floor(x / box + 0.5)
    q = np.tile(np.array([-0.834, 0.417, 0.417]), n_waters)
    n = x.shape[0]
    mu = np.zeros((n, 3))
    th = np.zeros((n, 6))
    if multipoles:
        v = rng.normal(size=(n, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        mu = v * rng.uniform(0.0, 0.5, size=(n, 1))
        th = rng.normal(0.0, 0.3, size=(n, 6))
        tr = (th[:, 0] + th[:, 3] + th[:, 5]) / 3.0
        th[:, 0] -= tr
        th[:, 3] -= tr
        th[:, 5] -= tr
    x32 = x.astype(np.float32)
    # float32 rounding may land exactly on +L/2; keep the half-open box
    x32 = np.where(x32 >= np.float32(box / 2), x32 - np.float32(box), x32).astype(np.float32)
    return Box(x=x32, q=q.astype(np.float32), mu=mu.astype(np.float32),
               theta=th.astype(np.float32), box=float(box), name=name)


# The five workloads (sizes and structure of the paper's water benchmarks).
CONFIGS = {
    1: dict(n_waters=216, box=18.64, multipoles=False,
            name="water_648_q"),
    2: dict(n_waters=8000, box=None, multipoles=True,
            name="water_24000_qmuTheta"),
    3: dict(n_waters=32000, box=None, multipoles=True,
            name="water_96000_qmuTheta"),
    4: dict(n_waters=336000, box=None, multipoles=True,
            name="water_1008000_qmuTheta"),
}


def config_box(idx: int) -> Box:
    c = CONFIGS[idx]
    return water_box(c["n_waters"], SEED_BASE + idx, box=c["box"],
                     multipoles=c["multipoles"], name=c["name"])


def replica_sizes(n_boxes: int = 64, seed: int = SEED_BASE + 5):
    """Atom counts of the batched-replica workload: U[3000, 48000] rounded
    down to a multiple of 3."""
    rng = np.random.default_rng(seed)
    n = rng.integers(3000, 48001, size=n_boxes)
    return (n // 3) * 3


def replica_boxes(n_boxes: int = 64):
    sizes = replica_sizes(n_boxes)
    return [water_box(int(s) // 3, SEED_BASE + 5 + 1000 * (b + 1), multipoles=True,
                      name=f"replica_{b}") for b, s in enumerate(sizes)]


def small_box(n_waters: int, seed: int, box: float | None = None, multipoles: bool = True) -> Box:
    return water_box(n_waters, seed, box=box, multipoles=multipoles, name=f"water_{3*n_waters}")
