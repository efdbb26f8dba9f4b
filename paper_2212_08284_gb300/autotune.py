"""Leaf-size autotuner.

The ANKH error is scale-free in the leaf edge h (xi h << 1), so the number
of leaves per axis n only trades work: near-field pairs grow like h^3, the
adjacent-leaf correction, the merged FFT grid and the P2M/L2P node work like
h^-3, and the near-field kernel's lane use depends on the atoms per leaf.
The autotuner measures one full energy + gradient evaluation on the device
(CUDA events around the library call) for candidate n around a 4.0 A leaf
edge, extends the window while the fastest count sits at its edge, and
returns the fastest.  Results are cached per (box, N, orders,
precision) for the life of the process.
"""
from __future__ import annotations

import math

from . import api

_cache: dict = {}


def smooth(m: int) -> bool:
    """True when m has no prime factor above 7 (the lengths the FFT takes)."""
    for p in (2, 3, 5, 7):
        while m % p == 0:
            m //= p
    return m == 1


def candidates(box: float, spread: int = 4, h0: float = 4.0, Lu: int = 5) -> list[int]:
    n0 = max(3, int(round(box / h0)))
    return sorted({max(3, n0 + d) for d in range(-spread, spread + 1) if smooth(max(3, n0 + d) * (Lu - 1))})


def autotune_n(box: float, x, q, mu=None, theta=None, Lu: int = 5, Lc: int = 0, mixed: bool = True,
               max_order: int = 2, cands: list[int] | None = None, reps: int = 4, warm: int = 2,
               nonperiodic: bool = False):
    """Return (best n, {n: milliseconds per evaluation})."""
    import torch
    key = (round(box, 6), int(x.shape[0]), Lu, Lc, mixed, max_order, nonperiodic)
    if key in _cache:
        return _cache[key]
    n_atoms = int(x.shape[0])
    dev = x.device
    out = {"dEdx": torch.empty((n_atoms, 3), device=dev), "dEdq": torch.empty(n_atoms, device=dev),
           "dEdmu": torch.empty((n_atoms, 3), device=dev), "dEdtheta": torch.empty((n_atoms, 6), device=dev)}
    table = {}
    stream = torch.cuda.current_stream()

    def measure(n):
        try:
            m = api.Ankh(box, n_atoms, n_cells=n, Lu=Lu, Lc=Lc, mixed=mixed, max_order=max_order,
                         nonperiodic=nonperiodic)
        except api.AnkhError:
            table[n] = math.inf          # not creatable (grid too large): never chosen
            return
        for _ in range(warm):
            api.ankh_energy_forces(m.h, x, q, mu, theta, sync=False, stream=stream, **out)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            api.ankh_energy_forces(m.h, x, q, mu, theta, sync=False, stream=stream, **out)
        e1.record(stream)
        e1.synchronize()
        table[n] = e0.elapsed_time(e1) / reps
        m.close()

    for n in (cands or candidates(box)):
        measure(n)
    if cands is None:
        # while the fastest count sits at an edge of the window, extend the
        # window past that edge (two counts at a time, at most 12 more)
        for _ in range(6):
            done = {k: v for k, v in table.items() if math.isfinite(v)}
            if not done:
                break
            best = min(done, key=done.get)
            if best == max(table):
                ext = [best + 1, best + 2]
            elif best == min(table) and best > 3:
                ext = [k for k in (best - 1, best - 2) if k >= 3]
            else:
                break
            for n in ext:
                measure(n)
    table = {k: v for k, v in table.items() if math.isfinite(v)}
    if not table:
        raise RuntimeError("no candidate leaf count could be created")
    best = min(table, key=table.get)
    _cache[key] = (best, table)
    return best, table
