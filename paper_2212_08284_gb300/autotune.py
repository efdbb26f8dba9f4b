"""Leaf-count and order autotuner, constrained by the library's accuracy table.

The candidates are the (n, L_u) pairs that the accuracy table allows for the
box (ankh_accuracy_rule: the leaf-edge range over which the method's own
error stayed within 3e-6 relative energy and 3e-5 relative RMS force on the
calibration water boxes of the box's size class) and whose merged grid the
library's FFT takes.  Within those, n only trades work -- near-field pairs
grow like h^3; the adjacent-leaf correction, the merged FFT grid and the
P2M/L2P node work like h^-3 and with the order -- so the autotuner measures
one full energy + gradient evaluation on the device (CUDA events around the
library call) for each candidate and returns the fastest.  Where the table
calibrates nothing for the box (an explicit order it does not cover, a box
with multipoles below 24,000 atoms), the candidates are leaf counts around a
4.0 A leaf edge at that order or L_u = 6 (no accuracy guarantee).  Results are cached
per (box, N, order, precision) for the life of the process.
"""
from __future__ import annotations

import math

from . import api

_cache: dict = {}


def smooth(m: int) -> bool:
    """True when m has no prime factor above 7 (the lengths the FFT takes)."""
    if m < 1:
        return False
    for p in (2, 3, 5, 7):
        while m % p == 0:
            m //= p
    return m == 1


def next_smooth(m: int) -> int:
    while not smooth(m):
        m += 1
    return m


def grid_ok(n: int, Lu: int, nonperiodic: bool = False) -> bool:
    ng = next_smooth(2 * (n * (Lu - 1) + 1) - 1) if nonperiodic else n * (Lu - 1)
    return ng <= 1024 and smooth(ng)


def allowed(box: float, n_atoms: int, Lu: int, nonperiodic: bool = False, per_order: int = 4,
            max_order: int = 2) -> list[int]:
    """Leaf counts the accuracy table allows at order Lu (largest first, at
    most per_order of them), or [] when Lu is not calibrated for the box."""
    rule = api.ankh_accuracy_rule(n_atoms, Lu, max_order)
    if rule is None:
        return []
    hmin, hmax = rule
    out = [n for n in range(int(math.floor(box / hmin)), 2, -1)
           if hmin <= box / n <= hmax and grid_ok(n, Lu, nonperiodic)]
    return out[:per_order]


def candidates(box: float, n_atoms: int, Lu: int = 0, nonperiodic: bool = False, spread: int = 4,
               h0: float = 4.0, max_order: int = 2) -> list[tuple[int, int]]:
    """(n, L_u) pairs to time: every calibrated order's allowed leaf counts
    (Lu = 0), one order's (Lu > 0), or, for an uncalibrated explicit order,
    the leaf counts within `spread` of a 4 A leaf edge."""
    orders = range(2, 9) if Lu == 0 else [Lu]
    out = [(n, L) for L in orders for n in allowed(box, n_atoms, L, nonperiodic, max_order=max_order)]
    if not out:
        # not calibrated (a box with multipoles below the smallest class):
        # leaf counts near a 4 A leaf edge at the given order, or L_u = 6
        Lu = Lu or 6
        n0 = max(3, int(round(box / h0)))
        out = [(n, Lu) for n in sorted({max(3, n0 + d) for d in range(-spread, spread + 1)})
               if grid_ok(n, Lu, nonperiodic)]
    return out


def autotune(box: float, x, q, mu=None, theta=None, Lu: int = 0, mixed: bool = True, max_order: int = 2,
             cands: list[tuple[int, int]] | None = None, reps: int = 4, warm: int = 2,
             nonperiodic: bool = False):
    """Return ((n, L_u) fastest, {"n,Lu": milliseconds per evaluation})."""
    import torch
    n_atoms = int(x.shape[0])
    key = (round(box, 6), n_atoms, Lu, mixed, max_order, nonperiodic)
    if key in _cache and cands is None:
        return _cache[key]
    dev = x.device
    out = {"dEdx": torch.empty((n_atoms, 3), device=dev), "dEdq": torch.empty(n_atoms, device=dev),
           "dEdmu": torch.empty((n_atoms, 3), device=dev), "dEdtheta": torch.empty((n_atoms, 6), device=dev)}
    table = {}
    stream = torch.cuda.current_stream()
    for n, L in (cands or candidates(box, n_atoms, Lu, nonperiodic, max_order=max_order)):
        try:
            m = api.Ankh(box, n_atoms, n_cells=n, Lu=L, Lc=L, mixed=mixed, max_order=max_order,
                         nonperiodic=nonperiodic)
        except api.AnkhError:
            continue                     # not creatable (e.g. grid too large): never chosen
        for _ in range(warm):
            api.ankh_energy_forces(m.h, x, q, mu, theta, sync=False, stream=stream, **out)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            api.ankh_energy_forces(m.h, x, q, mu, theta, sync=False, stream=stream, **out)
        e1.record(stream)
        e1.synchronize()
        table[(n, L)] = e0.elapsed_time(e1) / reps
        # one call that reads the energy and the error flag: a kernel that ran
        # into a bounded wait (ANKH_ETIMEOUT) or a numeric error stops the
        # search here instead of after every candidate
        api.ankh_energy_forces(m.h, x, q, mu, theta, stream=stream, **out)
        m.close()
    if not table:
        raise RuntimeError("no candidate (leaf count, order) could be created")
    best = min(table, key=table.get)
    res = (best, {f"{k[0]},{k[1]}": v for k, v in sorted(table.items())})
    if cands is None:
        _cache[key] = res
    return res
