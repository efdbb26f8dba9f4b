"""Benchmark: ANKH energy + forces evaluations per second on a synthetic
1,008,000-atom water box with charges, dipoles and quadrupoles.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload water_1008000|water_96000|water_24000] [--plain]
                  [--nonperiodic | --induce | --fmm]

One "step" is one full evaluation (bin/sort, P2M, merged-grid FFT far field,
adjacent-leaf correction, near field, L2P, gradient assembly, FP64 energy)
on inputs already resident in HBM; L2 is flushed (256 MiB write) between
timed steps and the step is timed with CUDA events on the launch stream.
Under torchrun each rank evaluates its own independent box (replicas; no
data-path collective), and the value is the whole-job rate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {"water_1008000": 4, "water_96000": 3, "water_24000": 2, "replicas64": 5}
METRIC = "energy+force evals/s and Matoms/s at <=1e-5 rel. energy error vs FP64 Ewald"
UNIT = "evals/s"
# Algorithmic FP32 work of the near field per UNORDERED pair of atoms in
# adjacent leaves: 400 flop for the energy, forces, fields and field gradients
# of both atoms (FMA = 2).  The kernel evaluates every ordered pair once in its
# source-field form, 262 flop each (150 for the potential, field and field
# gradient, 112 for the quadrupole force), i.e. 524 flop per unordered pair
# executed; both rates are reported.
NEAR_FLOPS_PER_PAIR = 400
NEAR_FLOPS_EXECUTED_PER_ORDERED_PAIR = 262
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per launch from one ncu capture of the same kernel
# code on the same workload and leaf count; keyed by (kernel, workload, n, L_u).
# Entries are removed whenever the kernel changes and re-measured.
DRAM_TRAFFIC: dict = {
    # stage: kernels (read + write per launch); the timed evaluation, ncu, one pass per kernel
    ("near", "water_1008000_qmuTheta", 54, 5): 95.81e6,      # k_near (one-warp blocks)
    ("corr", "water_1008000_qmuTheta", 54, 5): 336.45e6,     # k_split_f16 + k_corr_tc
    ("p2m", "water_1008000_qmuTheta", 54, 5): 93.69e6,       # k_p2m
    ("l2p", "water_1008000_qmuTheta", 54, 5): 368.92e6,      # k_l2p
}


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, name):
        """Wall-clock mark (the start or end of the timed region)."""
        setattr(self, name, time.time())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons, inside = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "load_start", None), getattr(self, "timed_end", None)
        ts0 = getattr(self, "timed_start", None)
        for tr, ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 10:
                continue
            # samples while the GPU runs the step: the untimed pre-roll and the timed region
            if t0 is not None and t1 is not None and not (t0 <= tr <= t1 + 0.06):
                continue
            try:
                sm.append(float(p[2]))
                mx = float(p[3])
            except ValueError:
                continue
            if ts0 is not None and ts0 <= tr <= t1 + 0.06:
                inside += 1
            for nm, v in zip(names, p[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm), "samples_in_timed_region": inside,
                "sampling": "nvidia-smi every 50 ms while the step runs (an untimed pre-roll of the same "
                            "step, then the timed steps)"}


def preroll(clocks, step, seconds=0.4):
    """Start the clock sampler and run the untimed step for `seconds` so that
    the samples (and the clocks) are those of the loaded GPU; marks the start
    of the timed region."""
    import torch
    clocks.start()
    time.sleep(0.15)                    # the sampler process starts
    clocks.mark("load_start")
    t = time.perf_counter()
    while time.perf_counter() - t < seconds:
        step()
        torch.cuda.synchronize()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def unordered_near_pairs(start: np.ndarray, n: int, nonperiodic: bool = False) -> int:
    cnt = np.diff(start.astype(np.int64)).reshape(n, n, n)
    if nonperiodic:
        pad = np.pad(cnt, 1)
        shifted = lambda dx, dy, dz: pad[1 + dx:n + 1 + dx, 1 + dy:n + 1 + dy, 1 + dz:n + 1 + dz]
    else:
        shifted = lambda dx, dy, dz: np.roll(cnt, (-dx, -dy, -dz), axis=(0, 1, 2))
    tot = 0
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                tot += int(np.sum(cnt * shifted(dx, dy, dz)))
    return (tot - int(cnt.sum())) // 2


def oracle_sample(box, nthreads: int | None = None, rows: int = 1000, kstride: int = 400):
    """Time the FP64 Ewald oracle on a bounded sample of the workload and
    extrapolate to one full energy + gradient evaluation.

    Real space: the rows (target atoms) of a random subset, timed at `rows`
    and 2 `rows`; reciprocal space: every `kstride`-th and every
    (`kstride`/2)-th k-vector.  The two sizes separate the fixed cost of a
    call (cell lists, setup: paid once per evaluation) from the cost per row
    or per k-vector (scaled to all atoms / all k-vectors)."""
    from oracle import ewald as ew
    x = box.x.astype(np.float64)
    mp = ew.pack_multipoles(box.q, box.mu, box.theta)
    alpha, rc, kc = ew.ewald_params(box.box, box.n, tol=1e-11)
    rng = np.random.default_rng(7)
    r1, r2 = min(rows, box.n), min(2 * rows, box.n)
    pick = rng.choice(box.n, size=r2, replace=False)
    t = []
    t0 = time.perf_counter()
    for r in (r1, r2):
        a = time.perf_counter()
        ew.ewald_real_rows(x, mp, box.box, alpha, rc, np.sort(pick[:r]), grad=True, nthreads=nthreads)
        t.append(time.perf_counter() - a)
    per_row = max(t[1] - t[0], 0.0) / max(r2 - r1, 1)
    real_full = max(t[0] - r1 * per_row, 0.0) + box.n * per_row
    k2 = max(kstride // 2, 1)
    tk = []
    for ks in (kstride, k2):
        a = time.perf_counter()
        ew.ewald_rec_only(x, mp, box.box, alpha, kc, grad=True, kstride=ks, nthreads=nthreads)
        tk.append(time.perf_counter() - a)
    # fraction of k-vectors sampled: 1/ks;  t = fixed + K/ks * per_k
    per_kfrac = max(tk[1] - tk[0], 0.0) / max(1.0 / k2 - 1.0 / kstride, 1e-30)
    rec_full = max(tk[0] - per_kfrac / kstride, 0.0) + per_kfrac
    full = real_full + rec_full
    return {"seconds_full_eval": full, "sample": (f"FP64 Ewald (alpha={alpha:.4f}, rc={rc:.1f} A, tol 1e-11): "
                                                 f"real-space rows of {r1} and {r2} of {box.n} atoms + every "
                                                 f"{kstride}-th and {k2}-th reciprocal k-vector, energy + gradient; "
                                                 f"fixed + per-row / per-k-vector costs fitted and extrapolated "
                                                 f"to one full evaluation"),
            "sample_seconds": time.perf_counter() - t0}


def oracle_ankh_sample(box, Lu: int):
    """The algorithm-matched CPU number: the oracle's literal FP64 ANKH-FFT
    (energy + gradient) on the 96,000-atom water box at the leaf edge nearest
    the GPU's default (about 4 A), scaled by atoms to this workload (all its
    stages are linear in N at fixed density, except the FFT)."""
    from oracle import ankh_ref as ar
    from paper_2212_08284_gb300 import synth
    sb = synth.config_box(3)
    n = max(3, int(round(sb.box / 4.0)))
    a = time.perf_counter()
    ar.ankh_energy(sb.x, sb.q, sb.mu, sb.theta, ar.Params(sb.box, n, Lu, Lu), grad=True)
    ts = time.perf_counter() - a
    return {"value": 1.0 / (ts * box.n / sb.n), "unit": UNIT, "cores": os.cpu_count() or 1,
            "kind": "oracle (FP64 ANKH-FFT, algorithm-matched)",
            "sample": f"oracle ANKH-FFT energy + gradient of the {sb.n}-atom water box, n = {n}, L_u = L_c = {Lu} "
                      f"({ts:.1f} s), scaled by atoms ({box.n}/{sb.n})"}


def oracle_sample_nonperiodic(box, nthreads: int | None = None, rows: int = 64):
    """Time the FP64 non-periodic direct sum on the gradient rows of `rows` and
    2 `rows` atoms (all sources each) and extrapolate the fitted per-row cost
    to one full energy + gradient evaluation (N rows)."""
    from oracle import ewald as ew
    x = box.x.astype(np.float64)
    mp = ew.pack_multipoles(box.q, box.mu, box.theta)
    pick = np.random.default_rng(7).choice(box.n, size=min(2 * rows, box.n), replace=False)
    t = []
    t0 = time.perf_counter()
    for r in (rows, 2 * rows):
        a = time.perf_counter()
        ew.direct_nonperiodic_rows(x, mp, np.sort(pick[:r]), nthreads=nthreads)
        t.append(time.perf_counter() - a)
    per_row = max(t[1] - t[0], 0.0) / rows
    full = max(t[0] - rows * per_row, 0.0) + box.n * per_row
    return {"seconds_full_eval": full, "sample": (f"FP64 non-periodic direct sum: gradient rows of {rows} and "
                                                 f"{2 * rows} of {box.n} atoms (all sources), fixed + per-row "
                                                 f"cost fitted and extrapolated to one full evaluation"),
            "sample_seconds": time.perf_counter() - t0}


def oracle_time(box, nthreads=None):
    """Seconds of one FP64 Ewald energy + gradient evaluation of the box on the
    host cores: the full oracle for boxes up to 5,000 atoms, else the bounded
    sample of oracle_sample extrapolated to a full evaluation."""
    if box.n <= 5000:
        from oracle import ewald as ew
        mp = ew.pack_multipoles(box.q, box.mu, box.theta)
        a = time.perf_counter()
        ew.ewald(box.x.astype(np.float64), mp, box.box, tol=1e-11, grad=True, nthreads=nthreads)
        return time.perf_counter() - a, f"FP64 Ewald oracle, full energy + gradient of the {box.n}-atom box"
    rows, kstride = (500, 400) if nthreads != 1 else (100, 2000)   # bounded: seconds of host time
    r = oracle_sample(box, nthreads=nthreads, rows=rows, kstride=kstride)
    return r["seconds_full_eval"], r["sample"]


def time_device(fn, steps, flush, stream):
    """Mean device time of one call: CUDA events on the launch stream around
    each call, L2 flushed before each, after three warm-up calls."""
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    tot = 0.0
    for k in range(steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1) / 1e3
    return tot / steps


def golden_errors(box, E, dEdx=None):
    """Relative energy error and sampled relative RMS force error against the
    FP64 Ewald reference of the box (tests/golden), or None without one."""
    gpath = os.path.join(ROOT, "tests", "golden", f"ewald_{box.name}.json")
    if not os.path.exists(gpath):
        return None
    gd = json.load(open(gpath))
    acc = {"rel_energy_error": abs(E - gd["E"]) / abs(gd["E"]), "reference": "FP64 Ewald oracle (tests/golden)"}
    if dEdx is not None:
        idx = np.array(gd["sample_idx"])
        ref = np.array(gd["sample_grad"])
        gx = dEdx.cpu().numpy().astype(np.float64)[idx]
        acc["rel_rms_force_error_sample"] = float(np.sqrt(np.mean((gx - ref[:, :3]) ** 2)) / gd["rms_all"]["dEdx"])
    return acc


def config_legs(args, dev, api, synth, flush, stream, steps):
    """The smaller water workloads at the library's default parameters (leaf
    count and order from its accuracy table): 648 atoms charges only (energy),
    24,000 atoms q/mu/Theta (energy), 96,000 atoms q/mu/Theta (energy, forces
    and torques); each with its error against the FP64 Ewald reference and the
    same-run oracle time on the host cores (and on one core for the two
    smallest)."""
    import torch
    legs = []
    for c in (1, 2, 3):
        box = synth.config_box(c)
        f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        x, q, mu, th = f32(box.x), f32(box.q), f32(box.mu), f32(box.theta)
        order = 0 if c == 1 else 2
        m = api.Ankh(box.box, box.n, n_cells=0, Lu=0, max_order=order)
        info = m.info
        forces = c == 3
        out = {"dEdx": torch.empty((box.n, 3), device=dev), "dEdq": torch.empty(box.n, device=dev),
               "dEdmu": torch.empty((box.n, 3), device=dev), "dEdtheta": torch.empty((box.n, 6), device=dev),
               "torque": torch.empty((box.n, 3), device=dev)}
        if forces:
            fn = lambda: api.ankh_energy_forces(m.h, x, q, mu, th, sync=False, stream=stream, **out)
        else:
            fn = lambda: api.ankh_energy(m.h, x, q, mu, th, stream=stream)
        t = time_device(fn, steps, flush, stream)
        E = (api.ankh_energy_forces(m.h, x, q, mu, th, stream=stream, **out) if forces
             else api.ankh_energy(m.h, x, q, mu, th, stream=stream))
        m.close()
        ot, osample = oracle_time(box)
        rec = {"config": c, "workload": box.name + ("_energy_forces_torques" if forces else "_energy"),
               "n_atoms": box.n, "box_A": round(box.box, 4), "n_cells": info["n_cells"], "Lu": info["Lu"],
               "call": "ankh_energy_forces" if forces else "ankh_energy (returns the energy: includes its sync)",
               "evals_per_s": 1.0 / t, "ms_per_eval": t * 1e3, "matoms_per_s": box.n / t / 1e6,
               "accuracy": golden_errors(box, E, out["dEdx"] if forces else None),
               "oracle": {"seconds_per_eval": ot, "cores": os.cpu_count() or 1, "sample": osample}}
        if c <= 2:
            ot1, _ = oracle_time(box, nthreads=1)
            rec["oracle"]["seconds_per_eval_one_core"] = ot1
        legs.append(rec)
    return legs


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, on the host cores."""
    from paper_2212_08284_gb300 import synth
    if rank != 0:
        return
    cfg = WORKLOADS[args.workload]
    box = synth.config_box(cfg)
    cores = os.cpu_count() or 1
    # sample size per step so that the whole run stays within ~3 minutes
    # (rows = 1000 / kstride = 400 take ~30 s on 16 host cores)
    f = min(1.0, max(0.1, 180.0 / (30.0 * max(args.steps + args.warmup, 1))))
    rows, kstride = max(50, int(1000 * f)), max(8, int(400 / f))
    for _ in range(args.warmup):
        oracle_sample(box, rows=rows, kstride=kstride)
    times, samples = [], []
    for _ in range(args.steps):
        r = oracle_sample(box, rows=rows, kstride=kstride)
        times.append(r["seconds_full_eval"])
        samples.append(r["sample_seconds"])
    per_eval = statistics.median(times)
    value = 1.0 / per_eval
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_eval * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": box.name + "_energy_forces", "n_atoms": box.n,
                                             "box_A": box.box},
            "matoms_per_s": value * box.n / 1e6,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def lpt_partition(costs, nparts):
    """Longest-processing-time greedy: items in decreasing cost (ties by
    index), each to the least-loaded part (ties to the lowest part index).
    Returns the sorted item indices of every part."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * nparts
    parts = [[] for _ in range(nparts)]
    for i in order:
        p = min(range(nparts), key=lambda k: (load[k], k))
        parts[p].append(i)
        load[p] += costs[i]
    return [sorted(p) for p in parts]


def max_over_ranks(value, dist, device):
    """The largest value over all ranks (the job's time is its slowest rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_measure(args, rank, world, dev, api, synth, dist=None, steps=None, e2e_steps=None,
                     cpu_baseline=True):
    """64 independent water boxes of uneven size (3,000-48,000 atoms), one
    batched call (one CUDA graph) per step.  With N ranks the same 64 boxes
    are split by cost (atoms) with LPT, each rank evaluating its share
    (strong scaling, no data-path collective).  Returns rank 0's line."""
    import torch
    steps = steps or args.steps
    e2e_steps = e2e_steps or args.e2e_steps
    all_boxes = synth.replica_boxes(64)
    mine = lpt_partition([b.n for b in all_boxes], world)[rank]
    boxes = [all_boxes[i] for i in mine]
    if not boxes:
        raise SystemExit("more ranks than boxes")
    cat = lambda f: np.ascontiguousarray(np.concatenate([f(b) for b in boxes]), dtype=np.float32)
    hx, hq, hmu, hth = cat(lambda b: b.x), cat(lambda b: b.q), cat(lambda b: b.mu), cat(lambda b: b.theta)
    x, q, mu, th = (torch.from_numpy(a).to(dev) for a in (hx, hq, hmu, hth))
    ntot = int(x.shape[0])
    bt = api.AnkhBatch([b.box for b in boxes], [b.n for b in boxes], Lu=args.Lu, mixed=not args.plain)
    out = {"dEdx": torch.empty((ntot, 3), device=dev), "dEdq": torch.empty(ntot, device=dev),
           "dEdmu": torch.empty((ntot, 3), device=dev), "dEdtheta": torch.empty((ntot, 6), device=dev),
           "torque": torch.empty((ntot, 3), device=dev)}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    api.ankh_batch_set_timing(bt.h, True)      # events around the batched near field, in the graph
    for _ in range(max(args.warmup, 3)):
        bt.energy_forces(x, q, mu, th, out=out)
    clocks = ClockSampler(dev.index)
    preroll(clocks, lambda: bt.energy_forces(x, q, mu, th, out=out))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark("timed_start")
    tot = 0.0
    near_s = 0.0
    for k in range(steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.energy_forces(x, q, mu, th, out=out)
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1) / 1e3
        near_s += api.ankh_batch_near_ms(bt.h) / 1e3
    torch.cuda.synchronize()
    clocks.mark("timed_end")
    clk = clocks.stop()
    if dist:
        dist.barrier()
    tot = max_over_ranks(tot, dist, dev)
    value = 64 * steps / tot
    ntot_all = sum(b.n for b in all_boxes)

    # end to end: the host arrays copied in (pinned), the batch call, the
    # gradients copied back, every step
    pin = lambda a: torch.from_numpy(a).pin_memory()
    px, pq, pmu, pth = pin(hx), pin(hq), pin(hmu), pin(hth)
    ho = {k: torch.empty(tuple(v.shape), dtype=torch.float32).pin_memory() for k, v in out.items()}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for d_, h_ in ((x, px), (q, pq), (mu, pmu), (th, pth)):
            d_.copy_(h_, non_blocking=True)
        bt.energy_forces(x, q, mu, th, out=out)
        for k_, v_ in out.items():
            ho[k_].copy_(v_, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)

    # the batched near field over all boxes (its duration from the events
    # the graph records around it) against the measured FP32 peak
    fp32_meas, _ = api.ankh_measure_fp32_peak(stream)
    pairs = 0
    for i in range(len(boxes)):
        hb = api.ankh_batch_box(bt.h, i)
        nb_ = int(api.ankh_get_info(hb)["n_cells"])
        pairs += unordered_near_pairs(api.ankh_debug_copy(hb, api.BUF_START).cpu().numpy(), nb_)
    near_rate = pairs * NEAR_FLOPS_PER_PAIR / 1e12 / (near_s / steps)
    roof = {"kernel": "near (one launch over all 64 boxes)", "bound": "alu", "achieved": near_rate,
            "peak": fp32_meas, "unit": "TFLOP/s", "frac": near_rate / fp32_meas, "traffic": None,
            "near_ms": near_s / steps * 1e3, "near_pairs_unordered": pairs,
            "peak_source": "FP32 FMA throughput measured on this GPU (ankh_measure_fp32_peak)"}

    cpu = None
    if rank == 0 and world == 1 and cpu_baseline:
        # the FP64 Ewald oracle on a bounded sample of four of the boxes
        # (smallest, two middle, largest), a power law in N fitted to their
        # extrapolated full-evaluation times, summed over all 64 boxes
        order = sorted(range(len(all_boxes)), key=lambda i: all_boxes[i].n)
        pick = [order[0], order[len(order) // 3], order[2 * len(order) // 3], order[-1]]
        ts, ns = [], []
        for i in pick:
            r = oracle_sample(all_boxes[i], rows=150, kstride=400)
            ts.append(r["seconds_full_eval"])
            ns.append(all_boxes[i].n)
        k_, c_ = np.polyfit(np.log(ns), np.log(ts), 1)
        t_all = float(sum(math.exp(c_) * b.n ** k_ for b in all_boxes))
        cpu = {"value": 64.0 / t_all, "unit": "box-evals/s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": (f"FP64 Ewald oracle, energy + gradient: real-space rows of 150 and 300 atoms and "
                          f"every 400-th / 200-th k-vector of boxes of {ns} atoms, each extrapolated to a full "
                          f"evaluation, t = {math.exp(c_):.3g} N^{k_:.3f} s fitted and summed over the 64 boxes")}
    line = {
        "metric": METRIC, "value": value, "unit": "box-evals/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": tot / steps * 1e3, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "replicas64_water_3000_48000_qmuTheta_energy_forces", "n_boxes": 64,
                   "n_atoms_total": ntot_all,
                   "Lu": args.Lu or "per box, with its leaf count, from the accuracy table",
                   "l2": "flushed: 256 MiB write between timed steps",
                   "execution": "one CUDA graph per rank, one branch per box",
                   "parallelism": f"boxes split over {world} GPU(s) by LPT on atom counts"},
        "matoms_per_s": value / 64 * ntot_all / 1e6, "clocks": clk, "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": 64 * e2e_steps / t_e2e, "unit": "box-evals/s",
                "h2d_bytes_per_step": 4 * ntot * (3 + 1 + 3 + 6),
                "d2h_bytes_per_step": 4 * ntot * (3 + 1 + 3 + 6 + 3)},
        "gpu_launches": api.ankh_batch_launch_count(bt.h) * steps}
    bt.close()
    return line


def run_replicas(args, rank, world, dev, api, synth, dist=None):
    line = replicas_measure(args, rank, world, dev, api, synth, dist, cpu_baseline=not args.no_cpu_baseline)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_fmm(args, rank, world, dev, api, synth, dist, cfg):
    """ANKH-FMM energy (Alg. 3, flag ANKH_FMM): one step = one energy
    evaluation (sort, P2M, M2M, mutual M2L on the tensor cores, root term,
    near field, self term) on inputs resident in HBM, L2 flushed between
    steps.  The tree is 2^E leaves per axis (default: the leaf edge nearest
    4 A, n = 64 for the 1M-atom box) with L = --Lu Chebyshev nodes per axis."""
    import torch
    box = synth.config_box(cfg) if rank == 0 else synth.water_box(
        synth.CONFIGS[cfg]["n_waters"], synth.SEED_BASE + cfg + 1000 * rank, multipoles=True,
        name=synth.CONFIGS[cfg]["name"])
    N = box.n
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    x, q, mu, th = f32(box.x), f32(box.q), f32(box.mu), f32(box.theta)
    L = args.Lu or 5
    n_cells, tune = args.n_cells, None
    if n_cells == 0:
        # tree depth by measurement (outside the timed region): the two powers
        # of two around a 4 A leaf edge, best of three energy evaluations each
        tune = {}
        e0 = max(2, min(7, int(math.floor(math.log2(box.box / 4.0)))))
        for nc in sorted({1 << e0, 1 << min(7, e0 + 1)}):
            mt = api.Ankh(box.box, N, n_cells=nc, Lu=L, Lc=L, fmm=True)
            best = float("inf")
            for _ in range(4):
                torch.cuda.synchronize()
                a = time.perf_counter()
                api.ankh_energy(mt.h, x, q, mu, th)
                best = min(best, time.perf_counter() - a)
            tune[str(nc)] = round(best * 1e3, 4)
            mt.close()
        n_cells = int(min(tune, key=tune.get))
    t_pre0 = time.perf_counter()
    model = api.Ankh(box.box, N, n_cells=n_cells, Lu=L, Lc=L, fmm=True)
    t_pre = time.perf_counter() - t_pre0
    info = model.info
    n = info["n_cells"]
    depth = int(round(math.log2(n)))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    api.ankh_set_timing(model.h, True)
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        api.ankh_energy(model.h, x, q, mu, th, stream=stream)
    clocks = ClockSampler(dev.index)
    preroll(clocks, lambda: api.ankh_energy(model.h, x, q, mu, th, stream=stream))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark("timed_start")
    names = {"sort": "sort", "self": "self", "p2m": "p2m", "merge": "m2m", "spectral": "root", "corr": "m2l",
             "near": "near", "reduce": "reduce"}
    stage_sum = {v: 0.0 for v in names.values()}
    t_dev = 0.0
    E = None
    for k in range(args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        E = api.ankh_energy(model.h, x, q, mu, th, stream=stream)
        e1.record(stream)
        e1.synchronize()
        t_dev += e0.elapsed_time(e1) / 1e3
        for s_, v in api.ankh_stage_times(model.h).items():
            if s_ in names:
                stage_sum[names[s_]] += v
    torch.cuda.synchronize()
    clocks.mark("timed_end")
    clk = clocks.stop()
    if dist:
        dist.barrier()
    t_max = max_over_ranks(t_dev, dist, dev)
    value = world * args.steps / t_max
    stage_ms = {k: v / args.steps for k, v in stage_sum.items()}

    # end to end: pinned host inputs copied in, energy read back, every step
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
    hx, hq, hmu, hth = pin(box.x), pin(box.q), pin(box.mu), pin(box.theta)
    api.ankh_set_timing(model.h, False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        x.copy_(hx, non_blocking=True)
        q.copy_(hq, non_blocking=True)
        mu.copy_(hmu, non_blocking=True)
        th.copy_(hth, non_blocking=True)
        api.ankh_energy(model.h, x, q, mu, th, stream=stream)
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)

    acc = None
    gpath = os.path.join(ROOT, "tests", "golden", f"ewald_{box.name}.json")
    if rank == 0 and os.path.exists(gpath):
        gd = json.load(open(gpath))
        acc = {"rel_energy_error": abs(E - gd["E"]) / abs(gd["E"]), "reference": "FP64 Ewald oracle (tests/golden)"}

    # M2L roofline: per level e, 8^e targets x 189 list members, each unordered
    # pair once (mutual), one P x P matrix-vector product + dot = 2 P^2 flop
    peaks, peak_kind = measured_peaks()
    P = L ** 3
    m2l_flop = sum(8 ** e for e in range(1, depth + 1)) * 189 / 2 * 2 * P * P
    achieved = m2l_flop / 1e12 / (stage_ms["m2l"] / 1e3)
    roof = {"kernel": "m2l", "bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"],
            "unit": "TFLOP/s", "frac": achieved / peaks["bf16_tflops"],
            "traffic": DRAM_TRAFFIC.get(("m2l", box.name, n, L)),
            "peak_source": f"{peak_kind} MEASURED_PEAKS bf16 (= fp16 rate; the split executes 3 products)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's ANKH-FMM on the 24,000-atom box (62.1 A) at the same
        # order and a leaf edge of 3.9 A, scaled per atom to this workload
        from oracle import ankh_fmm as fm
        sb = synth.config_box(2)
        a = time.perf_counter()
        fm.ankh_fmm_energy(sb.x, sb.q, sb.mu, sb.theta, sb.box, 4, L)
        ts = time.perf_counter() - a
        cpu = {"value": 1.0 / (ts * N / sb.n), "unit": "evals/s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"FP64 ANKH-FMM oracle, energy of the {sb.n}-atom water box at depth 4, L={L} "
                         f"({ts:.1f} s), scaled by atoms ({N}/{sb.n})"}

    if rank == 0:
        print(json.dumps({
            "metric": "ANKH-FMM energy evals/s", "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": box.name + "_fmm_energy", "n_atoms": N, "box_A": round(box.box, 4),
                       "n_cells": n, "depth": depth, "L": L, "xi": 0.01,
                       "leaf_count": "autotuned" if args.n_cells == 0 else "fixed", "autotune_ms": tune,
                       "precision": "mixed_2xfp16_m2l", "l2": "flushed: 256 MiB write between timed steps",
                       "parallelism": f"replicas{world}"},
            "matoms_per_s": value * N / 1e6, "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "precompute_s": t_pre, "accuracy": acc, "clocks": clk, "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": world * args.e2e_steps / t_e2e, "unit": "evals/s",
                    "h2d_bytes_per_step": 4 * N * (3 + 1 + 3 + 6), "d2h_bytes_per_step": 9 * 8},
            "gpu_launches": api.ankh_launch_count(model.h, False) * args.steps}), flush=True)
    model.close()


def run_induce(args, rank, world, dev, api, synth, dist, cfg):
    """Induced dipoles of the workload (point polarizability 0.005 A^3 per
    atom: positive definite down to 0.22 A separations): one step = one full
    conjugate-gradient solve to |r| <= 1e-6 |F|, each iteration one ANKH
    field evaluation.  Reported: solves/s, iterations, ms per iteration."""
    import torch
    box = synth.config_box(cfg)
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    x, q, mu, th = f32(box.x), f32(box.q), f32(box.mu), f32(box.theta)
    alpha = torch.full((box.n,), 0.005, device=dev)
    n_cells, Lu = args.n_cells, args.Lu
    if n_cells == 0:
        from paper_2212_08284_gb300 import autotune
        (n_cells, Lu), _ = autotune.autotune(box.box, x, q, mu, th, Lu=args.Lu, mixed=not args.plain,
                                             nonperiodic=args.nonperiodic)
    model = api.Ankh(box.box, box.n, n_cells=n_cells, Lu=Lu, Lc=Lu, mixed=not args.plain,
                     nonperiodic=args.nonperiodic)
    out = torch.empty((box.n, 3), device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        E_pol, it = api.ankh_induce(model.h, x, q, mu, th, alpha, out, tol=1e-6, stream=stream)
    clocks = ClockSampler(dev.index)
    preroll(clocks, lambda: api.ankh_induce(model.h, x, q, mu, th, alpha, out, tol=1e-6, stream=stream))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark("timed_start")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    its = []
    for _ in range(args.steps):
        E_pol, it = api.ankh_induce(model.h, x, q, mu, th, alpha, out, tol=1e-6, stream=stream)
        its.append(it)
    e1.record(stream)
    e1.synchronize()
    clocks.mark("timed_end")
    clk = clocks.stop()
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
    value = world * args.steps / t
    evals = args.steps * (statistics.mean(its) + 2)
    if rank == 0:
        print(json.dumps({
            "metric": "induced-dipole solves/s (CG to 1e-6 on the ANKH field)", "value": value,
            "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": box.name + ("_nonperiodic" if args.nonperiodic else "") + "_induce",
                       "n_atoms": box.n, "n_cells": n_cells, "Lu": Lu, "alpha_A3": 0.005, "tol": 1e-6,
                       "parallelism": f"replicas{world}"},
            "iterations": statistics.mean(its), "ms_per_field_evaluation": t * 1e3 / evals,
            "E_pol": E_pol, "clocks": clk, "roofline": None, "cpu_baseline": None, "e2e": None,
            # per solve: one evaluation's kernels per field evaluation (iterations + 2
            # of them), 3 vector kernels per iteration, 3 outside the loop
            "gpu_launches": int(round(args.steps * (api.ankh_launch_count(model.h, True)
                                                    * (statistics.mean(its) + 2) + 3 * statistics.mean(its) + 3)))}),
              flush=True)
    model.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="water_1008000", choices=sorted(WORKLOADS))
    ap.add_argument("--plain", action="store_true", help="plain FP32 adjacent-leaf correction")
    ap.add_argument("--induce", action="store_true",
                    help="time induced-dipole solves (conjugate gradients on the ANKH field) instead")
    ap.add_argument("--fmm", action="store_true",
                    help="time ANKH-FMM energy evaluations (Alg. 3) instead")
    ap.add_argument("--nonperiodic", action="store_true",
                    help="no periodic images (bare kernel, zero-padded far field, Sec. 5.2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain-FP32 leg and the other workloads after the main line's timing")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--n-cells", type=int, default=0, help="leaves per axis (0 = autotuned)")
    ap.add_argument("--Lu", type=int, default=0,
                    help="equispaced interpolation order (0: chosen with the leaf count from the accuracy table)")
    args = ap.parse_args()

    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_2212_08284_gb300 import api, build, synth

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    api.load_library()

    cfg = WORKLOADS[args.workload]
    if cfg == 5:
        run_replicas(args, rank, world, dev, api, synth, dist)
        return
    if args.induce:
        run_induce(args, rank, world, dev, api, synth, dist, cfg)
        return
    if args.fmm:
        run_fmm(args, rank, world, dev, api, synth, dist, cfg)
        return
    box = synth.config_box(cfg) if rank == 0 else synth.water_box(
        synth.CONFIGS[cfg]["n_waters"], synth.SEED_BASE + cfg + 1000 * rank, multipoles=True,
        name=synth.CONFIGS[cfg]["name"])
    N = box.n
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    x, q, mu, th = f32(box.x), f32(box.q), f32(box.mu), f32(box.theta)
    tune = None
    n_cells, Lu = args.n_cells, args.Lu
    if n_cells == 0:
        # leaf count and order picked by measurement (outside the timed region)
        # among the pairs that the library's accuracy table allows for the box
        from paper_2212_08284_gb300 import autotune
        (n_cells, Lu), tab = autotune.autotune(box.box, x, q, mu, th, Lu=args.Lu, mixed=not args.plain,
                                               nonperiodic=args.nonperiodic)
        tune = {k: round(v, 4) for k, v in tab.items()}
    t_pre0 = time.perf_counter()
    model = api.Ankh(box.box, N, n_cells=n_cells, Lu=Lu, Lc=Lu, mixed=not args.plain,
                     nonperiodic=args.nonperiodic)
    t_pre = time.perf_counter() - t_pre0
    info = model.info
    out = {"dEdx": torch.empty((N, 3), device=dev), "dEdq": torch.empty(N, device=dev),
           "dEdmu": torch.empty((N, 3), device=dev), "dEdtheta": torch.empty((N, 6), device=dev),
           "torque": torch.empty((N, 3), device=dev)}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream()

    def step():
        api.ankh_energy_forces(model.h, x, q, mu, th, sync=False, stream=stream, **out)

    api.ankh_set_timing(model.h, True)
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    E = api.ankh_energy_forces(model.h, x, q, mu, th, stream=stream, **out)

    # FP32 FMA throughput of this GPU (the near field's roofline denominator)
    fp32_meas, _ = api.ankh_measure_fp32_peak(stream)

    def flushed_step():
        flush.fill_(1.0)
        step()

    clocks = ClockSampler(dev.index)
    preroll(clocks, flushed_step)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark("timed_start")
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage_sum = {k: 0.0 for k in api.STAGES}
    for k in range(args.steps):
        flush.fill_(float(k))
        ev0[k].record(stream)
        step()
        ev1[k].record(stream)
        st = api.ankh_stage_times(model.h)     # waits for this step's events
        for s_, v in st.items():
            stage_sum[s_] += v
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks.mark("timed_end")
    clk = clocks.stop()
    t_dev = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)) / 1e3   # seconds, device time
    t_max = max_over_ranks(t_dev, dist, dev)
    value = world * args.steps / t_max
    ms_step = t_max / args.steps * 1e3
    stage_ms = {k: v / args.steps for k, v in stage_sum.items()}

    # end to end through the host-buffer entry point (pinned host memory)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
    hx, hq, hmu, hth = pin(box.x), pin(box.q), pin(box.mu), pin(box.theta)
    ho = {k: torch.empty(tuple(v.shape), dtype=torch.float32).pin_memory() for k, v in out.items()}
    api.ankh_set_timing(model.h, False)
    api.ankh_energy_forces_host(model.h, hx, hq, hmu, hth, stream=stream, **ho)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        api.ankh_energy_forces_host(model.h, hx, hq, hmu, hth, stream=stream, **ho)
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    h2d = 4 * N * (3 + 1 + 3 + 6)
    d2h = 4 * N * (3 + 1 + 3 + 6 + 3) + 8

    # accuracy against the FP64 Ewald reference of this workload (rank 0 box)
    acc = None
    gpath = os.path.join(ROOT, "tests", "golden", f"ewald_{box.name}.json")
    if rank == 0 and args.nonperiodic:
        # forces on 64 sampled atoms against the FP64 direct sum (all other atoms)
        from oracle import ewald as ew
        idx = np.sort(np.random.default_rng(9).choice(N, size=min(64, N), replace=False))
        ref = ew.direct_nonperiodic_rows(box.x.astype(np.float64), ew.pack_multipoles(box.q, box.mu, box.theta),
                                         idx)
        gx = out["dEdx"].cpu().numpy().astype(np.float64)[idx]
        acc = {"rel_energy_error": None,
               "rel_rms_force_error_sample": float(np.sqrt(np.mean((gx - ref[:, :3]) ** 2))
                                                   / np.sqrt(np.mean(ref[:, :3] ** 2))),
               "reference": "FP64 non-periodic direct sum, 64 sampled atoms (the O(N^2) energy is "
                            "checked at 648 atoms in tests/test_gpu_nonperiodic.py)"}
    elif rank == 0 and os.path.exists(gpath):
        gd = json.load(open(gpath))
        idx = np.array(gd["sample_idx"])
        ref = np.array(gd["sample_grad"])
        gx = out["dEdx"].cpu().numpy().astype(np.float64)[idx]
        acc = {"rel_energy_error": abs(E - gd["E"]) / abs(gd["E"]),
               "rel_rms_force_error_sample": float(np.sqrt(np.mean((gx - ref[:, :3]) ** 2))
                                                   / gd["rms_all"]["dEdx"]),
               "reference": "FP64 Ewald oracle (tests/golden)"}

    wname = box.name + ("_nonperiodic" if args.nonperiodic else "")
    # roofline of the dominant kernel
    peaks, peak_kind = measured_peaks()
    start = api.ankh_debug_copy(model.h, api.BUF_START).cpu().numpy()
    n = info["n_cells"]
    pairs = unordered_near_pairs(start, n, args.nonperiodic)
    dom = max(stage_ms, key=stage_ms.get)
    sm_mhz = clk["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_nominal = n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12   # TF/s at the sampled clock
    fp32_peak = fp32_meas
    P = info["Lu"] ** 3
    ncell = n ** 3
    M_grid = info["nf"] ** 3
    # Correction: psi_t = sum_d C_d M_(t+d) over all 27 offsets d (the forces
    # need psi at every leaf: the 13 mutual offsets give the energy alone, and
    # C_(-d) = C_d^T still has to be applied to M_t for psi_(t+d)), one
    # P x P block product per (leaf, offset), three products for the 2xFP16
    # split; unpadded P nodes, n^3 leaves.
    corr_flop = 2 * 27 * P * P * ncell * (3 if not args.plain else 1)
    models = {
        "near": ("alu", pairs * NEAR_FLOPS_PER_PAIR / 1e12, fp32_peak, "TFLOP/s"),
        "corr": ("tensor" if not args.plain else "alu", corr_flop / 1e12,
                 peaks["bf16_tflops"] if not args.plain else fp32_peak, "TFLOP/s"),
        # P2M: read 52 B per atom (position, q, mu, Theta), write 4 B per leaf node
        "p2m": ("hbm", (52 * N + 4 * ncell * P) / 1e9, peaks["hbm_gbs"], "GB/s"),
        # L2P (node potentials + gradient assembly): read the grid potential
        # (4 B per grid point), the correction potential (4 B per leaf node)
        # and 52 B per atom; write 64 B per atom (dE/dx, dE/dq, dE/dmu,
        # dE/dTheta, torque)
        "l2p": ("hbm", (4 * M_grid + 4 * ncell * P + 52 * N + 64 * N) / 1e9, peaks["hbm_gbs"], "GB/s"),
    }

    def roofline(k):
        bound, work, peak, unit = models[k]
        achieved = work / (stage_ms[k] / 1e3)
        r = {"kernel": k, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
             "frac": achieved / peak, "traffic": DRAM_TRAFFIC.get((k, wname, n, info["Lu"])),
             "peak_source": ("FP32 FMA throughput measured on this GPU (ankh_measure_fp32_peak); nominal "
                             f"{n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz sampled = "
                             f"{fp32_nominal:.1f} TFLOP/s" if bound == "alu" else
                             f"{peak_kind} MEASURED_PEAKS")}
        if k == "near":
            r["executed_tflops"] = 2 * pairs * NEAR_FLOPS_EXECUTED_PER_ORDERED_PAIR / 1e12 / (stage_ms[k] / 1e3)
        return r

    roof = roofline(dom) if dom in models else None
    roof_all = [roofline(k) for k in models if k in stage_ms and stage_ms[k] > 0]

    # the plain FP32 form of the same evaluation on the same box and leaf count
    plain_leg = None
    legs = None
    if rank == 0 and world == 1 and not args.no_extras and not args.plain and not args.nonperiodic:
        mp_ = api.Ankh(box.box, N, n_cells=n_cells, Lu=info["Lu"], Lc=info["Lu"], mixed=False)
        fn = lambda: api.ankh_energy_forces(mp_.h, x, q, mu, th, sync=False, stream=stream, **out)
        tp = time_device(fn, max(10, min(args.steps, 30)), flush, stream)
        Ep = api.ankh_energy_forces(mp_.h, x, q, mu, th, stream=stream, **out)
        mp_.close()
        plain_leg = {"precision": "plain_fp32 (FP32 CUDA-core correction)", "n_cells": n, "Lu": info["Lu"],
                     "evals_per_s": 1.0 / tp, "ms_per_eval": tp * 1e3,
                     "accuracy": golden_errors(box, Ep, out["dEdx"]),
                     "mixed_over_plain": (1.0 / ms_step * 1e3) / (1.0 / tp)}
        legs = config_legs(args, dev, api, synth, flush, stream, max(10, min(args.steps, 30)))
        legs.append(replicas_measure(args, 0, 1, dev, api, synth, None, steps=max(5, min(args.steps, 10)),
                                     e2e_steps=3, cpu_baseline=not args.no_cpu_baseline))

    cpu = None
    cpu_ankh = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_sample_nonperiodic(box) if args.nonperiodic else oracle_sample(box)
        cpu = {"value": 1.0 / r["seconds_full_eval"], "unit": UNIT, "cores": os.cpu_count() or 1,
               "kind": "oracle", "sample": r["sample"]}
        if not args.nonperiodic:
            cpu_ankh = oracle_ankh_sample(box, info["Lu"])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wname + "_energy_forces",
                       "n_atoms": N, "box_A": round(box.box, 4),
                       "n_cells": n, "Lu": info["Lu"], "Lc": info["Lc"], "nf": info["nf"],
                       "xi": 0.0 if args.nonperiodic else 0.01,
                       "precision": "plain_fp32" if args.plain else "mixed_2xfp16_correction",
                       "l2": "flushed: 256 MiB write between timed steps", "parallelism": f"replicas{world}",
                       "leaf_count": ("autotuned among the (n, L_u) the accuracy table allows" if args.n_cells == 0
                                      else "fixed"), "autotune_ms": tune},
            "matoms_per_s": value * N / 1e6,
            "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "near_pairs_unordered": pairs,
            "precompute_s": t_pre,
            "accuracy": acc,
            "clocks": clk,
            "roofline": roof,
            "rooflines": roof_all,
            "cpu_baseline": cpu,
            "cpu_baseline_ankh": cpu_ankh,
            "e2e": {"value": world * args.e2e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "plain_fp32": plain_leg,
            "other_configs": legs,
            "gpu_launches": api.ankh_launch_count(model.h, True) * args.steps,
        }
        print(json.dumps(line), flush=True)
    model.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
