"""The library's accuracy table (ankh_accuracy_rule, the defaults of
ankh_create) against the method-error map of the oracle
(tests/golden/error_map.json, written by make_error_map.py from the oracle
only).

Rule: for each calibration box (with multipoles: 24,000, 96,000 and
1,008,000 atoms; charges only: 648 atoms) and order L_u <= 6, the allowed
leaf edges start at the end of the run, from the largest measured edge
down, of consecutive measured leaf counts whose FP64 ANKH-FFT is within
5e-6 (relative energy) and 3e-5 (relative RMS force; energy only for the
charges-only box) of FP64 Ewald -- a run of at least three -- rounded
outwards to 1e-4 A.  No GPU needed (host-only entry point).
"""
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
E_BAR, F_BAR = 5e-6, 3e-5
CLASSES = {False: (1008000, 96000, 24000), True: (648,)}    # charges only -> class sizes


@pytest.fixture(scope="module")
def emap():
    return json.load(open(os.path.join(HERE, "golden", "error_map.json")))["entries"]


@pytest.fixture(scope="module")
def api():
    from paper_2212_08284_gb300 import api as A, build
    build.build()
    A.load_library()
    return A


def derived(entries):
    rows = {}
    for qonly, classes in CLASSES.items():
        for N in classes:
            for Lu in range(2, 7):
                v = sorted((e for e in entries if e["n_atoms"] == N and e["Lu"] == Lu
                            and (e["rel_rms_force_error"] is None) == qonly), key=lambda e: -e["h_A"])
                run, hmin = 0, None
                for e in v:
                    if e["rel_energy_error"] > E_BAR or (not qonly and e["rel_rms_force_error"] > F_BAR):
                        break
                    run += 1
                    if run >= 3:
                        hmin = e["h_A"]
                if hmin is not None:
                    rows[(N, qonly, Lu)] = (math.floor(hmin * 1e4) / 1e4, math.ceil(v[0]["h_A"] * 1e4) / 1e4)
    return rows


def test_library_table_is_the_map_rule(api, emap):
    want = derived(emap)
    assert want, "empty map"
    for qonly, classes in CLASSES.items():
        for N in classes:
            for Lu in range(2, 9):
                got = api.ankh_accuracy_rule(N, Lu, 0 if qonly else 2)
                if (N, qonly, Lu) in want:
                    assert got == pytest.approx(want[(N, qonly, Lu)], abs=1e-9), (N, Lu)
                else:
                    assert got is None, (N, Lu)


def test_every_allowed_map_point_meets_the_bars(api, emap):
    for e in emap:
        qonly = e["rel_rms_force_error"] is None
        if e["n_atoms"] not in CLASSES[qonly]:
            continue
        r = api.ankh_accuracy_rule(e["n_atoms"], e["Lu"], 0 if qonly else 2)
        if r and r[0] <= e["h_A"] <= r[1]:
            assert e["rel_energy_error"] <= E_BAR, e
            assert qonly or e["rel_rms_force_error"] <= F_BAR, e


def test_classes_by_atom_count(api):
    # a box uses the class of its kind with the largest atom count not above its own
    for N, cls in ((24000, 24000), (95999, 24000), (96000, 96000), (1007999, 96000), (1008000, 1008000),
                   (10 ** 8, 1008000)):
        for Lu in range(2, 9):
            assert api.ankh_accuracy_rule(N, Lu) == api.ankh_accuracy_rule(cls, Lu)
    for Lu in range(2, 9):
        assert api.ankh_accuracy_rule(23999, Lu) is None           # below the smallest class: not calibrated
        assert api.ankh_accuracy_rule(10 ** 6, Lu, 0) == api.ankh_accuracy_rule(648, Lu, 0)
    assert all(api.ankh_accuracy_rule(N, Lu, m) is None for N in (648, 10 ** 7) for Lu in (7, 8) for m in (0, 2))


def test_every_workload_has_accurate_candidates(api):
    from paper_2212_08284_gb300 import autotune, synth
    for c in (1, 2, 3, 4):
        b = synth.config_box(c)
        mo = 0 if c == 1 else 2
        cand = autotune.candidates(b.box, b.n, max_order=mo)
        assert cand, b.name
        for n, Lu in cand:
            lo, hi = api.ankh_accuracy_rule(b.n, Lu, mo)
            assert lo <= b.box / n <= hi and autotune.grid_ok(n, Lu)


def test_map_entry_reproduces_from_the_oracle(emap):
    """One map point recomputed (the 3,000-atom box, n = 7, L_u = 7): the file
    holds what the oracle gives."""
    from oracle import ankh_ref as ar
    from paper_2212_08284_gb300 import synth
    b = synth.small_box(1000, 31, box=31.1)
    gd = json.load(open(os.path.join(HERE, "golden", "ewald_water_3000.json")))
    e = next(x for x in emap if x["n_atoms"] == 3000 and x["Lu"] == 7 and x["n"] == 7)
    o = ar.ankh_energy(b.x, b.q, b.mu, b.theta, ar.Params(b.box, 7, 7, 7), grad=False)
    assert abs(o["E"] - gd["E"]) / abs(gd["E"]) == pytest.approx(e["rel_energy_error"], rel=1e-6)
