"""ANKH-FMM (Sec. 3, Alg. 3, flag ANKH_FMM) through the C ABI against the
FP64 oracle (oracle/ankh_fmm.py) at matched (depth, L), term by term.

Bars.  The near field and the self term are the FP32 kernels of ANKH-FFT
(total within 2e-6, as in test_gpu_parity.py).  The far terms carry the
fp16 hi + lo split of the M2L (~2^-22 per product) and FP32 expansions: their
absolute error scales with the largest M entries, which the (2/h)^p factors
of the quadrupoles make large while the far energy itself is small, so with
multipoles they are held to 1e-6 |E| (the bar of the tensor-core correction
of ANKH-FFT); with charges only, the M2L term is held to 1e-5 of itself.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import ankh_fmm as fm           # noqa: E402
from paper_2212_08284_gb300 import synth    # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def api(gpu):
    from paper_2212_08284_gb300 import api as A, build
    build.build()
    A.load_library()
    return A


def to_dev(b):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    mu = t(b.mu) if b.mu is not None else None
    th = t(b.theta) if b.theta is not None else None
    return t(b.x), t(b.q), mu, th


CASES = [  # (n_waters, seed, box, multipoles, depth, L): L = 3..6 covers 1-4 K chunks and 1-2 row slices
    (600, 7, 18.0, True, 3, 5),
    (600, 7, 18.0, False, 3, 5),
    (600, 7, 18.0, True, 2, 6),
    (216, 11, 18.64, True, 2, 4),
    (216, 11, 18.64, True, 3, 3),
]


@pytest.mark.parametrize("case", CASES)
def test_terms_match_the_fp64_oracle(api, case):
    nw, seed, box, mpl, depth, L = case
    b = synth.water_box(nw, seed, box=box, multipoles=mpl)
    o = fm.ankh_fmm_energy(b.x, b.q, b.mu, b.theta, b.box, depth, L)
    m = api.Ankh(b.box, b.n, n_cells=2 ** depth, Lu=L, Lc=L, fmm=True)
    E = m.energy(*to_dev(b))
    t = m.terms()
    assert E == pytest.approx(o["E"], rel=2e-6)
    assert t["near"] == pytest.approx(o["N_real"], rel=2e-6)
    assert t["self"] == pytest.approx(o["E_self"], rel=1e-6)
    assert t["far_k0"] == 0.0
    # the constant of the lattice sum (in the oracle's F_per) cancels E_neut
    assert abs(t["far"] - (o["F_per"] + o["E_neut"])) <= 1e-6 * abs(o["E"])
    assert abs(t["correction"] - o["F_real"]) <= 1e-6 * abs(o["E"])
    if not mpl:
        assert t["correction"] == pytest.approx(o["F_real"], rel=1e-5)


@pytest.mark.parametrize("depth,L", [(2, 7), (3, 2)])
def test_extreme_orders(api, depth, L):
    """L = 7: 343 nodes in three 128-row slices (the last one partial) and six
    K chunks; L = 2: the smallest order (8 nodes padded to 64)."""
    b = synth.water_box(216, 11, box=18.64, multipoles=True)
    o = fm.ankh_fmm_energy(b.x, b.q, b.mu, b.theta, b.box, depth, L)
    m = api.Ankh(b.box, b.n, n_cells=2 ** depth, Lu=L, Lc=L, fmm=True)
    E = m.energy(*to_dev(b))
    t = m.terms()
    assert E == pytest.approx(o["E"], rel=2e-6)
    assert abs(t["correction"] - o["F_real"]) <= 1e-6 * abs(o["E"])
    assert abs(t["far"] - (o["F_per"] + o["E_neut"])) <= 1e-6 * abs(o["E"])


def test_single_charged_atom(api):
    """One atom with a charge and a dipole (not neutral): only images
    interact, through the M2L of the direct images and the root term; the
    Q^2 constant of the lattice sum and the neutralising term are dropped
    together on the GPU and kept (cancelling) in the oracle."""
    import torch
    x = np.array([[1.3, -2.2, 0.7]])
    q, mu = np.array([0.8]), np.array([[0.1, -0.2, 0.3]])
    o = fm.ankh_fmm_energy(x, q, mu, np.zeros((1, 6)), 12.0, 2, 5)
    m = api.Ankh(12.0, 1, n_cells=4, Lu=5, Lc=5, fmm=True, max_order=1)
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    E = m.energy(t32(x), t32(q), t32(mu), None)
    t = m.terms()
    assert t["near"] == 0.0
    assert t["correction"] == pytest.approx(o["F_real"], rel=2e-6)
    assert t["far"] == pytest.approx(o["F_per"] + o["E_neut"], rel=2e-6)
    assert E == pytest.approx(o["E"], abs=2e-6 * (abs(o["F_real"]) + abs(o["F_per"] + o["E_neut"])))


def test_without_the_reciprocal_part(api):
    """Paper-literal screening (E_rec(xi) neglected): the root operator then
    carries only the band-limited difference of the second split."""
    b = synth.water_box(216, 11, box=18.64, multipoles=True)
    o = fm.ankh_fmm_energy(b.x, b.q, b.mu, b.theta, b.box, 3, 5, include_rec=False)
    m = api.Ankh(b.box, b.n, n_cells=8, Lu=5, Lc=5, fmm=True, include_rec=False)
    E = m.energy(*to_dev(b))
    assert E == pytest.approx(o["E"], rel=2e-6)
    assert abs(m.terms()["far"] - (o["F_per"] + o["E_neut"])) <= 1e-6 * abs(o["E"])


def test_24000_atoms_depth4_matches_oracle_and_ewald(api):
    """The 24,000-atom water box (62.1 A) at depth 4 (16 leaves per axis, the
    level-4 z-rows of 8 cells padded to 16 columns): against the oracle at the
    same (depth, L), and against Ewald within the oracle's own error plus 2e-6."""
    b = synth.config_box(2)
    L = 4
    o = fm.ankh_fmm_energy(b.x, b.q, b.mu, b.theta, b.box, 4, L)
    m = api.Ankh(b.box, b.n, n_cells=16, Lu=L, Lc=L, fmm=True)
    E = m.energy(*to_dev(b))
    assert E == pytest.approx(o["E"], rel=2e-6)
    ref = json.load(open(os.path.join(GOLDEN, "ewald_water_24000_qmuTheta.json")))["E"]
    assert abs(E - ref) <= abs(o["E"] - ref) + 2e-6 * abs(ref)


def test_deepest_tree_charges_against_ewald(api):
    """Depth 7 (128 leaves per axis; the level-7 copies are 3-D boxes of two
    z-row blocks of 64 rows) on the 600-water box with charges only, against
    Ewald.  With charges alone the method's error does not grow with the
    depth (measured 1.8e-5 to 2.8e-5 at depths 2-7); with multipoles it does,
    once the leaves are much smaller than the molecules (the FP64 oracle
    shows the same), so multipoles are checked at depths 2-4 above."""
    from oracle import ewald as ew
    b = synth.water_box(600, 7, box=18.0, multipoles=False)
    ref = ew.ewald(b.x, ew.pack_multipoles(b.q), b.box, grad=False)["E"]
    import torch
    m = api.Ankh(b.box, b.n, n_cells=128, Lu=5, Lc=5, fmm=True, max_order=0)
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    E = m.energy(t32(b.x), t32(b.q), None, None)
    assert E == pytest.approx(ref, rel=1e-4)


def test_charges_only_handle(api):
    """max_order = 0 (no dipole or quadrupole arrays) against the oracle."""
    import torch
    b = synth.water_box(600, 7, box=18.0, multipoles=False)
    o = fm.ankh_fmm_energy(b.x, b.q, None, None, b.box, 3, 5)
    m = api.Ankh(b.box, b.n, n_cells=8, Lu=5, Lc=5, fmm=True, max_order=0)
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    E = m.energy(t32(b.x), t32(b.q), None, None)
    assert E == pytest.approx(o["E"], rel=2e-6)


def test_one_million_atoms_against_ewald(api):
    """The 1,008,000-atom box at the benchmarked tree (n = 64, L = 5): the FP64
    Ewald energy within the method's error at this leaf size (the oracle at the
    same leaf edge and order, 24,000 atoms, 3.5e-6) plus FP32 rounding."""
    b = synth.config_box(4)
    m = api.Ankh(b.box, b.n, n_cells=64, Lu=5, Lc=5, fmm=True)
    E = m.energy(*to_dev(b))
    ref = json.load(open(os.path.join(GOLDEN, "ewald_water_1008000_qmuTheta.json")))["E"]
    assert E == pytest.approx(ref, rel=6e-6)


def test_repeatable_and_translated_box(api):
    """Repeat calls give the same bits (fixed reduction order, static schedule).
    A translated copy of the box (atoms wrapped across the faces, a different
    tree) is compared with the oracle on the same FP32-rounded coordinates:
    this system is stiff enough (near field ~2e6) that the rounding of the
    shifted coordinates alone moves its energy by ~1e-4 relative."""
    b = synth.water_box(600, 7, box=18.0, multipoles=True)
    m = api.Ankh(b.box, b.n, n_cells=8, Lu=5, Lc=5, fmm=True)
    x, q, mu, th = to_dev(b)
    E1 = m.energy(x, q, mu, th)
    assert m.energy(x, q, mu, th) == E1
    xs = (b.x.astype(np.float32) + np.array([0.37, -1.1, 2.9], dtype=np.float32)).astype(np.float32)
    import torch
    E2 = m.energy(torch.from_numpy(xs).cuda(), q, mu, th)
    o = fm.ankh_fmm_energy(xs, b.q, b.mu, b.theta, b.box, 3, 5)
    assert E2 == pytest.approx(o["E"], rel=2e-6)


def test_invalid_uses(api):
    b = synth.water_box(216, 11, box=18.64, multipoles=True)
    with pytest.raises(api.AnkhError) as e:
        api.Ankh(b.box, b.n, n_cells=6, Lu=5, Lc=5, fmm=True)        # not a power of two
    assert e.value.code == api.ANKH_EINVAL
    with pytest.raises(api.AnkhError) as e:
        api.Ankh(b.box, b.n, n_cells=4, Lu=5, Lc=6, fmm=True)        # one order for the tree
    assert e.value.code == api.ANKH_EINVAL
    with pytest.raises(api.AnkhError) as e:
        api.Ankh(b.box, b.n, n_cells=4, Lu=5, Lc=5, fmm=True, nonperiodic=True)
    assert e.value.code == api.ANKH_EINVAL
    m = api.Ankh(b.box, b.n, n_cells=4, Lu=5, Lc=5, fmm=True)
    with pytest.raises(api.AnkhError) as e:
        m.energy_forces(*to_dev(b))                                    # energy only (Alg. 3)
    assert e.value.code == api.ANKH_EINVAL
    x, q, mu, th = to_dev(b)
    import torch
    with pytest.raises(api.AnkhError) as e:
        m.induce(x, q, mu, th, torch.full((b.n,), 0.03, device=x.device))
    assert e.value.code == api.ANKH_EINVAL
    assert m.info["n_cells"] == 4
