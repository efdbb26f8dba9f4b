"""Pins of the ANKH-FMM oracle (Sec. 3, Alg. 3), each against something
other than the oracle's own formula: Ewald energies, brute-force image sums,
brute-force adjacency over the tree, and the exactness of polynomial
re-interpolation."""
import itertools

import numpy as np
import pytest
from scipy.special import erfc

from oracle import ankh_fmm as fm
from oracle import ankh_ref as ar
from oracle import ewald as ew
from paper_2212_08284_gb300 import synth


@pytest.fixture(scope="module")
def water600():
    b = synth.water_box(600, 7, box=18.0, multipoles=True)
    E_full = ew.ewald(b.x, ew.pack_multipoles(b.q, b.mu, b.theta), b.box, grad=False)["E"]
    E_q = ew.ewald(b.x, ew.pack_multipoles(b.q), b.box, grad=False)["E"]
    return b, E_full, E_q


def test_interaction_lists_cover_every_non_adjacent_pair_once():
    # Brute force over the 27-box region: for a leaf t of an n = 8 tree and every
    # leaf s of the box or a direct image (coordinates in [-n, 2n)), the pair is
    # taken at exactly one level (ancestor offsets in that level's list) if the
    # leaves are not adjacent, and at none if they are.
    depth = 3
    n = 2 ** depth
    rng = np.random.default_rng(0)
    for t in [tuple(rng.integers(0, n, 3)) for _ in range(3)] + [(0, 0, 0), (n - 1, n - 1, n - 1)]:
        for s in itertools.product(range(-n, 2 * n), repeat=3):
            hits = 0
            for e in range(1, depth + 1):
                sh = depth - e
                te = [c >> sh for c in t]
                se = [c >> sh for c in s]          # floor division for negative coordinates too
                d = tuple(b - a for a, b in zip(te, se))
                if d in fm.interaction_offsets(tuple(c % 2 for c in te)):
                    hits += 1
            adjacent = max(abs(a - b) for a, b in zip(t, s)) <= 1
            assert hits == (0 if adjacent else 1), (t, s, hits)


def test_interaction_list_is_symmetric():
    # s in Lambda(t) iff t in Lambda(s): the mutual M2L of Sec. 3.6 relies on it
    for par in itertools.product((0, 1), repeat=3):
        for d in fm.interaction_offsets(par):
            back = tuple((p + dd) % 2 for p, dd in zip(par, d))
            assert tuple(-dd for dd in d) in fm.interaction_offsets(back)
        assert len(fm.interaction_offsets(par)) == 6 ** 3 - 27


def test_m2m_equals_direct_expansion_of_the_parent(water600):
    # A parent's Lagrange basis is a polynomial of degree L-1 per axis, so its
    # interpolation on a child's Chebyshev grid is exact: M2M of the children's
    # modified charges equals the parent's modified charges computed directly
    # from the atoms (Eq. M2M).
    b, _, _ = water600
    L = 5
    mp = ew.pack_multipoles(b.q, b.mu, b.theta)
    V = fm.m2m_1d(L)

    def charges(n):
        p = ar.Params(b.box, n, L, L)
        cell, cvec, xw, _ = ar.bin_atoms(b.x, b.box, n)
        return ar.modified_charges(cell, ar.basis_derivs(xw, cvec, p, pmax=2), mp, p)

    Mc = charges(4).reshape(4, 4, 4, L, L, L)
    Mp = np.zeros((2, 2, 2, L, L, L))
    for bx, by, bz in itertools.product((0, 1), repeat=3):
        Mp += np.einsum("ka,lb,mc,xyzabc->xyzklm", V[bx], V[by], V[bz], Mc[bx::2, by::2, bz::2])
    direct = charges(2)
    assert np.max(np.abs(Mp.reshape(direct.shape) - direct)) <= 1e-11 * np.max(np.abs(direct))


def test_lattice_sum_matches_brute_force_images():
    # Without the reciprocal part and with a large screening the image sum
    # converges absolutely: Phi(z) = sum_m erfc(xi |z + L m|) / |z + L m|.
    box, xi = 10.0, 0.35
    rng = np.random.default_rng(1)
    ax, ay, az = (np.sort(rng.uniform(-0.9 * box, 0.9 * box, 4)) for _ in range(3))
    ax[1] = ay[2] = az[0] = 0.0
    got = fm.lattice_sum_grid(ax, ay, az, box, xi, include_rec=False)
    ms = np.array(list(itertools.product(range(-5, 6), repeat=3)), dtype=np.float64) * box
    for i, j, k in itertools.product(range(4), repeat=3):
        z = np.array([ax[i], ay[j], az[k]])
        r = np.linalg.norm(z + ms, axis=1)
        keep = r > 0                        # at z = 0 the entry is the sum without the origin
        ref = float(np.sum(erfc(xi * r[keep]) / r[keep]))
        assert got[i, j, k] == pytest.approx(ref, rel=1e-12, abs=1e-14)


def test_fmm_converges_to_ewald_with_multipoles(water600):
    b, E_full, _ = water600
    o = fm.ankh_fmm_energy(b.x, b.q, b.mu, b.theta, b.box, 3, 5)
    assert abs(o["E"] - E_full) <= 1e-6 * abs(E_full)
    o2 = fm.ankh_fmm_energy(b.x, b.q, b.mu, b.theta, b.box, 2, 5)
    assert abs(o2["E"] - E_full) <= 5e-6 * abs(E_full)


def test_fmm_charges_error_falls_with_the_order(water600):
    # The charge-only energy is small (neutral molecules), so the relative
    # error is larger than with multipoles, and it must fall with L.
    b, _, E_q = water600
    z3, z6 = np.zeros((b.n, 3)), np.zeros((b.n, 6))
    errs = [abs(fm.ankh_fmm_energy(b.x, b.q, z3, z6, b.box, 3, L)["E"] - E_q) / abs(E_q) for L in (4, 6)]
    assert errs[1] < errs[0] / 10
    assert errs[1] <= 3e-6


def test_fmm_nacl_madelung():
    # 8 ions of +-1 on a simple-cubic lattice of spacing a in a box 2a, with a
    # random offset so that no ion sits on a cell face: E = -N M / (2a).
    a = 2.3
    rng = np.random.default_rng(5)
    pts = np.array(list(itertools.product((0, 1), repeat=3)), dtype=np.float64)
    q = np.where(pts.sum(axis=1) % 2 == 0, 1.0, -1.0)
    x = pts * a - a + rng.uniform(0.1, 0.3, 3)
    # Ions two leaves apart meet in the level-2 M2L: the interpolation error
    # of a unit charge at distance 2h is the bar (3.6e-3 at L = 4, 1.4e-5 at L = 7).
    o = fm.ankh_fmm_energy(x, q, np.zeros((8, 3)), np.zeros((8, 6)), 2 * a, 2, 7, xi=0.2)
    madelung = 1.747564594633182
    assert o["E"] == pytest.approx(-8 * madelung / (2 * a), rel=3e-5)


def test_translation_of_the_whole_system_leaves_the_energy(water600):
    b, _, _ = water600
    e0 = fm.ankh_fmm_energy(b.x, b.q, b.mu, b.theta, b.box, 2, 5)["E"]
    e1 = fm.ankh_fmm_energy(b.x + np.array([0.37, -1.1, 2.9]), b.q, b.mu, b.theta, b.box, 2, 5)["E"]
    assert e1 == pytest.approx(e0, rel=5e-6)
    assert e1 != e0              # different trees: not the same arithmetic
