"""Leaf binning and sort on clustered inputs, and the near field on heavy
leaves, through the C ABI.

The sort is a stable radix sort by leaf id whose cost per atom does not
depend on the leaf occupancy; the near field takes a leaf's targets in work
items of at most 32, so a heavy leaf is spread over many warps.  Binning and
sorting are integer work: the permutation and the leaf offsets must equal the
oracle's (bin_atoms: the FP64 leaf definition, stable order by leaf, then by
atom index) bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import ankh_ref as ar          # noqa: E402
from cases import clustered_half_in_eight, clustered_one_leaf, heavy_leaf_box, uniform_box   # noqa: E402


@pytest.fixture(scope="module")
def api(gpu):
    from paper_2212_08284_gb300 import api as A, build
    build.build()
    A.load_library()
    return A


def ordering(api, b, n):
    m = api.Ankh(b.box, b.n, n_cells=n, Lu=5, max_order=0)
    import torch
    x = torch.from_numpy(np.ascontiguousarray(b.x)).cuda()
    q = torch.from_numpy(np.ascontiguousarray(b.q)).cuda()
    m.energy(x, q, None, None)
    perm = api.ankh_debug_copy(m.h, api.BUF_PERM).cpu().numpy()
    start = api.ankh_debug_copy(m.h, api.BUF_START).cpu().numpy()
    scell = api.ankh_debug_copy(m.h, api.BUF_SCELL).cpu().numpy()
    m.close()
    return perm, start, scell


def check_against_oracle(b, n, perm, start, scell):
    cell, _, _, operm = ar.bin_atoms(b.x, b.box, n)
    ostart = np.concatenate([[0], np.cumsum(np.bincount(cell, minlength=n ** 3))])
    assert np.array_equal(perm, operm)
    assert np.array_equal(start, ostart)
    assert np.array_equal(scell, cell[operm])
    return np.diff(ostart)


def test_sort_every_atom_in_one_leaf(api):
    b, n = clustered_one_leaf()
    occ = check_against_oracle(b, n, *ordering(api, b, n))
    assert occ.max() == b.n


def test_sort_half_the_atoms_in_eight_leaves(api):
    b, n = clustered_half_in_eight()
    occ = check_against_oracle(b, n, *ordering(api, b, n))
    assert np.sort(occ)[-8:].sum() >= b.n // 2


def test_heavy_leaf_energy_and_gradient_match_fp64_ankh(api):
    """1,000 atoms of a 3,000-atom water box moved onto a jittered 0.44 A
    lattice inside one leaf (32 near-field work items for that leaf, and 27
    leaves that see it as a neighbour), charges only: energy within 2e-6 of
    the literal FP64 ANKH-FFT, every gradient entry within 20 x 3e-5 of the
    RMS and the RMS within 3e-5."""
    import torch
    b, n = heavy_leaf_box()
    Lu = 5
    m = api.Ankh(b.box, b.n, n_cells=n, Lu=Lu, max_order=0, mixed=False)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    E, gr = m.energy_forces(t(b.x), t(b.q), None, None)
    o = ar.ankh_energy(b.x, b.q, b.mu, b.theta, ar.Params(b.box, n, Lu, Lu))
    assert E == pytest.approx(o["E"], rel=2e-6)
    G = np.concatenate([gr["dEdx"].cpu().numpy(), gr["dEdq"].cpu().numpy()[:, None]], axis=1).astype(np.float64)
    for sl in (slice(0, 3), slice(3, 4)):
        ref = o["grad"][:, sl]
        rms = np.sqrt(np.mean(ref ** 2))
        err = G[:, sl] - ref
        assert np.sqrt(np.mean(err ** 2)) <= 3e-5 * rms
        assert np.max(np.abs(err)) <= 20 * 3e-5 * rms
    m.close()


@pytest.mark.parametrize("N,n", [(20000, 8), (20000, 12), (30000, 16), (30000, 18), (700000, 16)],
                         ids=["9bit_one_pass", "11bit_wide", "12bit_wide", "13bit_two_passes",
                              "12bit_171_tiles_two_passes"])
def test_sort_plans_match_oracle(api, N, n):
    """Every shape of the radix plan (one pass of up to 10 bits; one wide pass
    of 11-12 bits where the 4,096-atom tiles fit one wave of the SMs; two
    passes otherwise) orders uniform random atoms exactly as the oracle."""
    b = uniform_box(N, seed=N + n)
    check_against_oracle(b, n, *ordering(api, b, n))


def test_wide_radix_pass_saves_three_launches(api):
    """12-bit leaf ids on one wave of tiles take one radix pass (histogram,
    scan, scatter), 13-bit ids two: the library's launch count differs by
    exactly those three kernels."""
    counts = []
    for n in (16, 18):
        m = api.Ankh(60.0, 30000, n_cells=n, Lu=5, max_order=0)
        counts.append(api.ankh_launch_count(m.h, False))
        m.close()
    assert counts[1] - counts[0] == 3
