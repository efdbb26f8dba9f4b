"""Non-periodic ANKH-FFT (Sec. 5.2) through the C ABI against the FP64 oracle.

Bars as in test_gpu_parity.py (FP32 arithmetic on the GPU): energy within
2e-6 and every gradient group within 3e-5 RMS of the literal FP64
non-periodic ANKH at the same (n, L_u, L_c); against the FP64 direct sum
within the method's own error plus 2e-6.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import ankh_ref as ar          # noqa: E402
from oracle import ewald as ew             # noqa: E402
from paper_2212_08284_gb300 import synth   # noqa: E402


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


def rel_rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)) / max(np.sqrt(np.mean(b ** 2)), 1e-300))


def rel_max(a, b):
    """Largest entry error relative to the RMS value of the reference."""
    return float(np.max(np.abs(a - b)) / max(np.sqrt(np.mean(b ** 2)), 1e-300))


def close_grad(a, b, bar=3e-5):
    """RMS error within the bar and every entry within 20 times it."""
    return rel_rms(a, b) <= bar and rel_max(a, b) <= 20 * bar


CASES = [  # (n_waters, seed, box, multipoles, n, Lu)
    (216, 11, 18.64, True, 3, 5),
    (216, 11, 18.64, True, 4, 4),
    (216, 12, 18.64, False, 5, 6),
    (700, 13, 27.5, True, 6, 5),
    (2000, 14, 39.0, True, 9, 5),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("mixed", [True, False])
def test_matches_fp64_nonperiodic_ankh(api, case, mixed):
    nw, seed, box, mpl, n, Lu = case
    b = synth.water_box(nw, seed, box=box, multipoles=mpl)
    m = api.Ankh(b.box, b.n, n_cells=n, Lu=Lu, Lc=Lu, mixed=mixed, nonperiodic=True)
    x, q, mu, th = to_dev(b)
    E, g = m.energy_forces(x, q, mu, th)
    o = ar.ankh_energy_nonperiodic(b.x, b.q, b.mu, b.theta, ar.Params(b.box, n, Lu, Lu), grad=True)
    assert E == pytest.approx(o["E"], rel=2e-6)
    ref = o["grad"]
    assert close_grad(g["dEdx"].cpu().numpy().astype(np.float64), ref[:, :3])
    assert close_grad(g["dEdq"].cpu().numpy().astype(np.float64), ref[:, 3])
    if mpl:
        assert close_grad(g["dEdmu"].cpu().numpy().astype(np.float64), ref[:, 4:7])
        assert close_grad(g["dEdtheta"].cpu().numpy().astype(np.float64), ref[:, 7:13])


def test_against_the_direct_sum(api):
    """At n = 3, L_u = 7 the method's error is ~1e-7 (oracle); the GPU result
    stays within FP32 rounding of the direct sum."""
    b = synth.water_box(216, 11, box=18.64, multipoles=True)
    Ed, gd = ew.direct_nonperiodic(b.x.astype(np.float64), ew.pack_multipoles(b.q, b.mu, b.theta))
    m = api.Ankh(b.box, b.n, n_cells=3, Lu=7, Lc=7, nonperiodic=True)
    E, g = m.energy_forces(*to_dev(b))
    assert E == pytest.approx(Ed, rel=3e-6)
    assert close_grad(g["dEdx"].cpu().numpy().astype(np.float64), gd[:, :3])


@pytest.mark.parametrize("mixed", [True, False])
def test_energy_only_equals_energy_with_forces(api, mixed):
    """The energy-only call sums the adjacent-leaf correction over d = 0 and
    the 13 positive offsets (C_(-d) = C_d^T, zero rows beyond the faces), the
    forces call over all 27: the same energy to rounding."""
    b = synth.water_box(700, 13, box=27.5, multipoles=True)
    m = api.Ankh(b.box, b.n, n_cells=6, Lu=5, nonperiodic=True, mixed=mixed)
    x, q, mu, th = to_dev(b)
    E1 = m.energy(x, q, mu, th)
    E2, _ = m.energy_forces(x, q, mu, th)
    assert E1 == pytest.approx(E2, rel=1e-6)


def test_atom_outside_the_box_is_rejected(api):
    import torch
    b = synth.water_box(216, 11, box=18.64, multipoles=True)
    m = api.Ankh(b.box, b.n, n_cells=4, Lu=5, nonperiodic=True)
    x, q, mu, th = to_dev(b)
    E0 = m.energy(x, q, mu, th)
    xo = x.clone()
    xo[17, 2] = 9.5   # beyond r_B = 9.32
    with pytest.raises(api.AnkhError) as e:
        m.energy(xo, q, mu, th)
    assert e.value.code == api.ANKH_EINVAL
    assert m.energy(x, q, mu, th) == E0
    del torch
