"""Pins of the non-periodic oracle (Sec. 5.2, Eq. relerrnonperio): the bare
Coulomb direct sum and the literal non-periodic ANKH-FFT, checked against
things other than themselves."""
import itertools
import math

import numpy as np
import pytest

from oracle import ankh_ref as ar
from oracle import ewald as ew
from paper_2212_08284_gb300 import synth


@pytest.fixture(scope="module")
def box648():
    b = synth.water_box(216, 11, box=18.64, multipoles=True)
    mp = ew.pack_multipoles(b.q, b.mu, b.theta)
    Ed, gd = ew.direct_nonperiodic(b.x.astype(np.float64), mp)
    return b, mp, Ed, gd


def test_direct_sum_charges_is_the_double_loop():
    rng = np.random.default_rng(3)
    x = rng.uniform(-5, 5, size=(30, 3))
    q = rng.normal(size=30)
    E, g = ew.direct_nonperiodic(x, ew.pack_multipoles(q))
    ref = 0.0
    fx = np.zeros((30, 3))
    for i, j in itertools.permutations(range(30), 2):
        d = x[i] - x[j]
        r = np.linalg.norm(d)
        ref += 0.5 * q[i] * q[j] / r
        fx[i] += -q[i] * q[j] * d / r ** 3
    assert E == pytest.approx(ref, rel=1e-13)
    assert np.allclose(g[:, :3], fx, rtol=1e-12, atol=1e-14)


def test_direct_sum_dipole_pair_closed_form():
    # two point dipoles: E = (mu1.mu2 - 3 (mu1.r)(mu2.r)/r^2) / r^3
    x = np.array([[0.0, 0.0, 0.0], [1.3, -0.4, 0.7]])
    mu = np.array([[0.2, -0.5, 0.3], [-0.1, 0.4, 0.6]])
    E, _ = ew.direct_nonperiodic(x, ew.pack_multipoles(np.zeros(2), mu))
    r = x[1] - x[0]
    rr = np.linalg.norm(r)
    ref = (mu[0] @ mu[1] - 3 * (mu[0] @ r) * (mu[1] @ r) / rr ** 2) / rr ** 3
    assert E == pytest.approx(ref, rel=1e-13)


def test_direct_rows_are_rows_of_the_direct_sum(box648):
    b, mp, _, gd = box648
    rows = [0, 17, 301, 647]
    gr = ew.direct_nonperiodic_rows(b.x.astype(np.float64), mp, rows)
    assert np.allclose(gr, gd[rows], rtol=1e-13, atol=1e-13)


def test_far_field_fft_equals_dense_double_loop(box648):
    b, mp, _, _ = box648
    for n, Lu in ((4, 4), (3, 5)):
        p = ar.Params(b.box, n, Lu, Lu)
        o = ar.ankh_energy_nonperiodic(b.x, b.q, b.mu, b.theta, p, grad=False)
        dense = ar.far_field_dense_nonperiodic(o["M"], p)
        assert o["E_far"] == pytest.approx(dense, rel=1e-12, abs=1e-12)


def test_geometric_convergence_to_the_direct_sum(box648):
    """Error against the independent direct sum falls geometrically with the
    interpolation order L = L_c = L_u (Sec. 5.2)."""
    b, mp, Ed, gd = box648
    errs = []
    for L in (3, 5, 7, 9):
        o = ar.ankh_energy_nonperiodic(b.x, b.q, b.mu, b.theta, ar.Params(b.box, 3, L, L), grad=True)
        errs.append(np.sqrt(np.mean((o["grad"] - gd) ** 2)) / np.sqrt(np.mean(gd ** 2)))
        last = o
    for a, c in zip(errs, errs[1:]):
        assert c < a / 5
    assert abs(last["E"] - Ed) / abs(Ed) < 1e-8


def test_equispaced_order_caps_the_accuracy(box648):
    """L_c >= L_u gives exactly the L_u = L_c result (the fused basis is the
    equispaced Lagrange basis): the error stagnates at the L_u level."""
    b, _, _, _ = box648
    e4 = ar.ankh_energy_nonperiodic(b.x, b.q, b.mu, b.theta, ar.Params(b.box, 4, 4, 4), grad=False)["E"]
    e48 = ar.ankh_energy_nonperiodic(b.x, b.q, b.mu, b.theta, ar.Params(b.box, 4, 4, 8), grad=False)["E"]
    assert e48 == pytest.approx(e4, rel=1e-12)


def test_adjoint_matches_finite_differences():
    b = synth.water_box(60, 5, box=12.0, multipoles=True)
    x = b.x.astype(np.float64)
    p = ar.Params(b.box, 3, 4, 4)
    o = ar.ankh_energy_nonperiodic(x, b.q, b.mu, b.theta, p, grad=True)
    h = (b.box / 3)
    frac = (x + b.box / 2) / h
    dist = np.min(np.abs(frac - np.round(frac)), axis=1) * h
    atoms = np.where(dist > 0.01)[0][:6]
    hfd = 1e-5
    for i in atoms:
        for c in range(3):
            xp = x.copy(); xp[i, c] += hfd
            xm = x.copy(); xm[i, c] -= hfd
            ep = ar.ankh_energy_nonperiodic(xp, b.q, b.mu, b.theta, p, grad=False)["E"]
            em = ar.ankh_energy_nonperiodic(xm, b.q, b.mu, b.theta, p, grad=False)["E"]
            assert o["grad"][i, c] == pytest.approx((ep - em) / (2 * hfd), rel=1e-6, abs=1e-7)
    # dE/dq by finite differences on one charge
    k = atoms[0]
    qp, qm = b.q.astype(np.float64).copy(), b.q.astype(np.float64).copy()
    qp[k] += 1e-6
    qm[k] -= 1e-6
    ep = ar.ankh_energy_nonperiodic(x, qp, b.mu, b.theta, p, grad=False)["E"]
    em = ar.ankh_energy_nonperiodic(x, qm, b.mu, b.theta, p, grad=False)["E"]
    assert o["grad"][k, 3] == pytest.approx((ep - em) / 2e-6, rel=1e-6)


def test_atoms_outside_the_box_are_rejected():
    b = synth.water_box(30, 2, box=10.0, multipoles=False)
    x = b.x.copy()
    x[0, 0] = 5.0 + 1e-3
    with pytest.raises(ValueError):
        ar.ankh_energy_nonperiodic(x, b.q, None, None, ar.Params(10.0, 3, 3, 3), grad=False)
    assert math.isfinite(ar.ankh_energy_nonperiodic(b.x, b.q, None, None, ar.Params(10.0, 3, 3, 3),
                                                    grad=False)["E"])
