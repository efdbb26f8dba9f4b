"""Pins of the induced-dipole oracle (oracle/polarization.py)."""
import numpy as np
import pytest

from oracle import ewald as ew
from oracle import polarization as pol
from paper_2212_08284_gb300 import synth


def _direct_field(x):
    def field(mu, q=None):
        n = len(x)
        _, g = ew.direct_nonperiodic(x, ew.pack_multipoles(np.zeros(n) if q is None else q, mu))
        return -g[:, 4:7]
    return field


def test_two_polarizable_charges_closed_form():
    alpha, r, q1, q2 = 1.2, 3.1, 0.7, -0.4
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, r]])
    field = _direct_field(x)
    Fp = field(np.zeros((2, 3)), q=np.array([q1, q2]))
    mu, E_pol, T = pol.induce_dense(field, np.array([alpha, alpha]), Fp)
    m1, m2 = pol.two_atom_closed_form(alpha, r, q1, q2)
    assert mu[0, 2] == pytest.approx(m1, rel=1e-12)
    assert mu[1, 2] == pytest.approx(m2, rel=1e-12)
    assert np.allclose(mu[:, :2], 0.0, atol=1e-15)
    assert E_pol == pytest.approx(-0.5 * (m1 * Fp[0, 2] + m2 * Fp[1, 2]), rel=1e-12)


def test_field_matrix_is_symmetric_and_solution_satisfies_the_equations():
    b = synth.water_box(12, 4, box=9.0, multipoles=True)
    x = b.x.astype(np.float64)
    alpha = np.where(b.q < 0, 0.84, 0.50)
    field = _direct_field(x)
    Fp = field(b.mu.astype(np.float64), q=b.q.astype(np.float64))
    mu, _, T = pol.induce_dense(field, alpha, Fp)
    assert np.max(np.abs(T - T.T)) <= 1e-12 * np.max(np.abs(T))
    # mu = alpha (F_perm + T mu), with T mu evaluated afresh by the field routine
    assert np.allclose(mu, alpha[:, None] * (Fp + field(mu)), rtol=1e-10, atol=1e-12)


def test_periodic_field_matrix_is_symmetric():
    b = synth.water_box(8, 2, box=7.5, multipoles=False)
    x = b.x.astype(np.float64)

    def field(mu):
        out = ew.ewald(x, ew.pack_multipoles(np.zeros(b.n), mu), b.box, grad=True)
        return -out["grad"][:, 4:7]

    T = pol.field_matrix(field, b.n)
    assert np.max(np.abs(T - T.T)) <= 1e-9 * np.max(np.abs(T))
