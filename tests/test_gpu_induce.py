"""Induced dipoles (ankh_induce) against the dense FP64 oracle solve
(oracle/polarization.py) with the oracle's own field at matched parameters,
and against the two-atom closed form.

Bars: the CG stops at |r| <= 1e-7 |F|; the remaining difference is the FP32
field (~1e-6 relative per evaluation, see test_gpu_parity.py), amplified by
the conditioning of diag(1/alpha) - T (a few): induced dipoles within 1e-4
RMS of their RMS, E_pol within 1e-5.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import ankh_ref as ar            # noqa: E402
from oracle import polarization as pol       # noqa: E402
from paper_2212_08284_gb300 import synth     # noqa: E402


@pytest.fixture(scope="module")
def api(gpu):
    from paper_2212_08284_gb300 import api as A, build
    build.build()
    A.load_library()
    return A


def t32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)))


def test_two_polarizable_charges_closed_form(api):
    alpha, r, q1, q2 = 1.2, 3.1, 0.7, -0.4
    x = np.array([[0.0, 0.0, -r / 2], [0.0, 0.0, r / 2]])
    m = api.Ankh(10.0, 2, n_cells=3, Lu=4, nonperiodic=True)
    mu_ind, E_pol, it = m.induce(t32(x), t32([q1, q2]), None, None, t32([alpha, alpha]), tol=1e-7)
    m1, m2 = pol.two_atom_closed_form(alpha, r, q1, q2)
    got = mu_ind.cpu().numpy()
    assert got[0, 2] == pytest.approx(m1, rel=1e-5)
    assert got[1, 2] == pytest.approx(m2, rel=1e-5)
    assert np.max(np.abs(got[:, :2])) < 1e-7
    assert E_pol == pytest.approx(-0.5 * (m1 * (-q2 / r ** 2) + m2 * (q1 / r ** 2)), rel=1e-5)
    assert 1 <= it <= 5


@pytest.mark.parametrize("nonperiodic", [False, True])
def test_water_box_matches_dense_oracle_solve(api, nonperiodic):
    b = synth.water_box(30, 21, box=9.7, multipoles=True)
    n, Lu = 3, 5
    p = ar.Params(b.box, n, Lu, Lu)
    energy = ar.ankh_energy_nonperiodic if nonperiodic else ar.ankh_energy
    zq, zt = np.zeros(b.n), np.zeros((b.n, 6))

    def field(mu):
        return -energy(b.x, zq, mu, zt, p, grad=True)["grad"][:, 4:7]

    alpha = np.where(b.q < 0, 0.04, 0.03)   # positive definite: min distance 0.51 A > (2 alpha)^(1/3)
    F_perm = -energy(b.x, b.q, b.mu, b.theta, p, grad=True)["grad"][:, 4:7]
    mu_ref, E_ref, _ = pol.induce_dense(field, alpha, F_perm)

    m = api.Ankh(b.box, b.n, n_cells=n, Lu=Lu, Lc=Lu, nonperiodic=nonperiodic)
    mu_ind, E_pol, it = m.induce(t32(b.x), t32(b.q), t32(b.mu), t32(b.theta), t32(alpha), tol=1e-7,
                                 max_iter=60)
    assert rel_rms(mu_ind.cpu().numpy().astype(np.float64), mu_ref) <= 1e-4
    assert E_pol == pytest.approx(E_ref, rel=1e-5)
    assert it < 60


def test_bad_polarizability_and_no_convergence(api):
    b = synth.water_box(30, 21, box=9.7, multipoles=True)
    m = api.Ankh(b.box, b.n, n_cells=3, Lu=5)
    x, q, mu, th = t32(b.x), t32(b.q), t32(b.mu), t32(b.theta)
    alpha = np.full(b.n, 0.03)
    bad = alpha.copy()
    bad[7] = 0.0
    with pytest.raises(api.AnkhError) as e:
        m.induce(x, q, mu, th, t32(bad))
    assert e.value.code == api.ANKH_EINVAL
    with pytest.raises(api.AnkhError) as e:
        m.induce(x, q, mu, th, t32(alpha), tol=1e-12, max_iter=1)
    assert e.value.code == api.ANKH_ENOTCONV
    _, _, it = m.induce(x, q, mu, th, t32(alpha), tol=1e-6)
    assert it >= 1
