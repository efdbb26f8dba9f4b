"""Pins of the FP64 Ewald oracle against facts outside itself.

Each test checks the oracle against mathematics or published values, not
against a retyped copy of its own formulas:
  * the two pair evaluators (explicit derivative tensors vs scalar expansion);
  * closed forms of the bare Coulomb charge-dipole and dipole-dipole energies;
  * quadrupole terms against finite differences of the charge potential;
  * NaCl Madelung constant 1.747564594633 (textbook value);
  * total energy independent of the splitting parameter alpha, per multipole
    order and for a non-traceless Theta (a wrong constant breaks it);
  * tin-foil energy of a simple cubic lattice of parallel dipoles,
    -(2 pi / 3) mu^2 / a^3 per dipole (Lorentz field, cubic symmetry);
  * the self term against -1/2 lim_{r->0} P_ii erf(a r)/r (series by sympy);
  * translation and permutation invariance; analytic gradient vs central FD.
"""
import math

import numpy as np
import pytest

from oracle import ewald as ew
from oracle import ankh_ref as ar


def rand_system(rng, n, box, q=True, mu=True, th=True, traceless=True, neutral=True):
    x = rng.uniform(-box / 2, box / 2, size=(n, 3))
    qq = rng.normal(size=n) if q else np.zeros(n)
    if neutral and q:
        qq -= qq.mean()
    mm = rng.normal(size=(n, 3)) * 0.4 if mu else np.zeros((n, 3))
    tt = rng.normal(size=(n, 6)) * 0.3 if th else np.zeros((n, 6))
    if th and traceless:
        tr = (tt[:, 0] + tt[:, 3] + tt[:, 5]) / 3
        tt[:, 0] -= tr
        tt[:, 3] -= tr
        tt[:, 5] -= tr
    return x, ew.pack_multipoles(qq, mm, tt)


def test_pair_tensor_equals_scalar():
    rng = np.random.default_rng(11)
    worst = 0.0
    for t in range(300):
        r = rng.normal(size=3) * rng.uniform(0.3, 4.0)
        mi, mk = rng.normal(size=10), rng.normal(size=10)
        a = [0.0, 0.01, 0.35][t % 3]
        o1 = ew.pair(r, mi, mk, a, tensor=True)
        o2 = ew.pair(r, mi, mk, a, tensor=False)
        worst = max(worst, np.max(np.abs(o1 - o2)) / np.max(np.abs(o1)))
    assert worst < 1e-12


def test_pair_closed_forms_bare_coulomb():
    rng = np.random.default_rng(12)
    for _ in range(20):
        r = rng.normal(size=3) * 2
        rn = np.linalg.norm(r)
        qi, qk = rng.normal(size=2)
        di, dk = rng.normal(size=3), rng.normal(size=3)
        # charge (target) - dipole (source): q mu.(x_i - x_k)/r^3
        mi = np.zeros(10); mi[0] = qi
        mk = np.zeros(10); mk[1:4] = dk
        e = ew.pair(r, mi, mk, 0.0, tensor=True)[0]
        assert e == pytest.approx(qi * dk @ r / rn ** 3, rel=1e-12)
        # dipole - dipole: (mu_i.mu_k - 3 (mu_i.r)(mu_k.r)/r^2)/r^3
        mi = np.zeros(10); mi[1:4] = di
        e = ew.pair(r, mi, mk, 0.0, tensor=True)[0]
        ref = (di @ dk - 3 * (di @ r) * (dk @ r) / rn ** 2) / rn ** 3
        assert e == pytest.approx(ref, rel=1e-12)


def test_pair_quadrupole_against_finite_differences():
    """Theta_k : grad grad acting on the source side equals the second
    difference of the charge-charge term (bare and screened kernels)."""
    rng = np.random.default_rng(13)
    hh = 1e-3
    for a in (0.0, 0.3):
        r = rng.normal(size=3) * 1.5 + np.array([2.0, 0.0, 0.0])
        th = rng.normal(size=6)
        full = np.array([[th[0], th[1], th[2]], [th[1], th[3], th[4]], [th[2], th[4], th[5]]])
        mi = np.zeros(10); mi[0] = 1.0
        mk = np.zeros(10); mk[4:10] = th
        e = ew.pair(r, mi, mk, a, tensor=True)[0]
        one = np.zeros(10); one[0] = 1.0
        f = lambda rr: ew.pair(rr, one, one, a, tensor=True)[0]
        fd = 0.0
        for i in range(3):
            for j in range(3):
                ei = np.eye(3)[i] * hh
                ej = np.eye(3)[j] * hh
                d2 = (f(r + ei + ej) - f(r + ei - ej) - f(r - ei + ej) + f(r - ei - ej)) / (4 * hh * hh)
                fd += full[i, j] * d2
        assert e == pytest.approx(fd, rel=2e-6)


def test_pair_gradients_against_fd():
    rng = np.random.default_rng(14)
    for a in (0.0, 0.05):
        r = rng.normal(size=3) + np.array([2.5, 0, 0])
        mi, mk = rng.normal(size=10), rng.normal(size=10)
        out = ew.pair(r, mi, mk, a)
        hh = 1e-5
        for c in range(3):
            d = np.eye(3)[c] * hh
            fd = (ew.pair(r + d, mi, mk, a)[0] - ew.pair(r - d, mi, mk, a)[0]) / (2 * hh)
            assert out[1 + c] == pytest.approx(fd, rel=1e-7, abs=1e-9)
        # e is linear in the target multipoles: exact differences
        base = ew.pair(r, mi * 0, mk, a)[0]
        assert base == pytest.approx(0.0, abs=1e-14)
        for c in range(10):
            u = np.zeros(10); u[c] = 1.0
            val = ew.pair(r, u, mk, a)[0]
            # a stored off-diagonal entry stands for both Theta_ab and Theta_ba,
            # so the unit perturbation gives the stored-entry derivative directly
            assert out[4 + c] == pytest.approx(val, rel=1e-12, abs=1e-13)


def nacl(a=1.0, shift=(0.123, 0.377, 0.051)):
    pos, q = [], []
    for i in range(2):
        for j in range(2):
            for k in range(2):
                pos.append([i * a, j * a, k * a])
                q.append((-1) ** (i + j + k))
    return np.array(pos) + np.array(shift), np.array(q, dtype=float)


def test_madelung_nacl():
    x, q = nacl()
    r = ew.ewald(x, ew.pack_multipoles(q), 2.0, tol=1e-14)
    M = 1.747564594633
    assert r["E"] == pytest.approx(-8 * M / 2.0, rel=2e-12)
    # larger supercell, different offset
    pos, qq = [], []
    for i in range(4):
        for j in range(4):
            for k in range(4):
                pos.append([i, j, k])
                qq.append((-1) ** (i + j + k))
    x2 = np.array(pos, float) * 1.7 + np.array([0.61, -0.2, 0.33])
    r2 = ew.ewald(x2, ew.pack_multipoles(np.array(qq, float)), 4 * 1.7, tol=1e-14)
    assert r2["E"] == pytest.approx(-64 * M / (2 * 1.7), rel=2e-12)


@pytest.mark.parametrize("kind", ["q", "mu", "theta", "theta_trace", "mixed", "mixed_charged"])
def test_alpha_invariance(kind):
    rng = np.random.default_rng({"q": 1, "mu": 2, "theta": 3, "theta_trace": 4,
                                 "mixed": 5, "mixed_charged": 6}[kind])
    box = 7.0
    opts = dict(q=kind in ("q", "mixed", "mixed_charged"), mu=kind in ("mu", "mixed", "mixed_charged"),
                th=kind in ("theta", "theta_trace", "mixed", "mixed_charged"),
                traceless=kind != "theta_trace" and kind != "mixed_charged",
                neutral=kind != "mixed_charged")
    x, mp = rand_system(rng, 12, box, **opts)
    vals = []
    for aL in (4.0, 7.0, 11.0):
        alpha = aL / box
        s = math.sqrt(-math.log(1e-15))
        r = ew.ewald(x, mp, box, alpha=alpha, rc=s / alpha, kc=2 * alpha * s, grad=False)
        vals.append(r["E"])
    ref = max(abs(v) for v in vals)
    assert max(vals) - min(vals) < 1e-10 * ref


def test_dipole_lattice_lorentz_energy():
    """Parallel dipoles on a simple cubic lattice, tin-foil: the spherical
    lattice sum vanishes by cubic symmetry, leaving -2 pi |M|^2 / (3V)."""
    a, mu = 2.3, 0.7
    for ncell in (1, 2):
        pos = np.array([[i, j, k] for i in range(ncell) for j in range(ncell) for k in range(ncell)],
                       float) * a + 0.31
        n = len(pos)
        mp = ew.pack_multipoles(np.zeros(n), np.tile([0.0, 0.0, mu], (n, 1)))
        r = ew.ewald(pos, mp, ncell * a, tol=1e-14)
        assert r["E"] == pytest.approx(-2 * math.pi / 3 * n * mu * mu / a ** 3, rel=1e-11)


def test_self_term_is_limit_of_erf_pair():
    """E_self = -1/2 sum_i lim_{r->0} P_ii erf(a r)/r.  The B-function limits
    of erf(a r)/r at r = 0 come from its Maclaurin series (sympy); the pair
    operator is the explicit tensor contraction."""
    sympy = pytest.importorskip("sympy")
    r_, a_ = sympy.symbols("r a", positive=True)
    f = sympy.erf(a_ * r_) / r_
    Bs = [f]
    for _ in range(5):
        Bs.append(sympy.simplify(-sympy.diff(Bs[-1], r_) / r_))
    alpha = 0.37
    B0 = np.array([float(sympy.limit(b.subs(a_, alpha), r_, 0)) for b in Bs])
    rng = np.random.default_rng(7)
    for _ in range(5):
        m = rng.normal(size=10)
        # tensor contraction at r = 0 with the limiting B values
        lib = ew._load()
        out = np.zeros(14)
        rr = np.array([0.0, 0.0, 0.0])
        lib.or_pair_tensor(ew._dp(rr), ew._dp(B0), ew._dp(m), ew._dp(m), ew._dp(out))
        es, _ = ar.self_energy(m[None, :], alpha)
        assert es == pytest.approx(-0.5 * out[0], rel=1e-12)


def test_translation_permutation_invariance_and_fd_gradient():
    rng = np.random.default_rng(21)
    box = 8.0
    x, mp = rand_system(rng, 10, box)
    r0 = ew.ewald(x, mp, box, tol=1e-14)
    t = rng.normal(size=3) * 3
    r1 = ew.ewald(x + t, mp, box, tol=1e-14, grad=False)
    assert r1["E"] == pytest.approx(r0["E"], rel=1e-12)
    pm = rng.permutation(len(x))
    r2 = ew.ewald(x[pm], mp[pm], box, tol=1e-14)
    assert r2["E"] == pytest.approx(r0["E"], rel=1e-12)
    assert np.allclose(r2["grad"], r0["grad"][pm], rtol=1e-9, atol=1e-11)
    hh = 1e-5
    g = r0["grad"]
    for i in (0, 3, 7):
        for c in range(3):
            xp = x.copy(); xp[i, c] += hh
            xm = x.copy(); xm[i, c] -= hh
            fd = (ew.ewald(xp, mp, box, tol=1e-14, grad=False)["E"]
                  - ew.ewald(xm, mp, box, tol=1e-14, grad=False)["E"]) / (2 * hh)
            assert g[i, c] == pytest.approx(fd, rel=1e-6, abs=1e-8)
        for c in range(10):
            mpp = mp.copy(); mpp[i, c] += hh
            mpm = mp.copy(); mpm[i, c] -= hh
            fd = (ew.ewald(x, mpp, box, tol=1e-14, grad=False)["E"]
                  - ew.ewald(x, mpm, box, tol=1e-14, grad=False)["E"]) / (2 * hh)
            assert g[i, 3 + c] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_torque_matches_rotation_fd():
    rng = np.random.default_rng(31)
    box = 8.0
    x, mp = rand_system(rng, 8, box)
    r0 = ew.ewald(x, mp, box, tol=1e-14)
    tau = ar.torques(mp, r0["grad"])

    def rotated(i, axis, ang):
        c, s = math.cos(ang), math.sin(ang)
        k = np.eye(3)[axis]
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        R = np.eye(3) + s * K + (1 - c) * K @ K
        m = mp.copy()
        m[i, 1:4] = R @ mp[i, 1:4]
        th = mp[i, 4:10]
        T = np.array([[th[0], th[1], th[2]], [th[1], th[3], th[4]], [th[2], th[4], th[5]]])
        T2 = R @ T @ R.T
        m[i, 4:10] = [T2[0, 0], T2[0, 1], T2[0, 2], T2[1, 1], T2[1, 2], T2[2, 2]]
        return m

    hh = 1e-5
    for i in (0, 5):
        for axis in range(3):
            ep = ew.ewald(x, rotated(i, axis, hh), box, tol=1e-14, grad=False)["E"]
            em = ew.ewald(x, rotated(i, axis, -hh), box, tol=1e-14, grad=False)["E"]
            assert -(ep - em) / (2 * hh) == pytest.approx(tau[i, axis], rel=1e-6, abs=1e-9)
