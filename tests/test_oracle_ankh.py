"""Pins of the literal FP64 ANKH-FFT reference against facts outside itself.

  * Chebyshev-Lagrange basis: S_k(r_j) = delta_kj, partition of unity;
  * differentiation matrix against numpy's Chebyshev derivative;
  * H D^p T reproduces the p-th derivative of polynomials of degree < L;
  * E_c direction: for L_u <= L_c the fused Chebyshev -> equispaced map equals
    the equispaced Lagrange basis and its derivatives (numpy polyfit/polyder);
  * the closed-form periodic kernel table against brute-force image sums;
  * the FFT-diagonalised far field against a dense double loop over leaf
    pairs, node pairs and images (Thm. 1 indexing, DFT normalisation);
  * geometric convergence towards the independent Ewald oracle;
  * the analytic adjoint against central finite differences;
  * bit-exact binning of atoms on and next to leaf faces;
  * moments of the modified charges: the leaf interpolation reproduces
    polynomials of degree < L_u, so per leaf sum_b M_b f(y_b) =
    sum_i (q_i + mu_i . grad + Theta_i : grad grad) f(x_i) for f = 1, y, y y^T.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as C
from scipy.special import erfc

from oracle import ankh_ref as ar
from oracle import ewald as ew
from paper_2212_08284_gb300 import synth


@pytest.mark.parametrize("L", [2, 3, 5, 8, 11])
def test_chebyshev_lagrange_basis(L):
    r = ar.cheb_nodes(L)
    S = ar.cheb_T(r, L) @ ar.cheb_H(L).T      # S[j, k] = S_k(r_j)
    assert np.allclose(S, np.eye(L), atol=1e-13)
    x = np.linspace(-1, 1, 17)
    assert np.allclose((ar.cheb_T(x, L) @ ar.cheb_H(L).T).sum(1), 1.0, atol=1e-13)


@pytest.mark.parametrize("L", [2, 4, 7, 10])
def test_differentiation_matrix(L):
    D = ar.cheb_D(L)
    for m in range(L):
        cm = np.zeros(L); cm[m] = 1.0
        d = C.chebder(cm)                   # coefficients of T_m' in the T basis
        ref = np.zeros(L); ref[:len(d)] = d
        assert np.allclose(D[m], ref, atol=1e-12)


def test_derivative_reproduction():
    rng = np.random.default_rng(3)
    L = 7
    r = ar.cheb_nodes(L)
    x = rng.uniform(-1, 1, 9)
    coef = rng.normal(size=L)               # polynomial of degree L-1
    f = np.polynomial.Polynomial(coef)
    Hm, Dm = ar.cheb_H(L), ar.cheb_D(L)
    T = ar.cheb_T(x, L)
    Dp = np.eye(L)
    for p in range(4):
        Sp = T @ (Hm @ Dp).T                # Sp[i, k] = S_k^(p)(x_i)
        assert np.allclose(Sp @ f(r), f.deriv(p)(x) if p else f(x), rtol=1e-10, atol=1e-10)
        Dp = Dm @ Dp


@pytest.mark.parametrize("Lu,Lc", [(3, 3), (4, 6), (5, 5), (5, 8), (6, 6)])
def test_reinterpolation_equals_equispaced_basis(Lu, Lc):
    x = np.linspace(-1, 1, 13)
    E = ar.reinterp_E(Lu, Lc)
    Hm, Dm = ar.cheb_H(Lc), ar.cheb_D(Lc)
    T = ar.cheb_T(x, Lc)
    e = ar.equi_nodes(Lu)
    Dp = np.eye(Lc)
    for p in range(4):
        W = E @ Hm @ Dp                     # (Lu, Lc)
        got = T @ W.T                       # (x, Lu)
        for b in range(Lu):
            yb = np.zeros(Lu); yb[b] = 1.0
            poly = np.polynomial.Polynomial.fit(e, yb, Lu - 1).convert()
            ref = poly.deriv(p)(x) if p else poly(x)
            assert np.allclose(got[:, b], ref, rtol=1e-9, atol=1e-9)
        Dp = Dm @ Dp


def test_lattice_kernel_table_against_image_sums():
    box, nf, xi = 5.0, 10, 0.35
    tab = ar.lattice_kernel_table(box, nf, xi, include_rec=False)
    delta = box / nf
    rng = np.random.default_rng(5)
    R = 6
    m = np.arange(-R, R + 1)
    MX, MY, MZ = np.meshgrid(m, m, m, indexing="ij")
    imgs = np.stack([MX.ravel(), MY.ravel(), MZ.ravel()], 1) * box
    for _ in range(12):
        j = rng.integers(0, nf, 3)
        z = j * delta
        r = np.linalg.norm(z + imgs, axis=1)
        if np.all(j == 0):
            # limit of Phi - H at z = 0: the sum over all other images
            rr = r[r > 0]
            ref = np.sum(erfc(xi * rr) / rr)
        else:
            ref = np.sum(erfc(xi * r) / r)
        assert tab[tuple(j)] == pytest.approx(ref, rel=1e-11, abs=1e-12)
    tab0 = tab[0, 0, 0]
    rr = np.linalg.norm(imgs, axis=1)
    rr = rr[rr > 0]
    assert tab0 == pytest.approx(np.sum(erfc(xi * rr) / rr), rel=1e-11)
    # include_rec adds (4 pi / V) sum_{k != 0} exp(-k^2/4 xi^2)/k^2 cos(k.z), summed explicitly
    tab2 = ar.lattice_kernel_table(box, nf, xi, include_rec=True)
    V = box ** 3
    kk = 2 * math.pi / box
    for _ in range(6):
        j = rng.integers(0, nf, 3)
        z = j * delta
        s = 0.0
        for mx in range(-12, 13):
            for my in range(-12, 13):
                for mz in range(-12, 13):
                    if mx == my == mz == 0:
                        continue
                    k = kk * np.array([mx, my, mz])
                    k2 = k @ k
                    s += math.exp(-k2 / (4 * xi * xi)) / k2 * math.cos(k @ z)
        assert tab2[tuple(j)] - tab[tuple(j)] == pytest.approx(4 * math.pi / V * s, rel=1e-10, abs=1e-12)


def test_fft_far_field_equals_dense_double_loop():
    b = synth.small_box(40, 99, box=9.0)
    p = ar.Params(box=b.box, n=3, Lu=3, Lc=4, xi=0.05, include_rec=False)
    out = ar.ankh_energy(b.x, b.q, b.mu, b.theta, p, grad=False)
    M = out["M"].reshape(p.n ** 3, -1)          # (cells, Lu^3)
    n, Lu = p.n, p.Lu
    nf = n * (Lu - 1)
    delta = p.box / nf
    Phi = ar.lattice_kernel_table(p.box, nf, p.xi, p.include_rec)
    cells = np.array([[a, bb, c] for a in range(n) for bb in range(n) for c in range(n)])
    nodes = np.array([[a, bb, c] for a in range(Lu) for bb in range(Lu) for c in range(Lu)])
    F = 0.0
    for t in range(n ** 3):
        for s in range(n ** 3):
            d = (cells[t] - cells[s]) % n
            adjacent = np.all((d == 0) | (d == 1) | (d == n - 1))
            dmin = np.where(d == n - 1, -1, d)
            for k in range(Lu ** 3):
                for l in range(Lu ** 3):
                    jv = (cells[t] - cells[s]) * (Lu - 1) + nodes[k] - nodes[l]
                    val = Phi[tuple(jv % nf)]
                    if adjacent:
                        z = (dmin * (Lu - 1) + nodes[k] - nodes[l]) * delta
                        rz = np.linalg.norm(z)
                        if rz > 0:
                            val -= erfc(p.xi * rz) / rz
                    F += 0.5 * M[t, k] * val * M[s, l]
    assert out["E_far"] == pytest.approx(F, rel=1e-11)
    assert out["spectrum_imag_rel"] < 1e-12


def test_composition_identity_and_convergence_to_ewald():
    b = synth.small_box(72, 7, box=12.0)
    mp = ew.pack_multipoles(b.q, b.mu, b.theta)
    ref = ew.ewald(b.x.astype(np.float64), mp, b.box, tol=1e-14, grad=False)["E"]
    e55 = ar.ankh_energy(b.x, b.q, b.mu, b.theta, ar.Params(b.box, 4, 5, 5), grad=False)["E"]
    e58 = ar.ankh_energy(b.x, b.q, b.mu, b.theta, ar.Params(b.box, 4, 5, 8), grad=False)["E"]
    assert e58 == pytest.approx(e55, rel=1e-12)
    errs = []
    for L in (3, 7, 11):
        e = ar.ankh_energy(b.x, b.q, b.mu, b.theta, ar.Params(b.box, 4, L, L), grad=False)["E"]
        errs.append(abs(e - ref) / abs(ref))
    # geometric decay O(nu^L) (Sec. 5.1-5.3): 8.8e-6, 2.1e-7, 6.7e-9 here
    assert errs[2] < 1e-8
    assert errs[0] > 30 * errs[1] > 30 * 30 * errs[2] * 0.5
    # paper-literal (neglects E_rec): differs from the full Ewald energy by E_rec(xi)
    lit = ar.ankh_energy(b.x, b.q, b.mu, b.theta, ar.Params(b.box, 4, 11, 11, include_rec=False),
                         grad=False)["E"]
    s = math.sqrt(-math.log(1e-15))
    erec = ew.ewald_rec_only(b.x.astype(np.float64), mp, b.box, 0.01, 2 * 0.01 * s)[0]
    assert lit + erec == pytest.approx(ref, rel=2e-8)


def test_nonneutral_system_matches_ewald():
    b = synth.small_box(60, 17, box=11.0)
    q = b.q.astype(np.float64) + 0.05
    mp = ew.pack_multipoles(q, b.mu, b.theta)
    ref = ew.ewald(b.x.astype(np.float64), mp, b.box, tol=1e-14, grad=False)["E"]
    e = ar.ankh_energy(b.x, q, b.mu, b.theta, ar.Params(b.box, 4, 10, 10), grad=False)["E"]
    # same interpolation error (~1e-7 at L = 10) as the neutral system
    assert e == pytest.approx(ref, rel=3e-7)


def test_adjoint_against_finite_differences():
    b = synth.small_box(30, 23, box=9.5)
    p = ar.Params(box=b.box, n=3, Lu=4, Lc=5, xi=0.05)
    x = b.x.astype(np.float64)
    out = ar.ankh_energy(x, b.q, b.mu, b.theta, p)
    g = out["grad"]
    h = p.box / p.n
    rng = np.random.default_rng(2)
    hh = 1e-5
    mpb = ew.pack_multipoles(b.q, b.mu, b.theta)
    # atoms far enough from every leaf face that the step does not switch near/far
    frac = (x + p.box / 2) / h
    dist = np.min(np.abs(frac - np.round(frac)), axis=1) * h
    cand = np.where(dist > 20 * hh)[0]
    for i in rng.choice(cand, 4, replace=False):
        for c in range(3):
            xp = x.copy(); xp[i, c] += hh
            xm = x.copy(); xm[i, c] -= hh
            fd = (ar.ankh_energy(xp, b.q, b.mu, b.theta, p, grad=False)["E"]
                  - ar.ankh_energy(xm, b.q, b.mu, b.theta, p, grad=False)["E"]) / (2 * hh)
            assert g[i, c] == pytest.approx(fd, rel=1e-6, abs=1e-8)
        for c in range(10):
            mpp = mpb.copy(); mpp[i, c] += 1e-4
            mpm = mpb.copy(); mpm[i, c] -= 1e-4
            ep = ar.ankh_energy(x, mpp[:, 0], mpp[:, 1:4], mpp[:, 4:10], p, grad=False)["E"]
            em = ar.ankh_energy(x, mpm[:, 0], mpm[:, 1:4], mpm[:, 4:10], p, grad=False)["E"]
            assert g[i, 3 + c] == pytest.approx((ep - em) / 2e-4, rel=1e-8, abs=1e-10)


def test_binning_on_faces():
    box, n = 10.0, 5
    h = box / n
    xs = np.array([-5.0, -5.0 + h, 5.0 - 1e-6, 5.0, 4.999999, -1e-7, 0.0, 2.0, 123.0, -7.5],
                  dtype=np.float32)
    x = np.stack([xs, np.zeros_like(xs), np.zeros_like(xs)], 1).astype(np.float32)
    cell, cvec, xw, perm = ar.bin_atoms(x, box, n)
    assert list(cvec[:, 0]) == [0, 1, 4, 0, 4, 2, 2, 3, 4, 3]
    assert np.all(xw >= -box / 2) and np.all(xw < box / 2)
    assert np.array_equal(perm, np.argsort(cell, kind="stable"))


@pytest.mark.parametrize("Lu,Lc", [(3, 3), (5, 6), (6, 6)])
def test_modified_charge_moments(Lu, Lc):
    """Alg. 2 with the E_c re-interpolation (reading of Sec. 4.1): the nodes'
    modified charges carry the atoms' multipole moments about the leaf
    centre exactly (to FP64 rounding): total charge; charge-weighted position
    plus dipole; charge-weighted second moment plus the dipole terms plus
    twice the quadrupole.  A sign slip on mu, a missing factor on an
    off-diagonal Theta entry or on the chain factor 2/h breaks one of them."""
    b = synth.small_box(400, 77, box=22.0)
    n = 4
    p = ar.Params(b.box, n, Lu, Lc)
    mp = ew.pack_multipoles(b.q, b.mu, b.theta)
    cell, cvec, xw, perm = ar.bin_atoms(b.x, p.box, n)
    S = ar.basis_derivs(xw, cvec, p, pmax=2)
    Q = ar.modified_charges(cell, S, mp, p)
    E = ar.reinterp_E(Lu, Lc)
    M = np.einsum("ak,bl,cm,sklm->sabc", E, E, E, Q)            # (n^3, Lu, Lu, Lu)
    h = p.box / n
    ctr = -p.box / 2.0 + (cvec + 0.5) * h
    r = xw - ctr                                                 # atom about its leaf centre
    e = ar.equi_nodes(Lu) * (h / 2.0)                            # node offsets about the centre
    ones = np.ones(Lu)
    ax = [np.einsum("a,b,c->abc", e, ones, ones), np.einsum("a,b,c->abc", ones, e, ones),
          np.einsum("a,b,c->abc", ones, ones, e)]
    q = mp[:, 0]
    mu = mp[:, 1:4]
    th = np.zeros((len(q), 3, 3))
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for k, (a, c) in enumerate(iu):
        th[:, a, c] = th[:, c, a] = mp[:, 4 + k]

    def per_leaf(v):
        out = np.zeros((n ** 3,) + v.shape[1:])
        np.add.at(out, cell, v)
        return out

    scale = np.max(np.abs(M))
    # f = 1
    assert np.allclose(M.sum(axis=(1, 2, 3)), per_leaf(q), atol=1e-12 * scale * Lu ** 3)
    # f = y_a
    for a in range(3):
        lhs = np.einsum("sabc,abc->s", M, ax[a])
        rhs = per_leaf(q * r[:, a] + mu[:, a])
        assert np.allclose(lhs, rhs, atol=1e-11 * scale * Lu ** 3 * h)
    # f = y_a y_c
    for a in range(3):
        for c in range(3):
            lhs = np.einsum("sabc,abc->s", M, ax[a] * ax[c])
            rhs = per_leaf(q * r[:, a] * r[:, c] + mu[:, a] * r[:, c] + mu[:, c] * r[:, a] + 2.0 * th[:, a, c])
            assert np.allclose(lhs, rhs, atol=1e-11 * scale * Lu ** 3 * h * h)

