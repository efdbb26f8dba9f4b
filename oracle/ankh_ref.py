"""Literal FP64 evaluation of the ANKH-FFT energy (Alg. 5) and its gradient.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import this module.  It shares
no code with the CUDA path.

It follows the paper's steps in the paper's order, at given parameters
(n cells per axis, Chebyshev order L_c, equispaced order L_u, screening xi):

  Step 1 (Alg. 2, Sec. 3.4 and 4.1): modified charges Q_s on the tensor
      Chebyshev grid of each leaf, using S^(p) = H D^p T with the Chebyshev
      differentiation matrix D, then M_s = E_s Q_s on the equispaced grid
      J_L of the leaf (Eq. fromchebtoequispaced).
  Step 2 (Sec. 4.2-4.5, Thm. 1, Cor. 1, Cor. 2): far field
      F = 1/2 v^T A v = (1 / 2 M6) sum_k D(A)_k |w_k|^2,  w = F6 chi v,
      with A built from its first column (Alg. 4) over the 6-D multi-index
      (cell, node) per axis; cell dimensions periodic, node dimensions
      embedded in a circulant of size 2 L_u - 1.
  Step 3 (Alg. 5 step 3): near field, all pairs in the same or the 26
      adjacent leaves (minimum image per offset), kernel H = erfc(xi r)/r.
  Step 4 (Eq. ewald): self term.
  (+) neutralising term -pi Q^2 / (2 V xi^2), see "readings" below.

Readings of passages that are silent or garbled (each is also listed in the
design notes of the repository):
  * Chebyshev nodes r_k = cos((2k+1) pi / (2 L)), k = 0..L-1 (Eq.
    lagrangechebinterp prints them without pi and with a shifted index).
  * The third factor of the tensor Lagrange polynomial is S_k(x_2) (Eq.
    multivariatepolynomials repeats x_1).
  * D is the matrix with T' = D T (strictly lower triangular in this row
    convention; the text calls it upper triangular); x_hat = 2 (x - ctr)/h
    with chain factor (2/h)^p.
  * E_s maps Chebyshev to equispaced nodes as (E)_{b,k} = U_b(r_k), so that
    C ~ E^T G E holds (Eq. fromchebtoequispaced).
  * The equispaced grid J_L spans the whole leaf, [-h/2, h/2] about its
    centre, nodes shared on faces (Fig. 4 caption).
  * Periodicity (Alg. 4, Sec. 4.3): the block of A between target leaf t and
    source leaf s holds, for every image of s that is NOT adjacent to t, the
    kernel H at the node pairs, i.e. Phi(z) - [s adjacent to t] H(z_adj) with
    the full lattice sum Phi(z) = sum_m H(z + L m) (the limit p -> infinity
    of Z_p); the adjacent image belongs to the near field.
  * Phi is evaluated in closed form by a second Ewald split with eta >> xi.
    With include_rec the smooth reciprocal part of the xi split is added to
    Phi as well, so that the result approximates the full Ewald energy
    instead of neglecting E_rec (the paper neglects it for xi = 0.01).
  * The constant pi/(V xi^2) contained in Phi multiplies Q^2 only; the
    tin-foil neutralising term -pi Q^2/(2 V xi^2) is added so that
    non-neutral systems match the Ewald convention (zero for neutral ones).
  * Energies are 1/2 sum over ordered pairs (Eq. 1); the "2 D D G" of the
    mutual loops in Alg. 3/5 counts each unordered pair once.

Non-periodic variant (ankh_energy_nonperiodic; Sec. 5.2, Eq. relerrnonperio):
the kernel is the bare H = 1/|x - y| (no images, no Ewald split: xi = 0),
the leaves tile the box [-r_B, r_B)^3 without wrapping (every atom must lie
inside), the far field couples every pair of NON-adjacent leaves of the box
(the 6-D operator is multilevel Toeplitz in the cell and node displacements
and is embedded in a circulant of size 2n - 1 per cell axis and 2 L_u - 1
per node axis), the near field couples the atoms of the same and adjacent
leaves inside the box, and there is no self or neutralising term.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import erfc

from . import ewald as ew


# ----------------------------------------------------------------------------
# One-dimensional interpolation building blocks (Sec. 3.4, 4.1)

def cheb_nodes(L: int) -> np.ndarray:
    """First-kind Chebyshev nodes r_k = cos((2k+1) pi / (2L)) (Eq. lagrangechebinterp)."""
    k = np.arange(L)
    return np.cos((2 * k + 1) * np.pi / (2 * L))


def cheb_T(xh: np.ndarray, L: int) -> np.ndarray:
    """T_0..T_{L-1} at xh by the three-term recurrence (Eq. recformulacheby)."""
    xh = np.asarray(xh, dtype=np.float64)
    T = np.empty(xh.shape + (L,))
    T[..., 0] = 1.0
    if L > 1:
        T[..., 1] = xh
    for m in range(2, L):
        T[..., m] = 2.0 * xh * T[..., m - 1] - T[..., m - 2]
    return T


def cheb_H(L: int) -> np.ndarray:
    """Matrix H with S(x) = H T(x): H[k,0] = 1/L, H[k,m] = 2 T_m(r_k)/L (Eq. lagrangechebymatrix)."""
    Tr = cheb_T(cheb_nodes(L), L)
    H = 2.0 * Tr / L
    H[:, 0] = 1.0 / L
    return H


def cheb_D(L: int) -> np.ndarray:
    """Differentiation matrix with T'(x) = D T(x) (Eq. derivemanytimes):
    T'_m = sum_{j<m, m-j odd} (2m / c_j) T_j, c_0 = 2, c_j = 1 otherwise."""
    D = np.zeros((L, L))
    for m in range(L):
        for j in range(m):
            if (m - j) % 2 == 1:
                D[m, j] = 2.0 * m / (2.0 if j == 0 else 1.0)
    return D


def equi_nodes(Lu: int) -> np.ndarray:
    """Equispaced nodes of J_L on [-1, 1] (Eq. tensorized_equispaced_grid, leaf-wide reading)."""
    return -1.0 + 2.0 * np.arange(Lu) / (Lu - 1)


def equi_lagrange(Lu: int, x: np.ndarray) -> np.ndarray:
    """Equispaced Lagrange basis U_b(x), b = 0..Lu-1 (product formula)."""
    e = equi_nodes(Lu)
    x = np.asarray(x, dtype=np.float64)
    U = np.ones(x.shape + (Lu,))
    for b in range(Lu):
        for c in range(Lu):
            if c != b:
                U[..., b] *= (x - e[c]) / (e[b] - e[c])
    return U


def reinterp_E(Lu: int, Lc: int) -> np.ndarray:
    """Chebyshev -> equispaced re-interpolation, (E)_{b,k} = U_b(r_k) (Eq. fromchebtoequispaced)."""
    return equi_lagrange(Lu, cheb_nodes(Lc)).T.copy()


# ----------------------------------------------------------------------------

@dataclass
class Params:
    box: float          # edge L = 2 r_B
    n: int              # leaves per axis
    Lu: int             # equispaced order
    Lc: int             # Chebyshev order
    xi: float = 0.01    # Ewald screening (Sec. 5: always 0.01)
    include_rec: bool = True


def bin_atoms(x32: np.ndarray, box: float, n: int):
    """Leaf index of each atom (octree leaves of a perfect tree, uniform grid).

    FP64, correctly rounded, no fused operations:
      s = (x + r_B) * (1/L); s -= floor(s); c = min(floor(s * n), n - 1).
    Returns (cell ids (N,), integer cell coords (N,3), wrapped FP64 positions,
    stable permutation sorting atoms by cell)."""
    x = np.asarray(x32, dtype=np.float64)
    rB = box / 2.0
    inv = 1.0 / box
    s = (x + rB) * inv
    s = s - np.floor(s)
    c = np.minimum(np.floor(s * n), n - 1).astype(np.int64)
    cell = (c[:, 0] * n + c[:, 1]) * n + c[:, 2]
    perm = np.argsort(cell, kind="stable")
    xw = s * box - rB
    return cell, c, xw, perm


def lattice_kernel_table(box: float, nf: int, xi: float, include_rec: bool) -> np.ndarray:
    """Phi(z_j) = sum_m H(z_j + L m) on the periodic grid z_j = j L / nf.

    Closed form by a second Ewald split with eta = 12/L (erfc(eta L/2) ~ 2e-17):
      Phi(z) = sum_m erfc(eta|z+Lm|)/|z+Lm|
             + (4 pi/V) sum_{k!=0} (exp(-k^2/4eta^2) - [not include_rec] exp(-k^2/4xi^2))/k^2 cos(k.z)
             + (pi/V)(1/xi^2 - 1/eta^2).
    At j = 0 the entry holds the finite limit of Phi(z) - H(z) as z -> 0."""
    V = box ** 3
    eta = 12.0 / box
    delta = box / nf
    j = np.arange(nf)
    jm = np.where(j > nf // 2, j - nf, j).astype(np.float64) * delta
    zx, zy, zz = np.meshgrid(jm, jm, jm, indexing="ij")
    real = np.zeros((nf, nf, nf))
    for mx in (-1, 0, 1):
        for my in (-1, 0, 1):
            for mz in (-1, 0, 1):
                r = np.sqrt((zx + box * mx) ** 2 + (zy + box * my) ** 2 + (zz + box * mz) ** 2)
                with np.errstate(divide="ignore", invalid="ignore"):
                    t = erfc(eta * r) / r
                if mx == 0 and my == 0 and mz == 0:
                    t[0, 0, 0] = 2.0 / math.sqrt(math.pi) * (xi - eta)
                real += t
    # reciprocal part, separable contraction over the three axes
    kmax = 12.6 * eta
    mmax = int(math.ceil(kmax * box / (2 * math.pi)))
    m = np.arange(-mmax, mmax + 1)
    MX, MY, MZ = np.meshgrid(m, m, m, indexing="ij")
    k2 = (2 * math.pi / box) ** 2 * (MX ** 2 + MY ** 2 + MZ ** 2).astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        c = np.exp(-k2 / (4 * eta * eta))
        if not include_rec:
            c = c - np.exp(-k2 / (4 * xi * xi))
        c = (4 * math.pi / V) * c / k2
    c[mmax, mmax, mmax] = 0.0
    ph = np.exp(2j * math.pi * np.outer(m, j) / nf)      # (2mmax+1, nf)
    A = np.tensordot(c.astype(np.complex128), ph, axes=([2], [0]))   # (mx, my, jz)
    Bm = np.tensordot(A, ph, axes=([1], [0]))                        # (mx, jz, jy)
    R = np.tensordot(ph, Bm, axes=([0], [0]))                         # (jx, jz, jy)
    R = np.transpose(R, (0, 2, 1)).real
    const = (math.pi / V) * (1.0 / (xi * xi) - 1.0 / (eta * eta))
    return real + R + const


def self_energy(mp: np.ndarray, xi: float):
    """E_self of Eq. ewald for general symmetric Theta (reduces to the printed
    form when Theta is traceless) and its gradient (N x 13)."""
    c = xi / math.sqrt(math.pi)
    a2, a4 = xi * xi, xi ** 4
    q = mp[:, 0]
    mu = mp[:, 1:4]
    th = mp[:, 4:10]
    tr = th[:, 0] + th[:, 3] + th[:, 5]
    TT = th[:, 0] ** 2 + th[:, 3] ** 2 + th[:, 5] ** 2 + 2 * (th[:, 1] ** 2 + th[:, 2] ** 2 + th[:, 4] ** 2)
    e = -c * (q * q + (2 * a2 / 3) * (mu * mu).sum(1) - (4 * a2 / 3) * q * tr
              + (8 * a4 / 5) * TT + (4 * a4 / 5) * tr * tr)
    g = np.zeros((mp.shape[0], 13))
    g[:, 3] = -c * (2 * q - (4 * a2 / 3) * tr)
    g[:, 4:7] = -c * (4 * a2 / 3) * mu
    dg = -(4 * a2 / 3) * q + (8 * a4 / 5) * tr
    k = 16 * a4 / 5
    g[:, 7] = -c * (dg + k * th[:, 0])
    g[:, 8] = -c * 2 * k * th[:, 1]
    g[:, 9] = -c * 2 * k * th[:, 2]
    g[:, 10] = -c * (dg + k * th[:, 3])
    g[:, 11] = -c * 2 * k * th[:, 4]
    g[:, 12] = -c * (dg + k * th[:, 5])
    return float(np.sum(e)), g


# The ten terms of Alg. 2: (multipole column, x/y/z derivative orders, factor)
ALG2_TERMS = [
    (0, (0, 0, 0), 1.0),   # q
    (1, (1, 0, 0), 1.0),   # mu_x
    (2, (0, 1, 0), 1.0),   # mu_y
    (3, (0, 0, 1), 1.0),   # mu_z
    (4, (2, 0, 0), 1.0),   # Theta_xx
    (5, (1, 1, 0), 2.0),   # Theta_xy (x2, symmetry)
    (6, (1, 0, 1), 2.0),   # Theta_xz
    (7, (0, 2, 0), 1.0),   # Theta_yy
    (8, (0, 1, 1), 2.0),   # Theta_yz
    (9, (0, 0, 2), 1.0),   # Theta_zz
]


def basis_derivs(xw, cvec, p: Params, pmax: int = 3):
    """S^(k) = (2/h)^k H D^k T(x_hat) for k = 0..pmax, per axis: (pmax+1, N, 3, Lc)."""
    h = p.box / p.n
    ctr = -p.box / 2.0 + (cvec + 0.5) * h
    xh = 2.0 * (xw - ctr) / h
    T = cheb_T(xh, p.Lc)
    Hm = cheb_H(p.Lc)
    Dm = cheb_D(p.Lc)
    out = []
    Dk = np.eye(p.Lc)
    for k in range(pmax + 1):
        W = Hm @ Dk
        out.append((2.0 / h) ** k * np.einsum("kl,nal->nak", W, T))
        Dk = Dm @ Dk
    return np.stack(out)


def modified_charges(cell, S, mp, p: Params):
    """Alg. 2: Q_s on the Chebyshev grid of every leaf, (n^3, Lc, Lc, Lc)."""
    N = mp.shape[0]
    Lc = p.Lc
    contrib = np.zeros((N, Lc, Lc, Lc))
    for col, (ox, oy, oz), fac in ALG2_TERMS:
        w = fac * mp[:, col]
        if not np.any(w):
            continue
        contrib += w[:, None, None, None] * (S[ox][:, 0, :, None, None] * S[oy][:, 1, None, :, None]
                                             * S[oz][:, 2, None, None, :])
    Q = np.zeros((p.n ** 3, Lc ** 3))
    np.add.at(Q, cell, contrib.reshape(N, -1))
    return Q.reshape(p.n ** 3, Lc, Lc, Lc)


def far_field_matrix_column(p: Params) -> np.ndarray:
    """First column of the 6-D circulant embedding of A (Alg. 4 reading).

    Shape (n, 2Lu-1, n, 2Lu-1, n, 2Lu-1) in the multi-index order (cell_x,
    node_x, cell_y, node_y, cell_z, node_z) of Sec. 4.2."""
    n, Lu = p.n, p.Lu
    h = p.box / n
    nf = n * (Lu - 1)
    delta = h / (Lu - 1)
    P = 2 * Lu - 1
    Phi = lattice_kernel_table(p.box, nf, p.xi, p.include_rec)
    d = np.arange(n)
    slot = np.arange(P)
    e = np.where(slot < Lu, slot, slot - P)
    J = (d[:, None] * (Lu - 1) + e[None, :]) % nf                       # (n, P)
    col = Phi[J[:, :, None, None, None, None], J[None, None, :, :, None, None],
              J[None, None, None, None, :, :]]
    # remove the adjacent image (it is part of the near field)
    adj = (d == 0) | (d == 1) | (d == n - 1)
    dmin = np.where(d == n - 1, -1, d)
    z = (dmin[:, None] * (Lu - 1) + e[None, :]) * delta                 # (n, P)
    zx = z[:, :, None, None, None, None]
    zy = z[None, None, :, :, None, None]
    zz = z[None, None, None, None, :, :]
    r = np.sqrt(zx * zx + zy * zy + zz * zz)
    mask = (adj[:, None, None, None, None, None] & adj[None, None, :, None, None, None]
            & adj[None, None, None, None, :, None])
    mask = np.broadcast_to(mask, r.shape) & (r > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        Hz = np.where(mask, erfc(p.xi * r) / np.where(r > 0, r, 1.0), 0.0)
    return col - Hz


def near_pairs(cvec, perm, p: Params, xw):
    """Ordered pairs (i, j, shift) with j in the same or an adjacent leaf of i
    (periodic, minimum image per offset; i == j at zero offset excluded), in
    CSR form by target."""
    n = p.n
    N = cvec.shape[0]
    cell = (cvec[:, 0] * n + cvec[:, 1]) * n + cvec[:, 2]
    counts = np.bincount(cell, minlength=n ** 3)
    start = np.concatenate([[0], np.cumsum(counts)])
    rows_i, rows_j, rows_s = [], [], []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                sc = cvec + np.array([dx, dy, dz])
                wrap = np.floor_divide(sc, n)
                sc = sc - wrap * n
                scell = (sc[:, 0] * n + sc[:, 1]) * n + sc[:, 2]
                cnt = counts[scell]
                ii = np.repeat(np.arange(N), cnt)
                base = np.repeat(start[scell], cnt)
                off = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
                jj = perm[base + off]
                sh = np.repeat(wrap * p.box, cnt, axis=0).astype(np.float64)
                if dx == 0 and dy == 0 and dz == 0:
                    keep = ii != jj
                    ii, jj, sh = ii[keep], jj[keep], sh[keep]
                rows_i.append(ii)
                rows_j.append(jj)
                rows_s.append(sh)
    ii = np.concatenate(rows_i)
    jj = np.concatenate(rows_j)
    sh = np.concatenate(rows_s)
    order = np.argsort(ii, kind="stable")
    ii, jj, sh = ii[order], jj[order], sh[order]
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(ii, minlength=N))]).astype(np.int64)
    return rowptr, jj.astype(np.int32), sh


def ankh_energy(x32, q, mu, theta, p: Params, grad: bool = True, tensor_pairs: bool = False,
                nthreads: int | None = None) -> dict:
    """ANKH-FFT energy (and its exact gradient) at parameters p, in FP64."""
    if p.n < 3:
        raise ValueError("at least 3 leaves per axis are needed")
    N = len(q)
    mp = ew.pack_multipoles(q, mu, theta)
    cell, cvec, xw, perm = bin_atoms(x32, p.box, p.n)
    n, Lu, Lc = p.n, p.Lu, p.Lc
    V = p.box ** 3

    # Step 1: modified charges (Alg. 2) and re-interpolation (M_s = E_s Q_s)
    S = basis_derivs(xw, cvec, p, pmax=3 if grad else 2)
    Q = modified_charges(cell, S, mp, p)
    E = reinterp_E(Lu, Lc)
    M = np.einsum("ak,bl,cm,sklm->sabc", E, E, E, Q)                   # (n^3, Lu, Lu, Lu)

    # Step 2: far field by the diagonalised circulant embedding (Cor. 1, Cor. 2)
    P = 2 * Lu - 1
    col = far_field_matrix_column(p)
    Dspec = np.fft.fftn(col)
    v = np.zeros((n, P, n, P, n, P))
    v[:, :Lu, :, :Lu, :, :Lu] = M.reshape(n, n, n, Lu, Lu, Lu).transpose(0, 3, 1, 4, 2, 5)
    w = np.fft.fftn(v)
    M6 = v.size
    E_far = float(np.sum(Dspec.real * (w.real ** 2 + w.imag ** 2)) / (2.0 * M6))
    spec_imag = float(np.max(np.abs(Dspec.imag)) / max(np.max(np.abs(Dspec.real)), 1e-300))

    # Step 3: near field (mutual P2P over adjacent leaves)
    rowptr, colj, shift = near_pairs(cvec, perm, p, xw)
    e_pairs, g_near = ew.pair_csr(xw, mp, rowptr, colj, shift, p.xi, tensor=tensor_pairs,
                                  grad=grad, nthreads=nthreads)
    E_near = 0.5 * e_pairs

    # Step 4: self; (+) neutralising term
    E_self, g_self = self_energy(mp, p.xi)
    Qtot = float(np.sum(mp[:, 0]))
    E_neut = -math.pi * Qtot * Qtot / (2.0 * V * p.xi * p.xi)

    out = {"E": E_far + E_near + E_self + E_neut, "E_far": E_far, "E_near": E_near,
           "E_self": E_self, "E_neut": E_neut, "spectrum_imag_rel": spec_imag,
           "M": M, "cell": cell, "perm": perm}
    if not grad:
        return out

    # Adjoint: node potentials Pi = A v, then back through E^T and Alg. 2
    Pi6 = np.fft.ifftn(Dspec * w).real
    Pi = Pi6[:, :Lu, :, :Lu, :, :Lu].transpose(0, 2, 4, 1, 3, 5).reshape(n ** 3, Lu, Lu, Lu)
    PiQ = np.einsum("ak,bl,cm,sabc->sklm", E, E, E, Pi)                # (n^3, Lc, Lc, Lc)
    Pc = PiQ[cell]                                                     # (N, Lc, Lc, Lc)
    Vv = {}
    for ox in range(4):
        X = np.einsum("iklm,ik->ilm", Pc, S[ox][:, 0, :])
        for oy in range(4 - ox):
            Y = np.einsum("ilm,il->im", X, S[oy][:, 1, :])
            for oz in range(4 - ox - oy):
                Vv[(ox, oy, oz)] = np.einsum("im,im->i", Y, S[oz][:, 2, :])
    g_far = np.zeros((N, 13))
    for col_, (ox, oy, oz), fac in ALG2_TERMS:
        g_far[:, 3 + col_] = fac * Vv[(ox, oy, oz)]
        for a, sh in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            g_far[:, a] += fac * mp[:, col_] * Vv[(ox + sh[0], oy + sh[1], oz + sh[2])]
    g_neut = np.zeros((N, 13))
    g_neut[:, 3] = -math.pi * Qtot / (V * p.xi * p.xi)
    out["grad"] = g_far + g_near + g_self + g_neut
    out["grad_far"] = g_far
    out["grad_near"] = g_near
    return out


def torques(mp: np.ndarray, grad: np.ndarray) -> np.ndarray:
    """Torque tau = -dE/d(omega) of a rigid rotation of each atom's multipoles.

    With g = dE/dmu and G_ab = dE/dTheta_ab (each of the nine entries
    independent; the stored off-diagonal derivative is 2 G_ab):
      tau = -(mu x g) - 2 * axial(G Theta),   axial(X)_d = eps_dca X_ac ... written out below."""
    mu = mp[:, 1:4]
    g = grad[:, 4:7]
    th = mp[:, 4:10]
    gd = grad[:, 7:13]
    T = np.stack([np.stack([th[:, 0], th[:, 1], th[:, 2]], 1),
                  np.stack([th[:, 1], th[:, 3], th[:, 4]], 1),
                  np.stack([th[:, 2], th[:, 4], th[:, 5]], 1)], 1)
    G = np.stack([np.stack([gd[:, 0], gd[:, 1] / 2, gd[:, 2] / 2], 1),
                  np.stack([gd[:, 1] / 2, gd[:, 3], gd[:, 4] / 2], 1),
                  np.stack([gd[:, 2] / 2, gd[:, 4] / 2, gd[:, 5]], 1)], 1)
    # dE/domega_d = (mu x g)_d + 2 sum_{a,c} eps_{a d c} (G Theta)_{a c}
    X = np.einsum("nab,nbc->nac", G, T)
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    dW = np.cross(mu, g) + 2.0 * np.einsum("adc,nac->nd", eps, X)
    return -dW


# ----------------------------------------------------------------------------
# Non-periodic ANKH-FFT (Sec. 5.2): bare kernel 1/r, no images

def bin_atoms_nonperiodic(x32: np.ndarray, box: float, n: int):
    """Leaf of each atom of the box [-r_B, r_B)^3 without wrapping (FP64,
    correctly rounded: s = (x + r_B) * (1/L), c = min(floor(s * n), n - 1)).
    Raises if an atom lies outside the box."""
    x = np.asarray(x32, dtype=np.float64)
    rB = box / 2.0
    s = (x + rB) * (1.0 / box)
    if np.any(s < 0.0) or np.any(s >= 1.0):
        raise ValueError("non-periodic: every atom must lie inside the box")
    c = np.minimum(np.floor(s * n), n - 1).astype(np.int64)
    cell = (c[:, 0] * n + c[:, 1]) * n + c[:, 2]
    perm = np.argsort(cell, kind="stable")
    return cell, c, x, perm


def far_field_column_nonperiodic(p: Params) -> np.ndarray:
    """First column of the circulant embedding of the non-periodic far-field
    operator: entry (dc, da) per axis (cell displacement dc in
    [-(n-1), n-1], node displacement da in [-(L_u-1), L_u-1], both embedded
    circularly) holds H(z) = 1/|z| at z = dc h + da delta when the cells are
    NOT adjacent (max |dc| > 1), else 0.  Shape (2n-1, 2Lu-1) x 3."""
    n, Lu = p.n, p.Lu
    h = p.box / n
    delta = h / (Lu - 1)
    Pc, Pn = 2 * n - 1, 2 * Lu - 1
    dc = np.where(np.arange(Pc) < n, np.arange(Pc), np.arange(Pc) - Pc)
    da = np.where(np.arange(Pn) < Lu, np.arange(Pn), np.arange(Pn) - Pn)
    z = dc[:, None] * h + da[None, :] * delta                          # (Pc, Pn)
    zx = z[:, :, None, None, None, None]
    zy = z[None, None, :, :, None, None]
    zz = z[None, None, None, None, :, :]
    r = np.sqrt(zx * zx + zy * zy + zz * zz)
    far = (np.abs(dc) > 1)
    nonadj = (far[:, None, None, None, None, None] | far[None, None, :, None, None, None]
              | far[None, None, None, None, :, None])
    nonadj = np.broadcast_to(nonadj, r.shape)
    with np.errstate(divide="ignore"):
        return np.where(nonadj, 1.0 / np.where(r > 0, r, 1.0), 0.0)


def near_pairs_nonperiodic(cvec, perm, p: Params):
    """Ordered pairs (i, j) with j in the same or an adjacent leaf of i inside
    the box (no wrapping; i == j excluded), CSR by target, zero shifts."""
    n = p.n
    N = cvec.shape[0]
    cell = (cvec[:, 0] * n + cvec[:, 1]) * n + cvec[:, 2]
    counts = np.bincount(cell, minlength=n ** 3)
    start = np.concatenate([[0], np.cumsum(counts)])
    rows_i, rows_j = [], []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                sc = cvec + np.array([dx, dy, dz])
                inside = np.all((sc >= 0) & (sc < n), axis=1)
                scell = np.where(inside, (sc[:, 0] * n + sc[:, 1]) * n + sc[:, 2], 0)
                cnt = np.where(inside, counts[scell], 0)
                ii = np.repeat(np.arange(N), cnt)
                base = np.repeat(start[scell], cnt)
                off = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
                jj = perm[base + off]
                if dx == 0 and dy == 0 and dz == 0:
                    keep = ii != jj
                    ii, jj = ii[keep], jj[keep]
                rows_i.append(ii)
                rows_j.append(jj)
    ii = np.concatenate(rows_i)
    jj = np.concatenate(rows_j)
    order = np.argsort(ii, kind="stable")
    ii, jj = ii[order], jj[order]
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(ii, minlength=N))]).astype(np.int64)
    return rowptr, jj.astype(np.int32), np.zeros((len(jj), 3))


def ankh_energy_nonperiodic(x32, q, mu, theta, p: Params, grad: bool = True, tensor_pairs: bool = False,
                            nthreads: int | None = None) -> dict:
    """Non-periodic ANKH-FFT energy (and its exact gradient) in FP64.

    Steps as in ankh_energy (Alg. 2 and E_s, far field by the diagonalised
    circulant embedding, near field), with the bare kernel and the aperiodic
    (multilevel Toeplitz) far-field operator; xi and include_rec of p are
    not used."""
    N = len(q)
    mp = ew.pack_multipoles(q, mu, theta)
    cell, cvec, xw, perm = bin_atoms_nonperiodic(x32, p.box, p.n)
    n, Lu, Lc = p.n, p.Lu, p.Lc
    S = basis_derivs(xw, cvec, p, pmax=3 if grad else 2)
    Q = modified_charges(cell, S, mp, p)
    E = reinterp_E(Lu, Lc)
    M = np.einsum("ak,bl,cm,sklm->sabc", E, E, E, Q)                   # (n^3, Lu, Lu, Lu)

    Pc, Pn = 2 * n - 1, 2 * Lu - 1
    col = far_field_column_nonperiodic(p)
    Dspec = np.fft.fftn(col)
    v = np.zeros((Pc, Pn, Pc, Pn, Pc, Pn))
    v[:n, :Lu, :n, :Lu, :n, :Lu] = M.reshape(n, n, n, Lu, Lu, Lu).transpose(0, 3, 1, 4, 2, 5)
    w = np.fft.fftn(v)
    E_far = float(np.sum(Dspec.real * (w.real ** 2 + w.imag ** 2)) / (2.0 * v.size))

    rowptr, colj, shift = near_pairs_nonperiodic(cvec, perm, p)
    e_pairs, g_near = ew.pair_csr(xw, mp, rowptr, colj, shift, 0.0, tensor=tensor_pairs, grad=grad,
                                  nthreads=nthreads)
    E_near = 0.5 * e_pairs
    out = {"E": E_far + E_near, "E_far": E_far, "E_near": E_near, "M": M, "cell": cell, "perm": perm}
    if not grad:
        return out
    Pi6 = np.fft.ifftn(Dspec * w).real
    Pi = Pi6[:n, :Lu, :n, :Lu, :n, :Lu].transpose(0, 2, 4, 1, 3, 5).reshape(n ** 3, Lu, Lu, Lu)
    PiQ = np.einsum("ak,bl,cm,sabc->sklm", E, E, E, Pi)
    Pcq = PiQ[cell]
    Vv = {}
    for ox in range(4):
        X = np.einsum("iklm,ik->ilm", Pcq, S[ox][:, 0, :])
        for oy in range(4 - ox):
            Y = np.einsum("ilm,il->im", X, S[oy][:, 1, :])
            for oz in range(4 - ox - oy):
                Vv[(ox, oy, oz)] = np.einsum("im,im->i", Y, S[oz][:, 2, :])
    g_far = np.zeros((N, 13))
    for col_, (ox, oy, oz), fac in ALG2_TERMS:
        g_far[:, 3 + col_] = fac * Vv[(ox, oy, oz)]
        for a, sh in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            g_far[:, a] += fac * mp[:, col_] * Vv[(ox + sh[0], oy + sh[1], oz + sh[2])]
    out["grad"] = g_far + g_near
    out["grad_far"] = g_far
    out["grad_near"] = g_near
    return out


def far_field_dense_nonperiodic(M: np.ndarray, p: Params) -> float:
    """The non-periodic far field written out: 1/2 sum over ordered pairs of
    non-adjacent leaves (t, s) and their equispaced nodes of
    M_t[k] M_s[l] / |x_tk - x_sl|.  For tests (O((n^3 L_u^3)^2))."""
    n, Lu = p.n, p.Lu
    h = p.box / n
    nodes1 = -h / 2 + np.arange(Lu) * (h / (Lu - 1))
    off = np.stack(np.meshgrid(nodes1, nodes1, nodes1, indexing="ij"), -1).reshape(-1, 3)
    cidx = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    ctr = -p.box / 2 + (cidx + 0.5) * h
    pos = (ctr[:, None, :] + off[None, :, :])                            # (n^3, Lu^3, 3)
    Mf = M.reshape(n ** 3, -1)
    tot = 0.0
    for t in range(n ** 3):
        far = np.max(np.abs(cidx - cidx[t]), axis=1) > 1
        if not np.any(far):
            continue
        d = pos[t][:, None, None, :] - pos[far][None, :, :, :]           # (P, nf, P, 3)
        r = np.sqrt(np.sum(d * d, axis=-1))
        tot += float(np.einsum("k,ksl,sl->", Mf[t], 1.0 / r, Mf[far]))
    return 0.5 * tot
