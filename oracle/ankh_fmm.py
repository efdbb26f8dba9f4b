"""Literal FP64 ANKH-FMM energy (Sec. 3, Alg. 3).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import this module.  It shares
no code with the CUDA path.

Steps in the paper's order, on a perfect octree of depth E (n = 2^E leaves
per axis) over the box [-r_B, r_B)^3, with a tensor Chebyshev grid of L nodes
per axis in every cell of every level (Sec. 3.5: Lagrange interpolation over
products of 1-D Chebyshev grids along the whole tree):

  Step 1: modified charges Q_s of every leaf (Alg. 2, S^(p) = (2/h)^p H D^p T)
          taken as its multipole expansion M_s; M2M up the tree,
          M_parent += V[parent, child] M_child with
          V[parent, child]_{k,l} = S_k[parent](y_l^child) (Eq. M2M).
  Step 2: far field of the box and its 3^3 - 1 direct images by mutual M2L:
          at every level e >= 1 each cell t of the box interacts with the
          cells s (of the box or of a direct image) whose parent is adjacent
          to t's parent but which are not adjacent to t,
              F_real = 1/2 sum_e sum_t sum_{s in Lambda(t)} M_t^T C[t,s] M_s,
          C[t,s]_{k,l} = H(x_k^t - y_l^s), H = erfc(xi r)/r; a cell of an image
          carries the expansion of its copy in the box (Sec. 3.6).
  Step 3: near field: all pairs in the same or adjacent leaves (as ANKH-FFT).
  Step 4: periodic influence of the images beyond the direct ones, with the
          root expansion M_B:  F_per = 1/2 M_B^T K M_B,
              K_{k,l} = sum_{|I|_inf >= 2} H(x_k - x_l - 2 r_B I)
          evaluated as the full lattice sum minus the 27 nearest terms (the
          limit p -> infinity of Z_p, as for ANKH-FFT).
  Step 5: self term (Eq. ewald); (+) the neutralising term.
  Step 6: E = F_real + N_real + F_per + E_self (+ E_neut).

Readings: the mutual M2L of Alg. 3 (2 M_s^T C[s,t] M_t per unordered pair)
is written here as the ordered sum with the factor 1/2 (the same number);
the Eq. ewald self-term line is used (Alg. 3 step 5 misses a '+').  The
paper diagonalises the step-4 operator by a circulant embedding over an
equispaced root grid (Sec. 3.3); here K is applied directly (it is only
L^3 x L^3), which is the same operator.  With include_rec the smooth
reciprocal part of the xi split is added to K (for all pairs; it is smooth
over the box) so that the result approximates the full Ewald energy; without
it E_rec(xi) is neglected as in the paper.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

from . import ankh_ref as ar
from . import ewald as ew


def lagrange_cheb(L: int, x: np.ndarray) -> np.ndarray:
    """S_k(x) for k = 0..L-1 at points x (Eq. lagrangechebymatrix: S = H T); (len(x), L)."""
    T = ar.cheb_T(np.asarray(x, dtype=np.float64), L)             # (..., L)
    return T @ ar.cheb_H(L).T


def m2m_1d(L: int) -> np.ndarray:
    """V_b[k, l] = S_k((2b - 1 + r_l) / 2): the parent's 1-D basis at the nodes of
    its lower (b = 0) and upper (b = 1) child, in the parent's [-1, 1] frame."""
    r = ar.cheb_nodes(L)
    return np.stack([lagrange_cheb(L, (2 * b - 1 + r) / 2.0).T for b in (0, 1)])   # (2, L, L)


def lattice_sum_grid(ax: np.ndarray, ay: np.ndarray, az: np.ndarray, box: float, xi: float,
                     include_rec: bool) -> np.ndarray:
    """Phi(z) = sum_m erfc(xi |z + L m|)/|z + L m| on the tensor grid of points
    z = (ax[i], ay[j], az[k]), all |components| < L, by a second Ewald split with
    eta = 12/L (as ankh_ref.lattice_kernel_table): real images of erfc(eta r)/r,
    the band-limited reciprocal difference (separable over the axes) and the
    constant (pi/V)(1/xi^2 - 1/eta^2); include_rec adds the xi reciprocal part.
    At z = 0 the entry is the limit of Phi(z) - H(z) (the lattice without the
    origin term)."""
    V = box ** 3
    eta = 12.0 / box
    X, Y, Z = np.meshgrid(ax, ay, az, indexing="ij")
    out = np.zeros(X.shape)
    for mx in (-1, 0, 1):
        for my in (-1, 0, 1):
            for mz in (-1, 0, 1):
                r = np.sqrt((X + box * mx) ** 2 + (Y + box * my) ** 2 + (Z + box * mz) ** 2)
                with np.errstate(divide="ignore", invalid="ignore"):
                    t = erfc(eta * r) / r
                if mx == 0 and my == 0 and mz == 0:
                    t = np.where(r > 0, t, 2.0 / math.sqrt(math.pi) * (xi - eta))
                out += t
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
    ph = lambda a: np.exp(2j * math.pi * np.outer(m, a) / box)          # (2mmax+1, len(a))
    R = np.einsum("abc,ai,bj,ck->ijk", c.astype(np.complex128), ph(ax), ph(ay), ph(az), optimize=True).real
    return out + R + (math.pi / V) * (1.0 / (xi * xi) - 1.0 / (eta * eta))


def node_offsets(L: int, h: float) -> np.ndarray:
    """Tensor Chebyshev nodes of a cell of edge h about its centre, (L^3, 3), index (kx, ky, kz)."""
    r = ar.cheb_nodes(L) * (h / 2.0)
    return np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)


def interaction_offsets(parity):
    """Offsets d (cell units) of Lambda(t) for a cell of the given parity (t mod 2 per
    axis): the parent of t + d adjacent to t's parent, t + d not adjacent to t."""
    rng = [range(-2 - p, 4 - p) for p in parity]
    return [(dx, dy, dz) for dx in rng[0] for dy in rng[1] for dz in rng[2]
            if max(abs(dx), abs(dy), abs(dz)) >= 2]


def ankh_fmm_energy(x32, q, mu, theta, box: float, depth: int, L: int, xi: float = 0.01,
                    include_rec: bool = True, nthreads: int | None = None) -> dict:
    """ANKH-FMM energy at tree depth E = depth (n = 2^depth leaves per axis) and
    Chebyshev order L in every cell, FP64."""
    n = 2 ** depth
    if n < 4:
        raise ValueError("depth >= 2 (at least 4 leaves per axis)")
    mp = ew.pack_multipoles(q, mu, theta)
    p = ar.Params(box, n, L, L, xi=xi, include_rec=include_rec)
    cell, cvec, xw, perm = ar.bin_atoms(x32, box, n)
    # Step 1: leaf modified charges = leaf multipole expansions, then M2M
    S = ar.basis_derivs(xw, cvec, p, pmax=2)
    M = {depth: ar.modified_charges(cell, S, mp, p)}                  # (n^3, L, L, L)
    V = m2m_1d(L)
    for e in range(depth - 1, -1, -1):
        nc, ne = 2 ** (e + 1), 2 ** e
        Mc = M[e + 1].reshape(nc, nc, nc, L, L, L)
        Mp = np.zeros((ne, ne, ne, L, L, L))
        for bx in (0, 1):
            for by in (0, 1):
                for bz in (0, 1):
                    ch = Mc[bx::2, by::2, bz::2]
                    Mp += np.einsum("ka,lb,mc,xyzabc->xyzklm", V[bx], V[by], V[bz], ch)
        M[e] = Mp.reshape(ne ** 3, L, L, L)
    # Step 2: mutual M2L over the box and its direct images, every level e >= 1
    F_real = 0.0
    for e in range(1, depth + 1):
        ne = 2 ** e
        h = box / ne
        off = node_offsets(L, h)
        Me = M[e].reshape(ne, ne, ne, L ** 3)
        cache = {}
        for px in (0, 1):
            for py in (0, 1):
                for pz in (0, 1):
                    Mt = Me[px::2, py::2, pz::2]                         # target cells of this parity
                    tx, ty, tz = np.meshgrid(np.arange(px, ne, 2), np.arange(py, ne, 2),
                                             np.arange(pz, ne, 2), indexing="ij")
                    for d in interaction_offsets((px, py, pz)):
                        if d not in cache:
                            z = off[:, None, :] - off[None, :, :] - np.asarray(d, dtype=np.float64) * h
                            r = np.sqrt(np.sum(z * z, axis=-1))
                            cache[d] = erfc(xi * r) / r                  # (L^3, L^3)
                        Ms = Me[(tx + d[0]) % ne, (ty + d[1]) % ne, (tz + d[2]) % ne]
                        F_real += 0.5 * float(np.einsum("xyzk,kl,xyzl->", Mt, cache[d], Ms))
    # Step 3: near field
    rowptr, colj, shift = ar.near_pairs(cvec, perm, p, xw)
    e_pairs, _ = ew.pair_csr(xw, mp, rowptr, colj, shift, xi, grad=False, nthreads=nthreads)
    N_real = 0.5 * e_pairs
    # Step 4: images beyond the direct ones, through the root expansion.
    # Node differences of the root's tensor grid are a tensor grid themselves.
    r1 = ar.cheb_nodes(L) * (box / 2.0)
    d1 = (r1[:, None] - r1[None, :]).reshape(-1)                          # (L^2,), index (k, l)
    G = lattice_sum_grid(d1, d1, d1, box, xi, include_rec)                # (L^2, L^2, L^2)
    D = np.stack(np.meshgrid(d1, d1, d1, indexing="ij"), -1)
    for Ix in (-1, 0, 1):
        for Iy in (-1, 0, 1):
            for Iz in (-1, 0, 1):
                s = D + box * np.array([Ix, Iy, Iz])
                r = np.sqrt(np.sum(s * s, axis=-1))
                with np.errstate(divide="ignore", invalid="ignore"):
                    G -= np.where(r > 0, erfc(xi * r) / np.where(r > 0, r, 1.0), 0.0)
    # G[(kx,lx),(ky,ly),(kz,lz)] -> K[(kx,ky,kz),(lx,ly,lz)]
    K = G.reshape(L, L, L, L, L, L).transpose(0, 2, 4, 1, 3, 5).reshape(L ** 3, L ** 3)
    Mb = M[0].reshape(-1)
    F_per = 0.5 * float(Mb @ K @ Mb)
    # Step 5: self term; neutralising term
    E_self, _ = ar.self_energy(mp, xi)
    Qtot = float(np.sum(mp[:, 0]))
    E_neut = -math.pi * Qtot * Qtot / (2.0 * box ** 3 * xi * xi)
    return {"E": F_real + N_real + F_per + E_self + E_neut, "F_real": F_real, "N_real": N_real,
            "F_per": F_per, "E_self": E_self, "E_neut": E_neut, "M_root": M[0]}
