"""Induced dipoles of point-polarizable atoms, FP64 (test infrastructure).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import this module.  It shares
no code with the CUDA path.

The use of the method named in Sec. 1 and 6 of the paper (polarizable force
fields: repeated field evaluations): each atom i carries an isotropic
polarizability alpha_i and an induced dipole

    mu_i = alpha_i (F_i^perm + F_i(mu)),

where F_i^perm is the electric field of the permanent multipoles at atom i
and F_i(mu) the field of the induced dipoles of all OTHER atoms (and of all
periodic images, the atom's own included).  The field is minus the gradient
of the energy with respect to the atom's dipole, F_i = -dE/dmu_i, which is
what every energy routine of the oracle returns.  The field of a dipole
distribution is linear in it, F(mu) = T mu with T symmetric (T is the
second derivative of -E), so

    (diag(1/alpha) - T) mu = F^perm.

`induce_dense` builds T column by column from unit dipoles and solves this
system directly: plain and slow, for small systems.  The polarization energy
is E_pol = -1/2 sum_i mu_i . F_i^perm.
"""
from __future__ import annotations

import numpy as np


def field_matrix(field_fn, n_atoms: int) -> np.ndarray:
    """T (3N x 3N) with T[3i+a, 3j+b] = a-component of the field at atom i of
    a unit dipole along b on atom j (all other atoms' dipoles zero)."""
    T = np.zeros((3 * n_atoms, 3 * n_atoms))
    for j in range(n_atoms):
        for b in range(3):
            mu = np.zeros((n_atoms, 3))
            mu[j, b] = 1.0
            T[:, 3 * j + b] = field_fn(mu).reshape(-1)
    return T


def induce_dense(field_fn, alpha: np.ndarray, F_perm: np.ndarray):
    """Solve (diag(1/alpha) - T) mu = F_perm; returns (mu N x 3, E_pol, T)."""
    n = len(alpha)
    T = field_matrix(field_fn, n)
    A = np.diag(np.repeat(1.0 / np.asarray(alpha, dtype=np.float64), 3)) - T
    mu = np.linalg.solve(A, np.asarray(F_perm, dtype=np.float64).reshape(-1)).reshape(n, 3)
    E_pol = -0.5 * float(np.sum(mu * F_perm))
    return mu, E_pol, T


def two_atom_closed_form(alpha: float, r: float, q1: float, q2: float):
    """Two polarizable charges on the z axis (atom 1 at 0, atom 2 at +r), no
    images: the permanent fields are F1 = -q2/r^2, F2 = +q1/r^2 (along z),
    the dipole-dipole field along the axis is 2 mu/r^3, so
        mu1 = alpha (F1 + 2 mu2 / r^3),  mu2 = alpha (F2 + 2 mu1 / r^3).
    Returns (mu1_z, mu2_z)."""
    F1, F2 = -q2 / r ** 2, q1 / r ** 2
    c = 2.0 * alpha / r ** 3
    det = 1.0 - c * c
    mu1 = alpha * (F1 + c * F2) / det
    mu2 = alpha * (F2 + c * F1) / det
    return mu1, mu2
