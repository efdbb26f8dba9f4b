"""The far-field factorisation that the CUDA path uses, written out in FP64
here, against the paper's literal far field (the oracle's masked 6-D block
Toeplitz operator with duplicated face nodes, Alg. 4 / Thm. 1).

The CUDA path merges the duplicated face nodes onto one periodic grid of
n (L_u - 1) points per axis and applies one circulant kernel
  G(z) = Phi(z) - [|z|_inf < h] H(z),
then removes, for every pair of adjacent leaves (t, t + d), the node pairs at
|z|_inf >= h that G still holds:
  F = (1/2M) sum_k D_k |rho^_k|^2 - 1/2 sum_t sum_d M_t^T C_d M_(t+d),
  (C_d)_kl = H((k - l - d (L_u - 1)) delta) [ |k - l - d (L_u - 1)|_inf >= L_u - 1 ].
Both are exact rewritings of the same energy, so they agree to rounding.
"""
import math

import numpy as np
import pytest
from scipy.special import erfc

from oracle import ankh_ref as ar
from paper_2212_08284_gb300 import synth


def merged_far_field(M, box, n, Lu, xi):
    nf = n * (Lu - 1)
    dl = box / n / (Lu - 1)
    Phi = ar.lattice_kernel_table(box, nf, xi, True)
    j = np.arange(nf)
    jm = np.where(j > nf // 2, j - nf, j)
    JX, JY, JZ = np.meshgrid(jm, jm, jm, indexing="ij")
    jmax = np.maximum(np.maximum(abs(JX), abs(JY)), abs(JZ))
    with np.errstate(divide="ignore", invalid="ignore"):
        H = erfc(xi * dl * np.sqrt(JX ** 2 + JY ** 2 + JZ ** 2)) / (dl * np.sqrt(JX ** 2 + JY ** 2 + JZ ** 2))
    G = Phi - np.where((jmax < Lu - 1) & (jmax > 0), H, 0.0)   # j = 0 holds the limit of Phi - H already
    D = np.fft.fftn(G).real
    Mg = M.reshape(n, n, n, Lu, Lu, Lu)
    rho = np.zeros((nf, nf, nf))
    idx = lambda a: (np.arange(n) * (Lu - 1) + a) % nf
    for a in range(Lu):
        for b in range(Lu):
            for c in range(Lu):
                rho[np.ix_(idx(a), idx(b), idx(c))] += Mg[:, :, :, a, b, c]
    F_glob = float(np.sum(D * np.abs(np.fft.fftn(rho)) ** 2) / (2.0 * nf ** 3))
    P = Lu ** 3
    kv = np.array(np.unravel_index(np.arange(P), (Lu, Lu, Lu))).T
    Mf = Mg.reshape(n, n, n, P)
    E_corr = 0.0
    for d in range(27):
        dv = np.array([d // 9 - 1, (d // 3) % 3 - 1, d % 3 - 1])
        jj = kv[:, None, :] - kv[None, :, :] - dv * (Lu - 1)
        rr = dl * np.sqrt((jj ** 2).sum(axis=2))
        with np.errstate(divide="ignore", invalid="ignore"):
            C = np.where(np.abs(jj).max(axis=2) >= Lu - 1, erfc(xi * rr) / rr, 0.0)
        Ms = np.roll(Mf, shift=tuple(-dv), axis=(0, 1, 2))
        E_corr += -0.5 * float(np.einsum("xyzk,kl,xyzl->", Mf, C, Ms))
    return F_glob, E_corr


@pytest.mark.parametrize("nw,n,Lu", [(300, 5, 5), (300, 6, 4), (300, 5, 6)])
def test_merged_grid_and_correction_equal_the_literal_far_field(nw, n, Lu):
    b = synth.small_box(nw, 61, box=21.0)
    p = ar.Params(b.box, n, Lu, Lu)
    o = ar.ankh_energy(b.x, b.q, b.mu, b.theta, p, grad=False)
    F_glob, E_corr = merged_far_field(o["M"], b.box, n, Lu, p.xi)
    assert F_glob + E_corr == pytest.approx(o["E_far"], rel=1e-10, abs=1e-10 * abs(o["E"]))
    # the correction is not a small term (the factorisation is a real rewriting)
    assert abs(E_corr) > 1e-3 * abs(o["E_far"])
