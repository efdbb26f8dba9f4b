"""The hand-written 3-D real FFT of the merged grid (mixed-radix Stockham in
shared memory, the spectral product fused into the pass along x) against
numpy's FP64 transforms, element by element, on even and odd grids whose
lengths use every radix the plans pick (15 = 5.3, 48 = 8.6, 196 = 7.7.4,
225 = 5.5.3.3 with the run-time plans; 216 = 6.6.6, 80 = 8.5.2,
72 = 8.3.3, 24 = 4.3.2, 40 = 5.4.2, 45 = 5.3.3, 70 = 7.5.2, 90 = 6.5.3 and
54 = 9.3.2 with the compile-time plans).

Bars (FP32 transforms of M = L^3 points, ~log2 M stages of one rounding
each): RMS error <= 2e-6 of the RMS value, every element within 2e-5 of the
RMS value; the energy term within 1e-6 of the sum of the magnitudes of
its terms, (1/2M) sum |D| |rho^|^2 (the test spectrum has both signs, so
the sum itself cancels).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api(gpu):
    from paper_2212_08284_gb300 import api as A, build
    build.build()
    A.load_library()
    return A


# (n, L_u): L = n (L_u - 1) = 15, 48, 196, 225 (run-time plans); 216, 80, 72, 24, 40, 45, 70, 90,
# 54 (compile-time plans; 54 = 9.3.2 with eight lines per block, as the 432-point plan)
SIZES = [(5, 4), (12, 5), (49, 5), (45, 6), (54, 5), (16, 6), (18, 5), (6, 5), (8, 6), (9, 6), (14, 6), (18, 6),
         (18, 4)]


def random_even_spectrum(rng, L):
    """Half spectrum [x][y][kz] of a real kernel even under z -> -z (real)."""
    g = rng.normal(size=(L, L, L))
    neg = lambda a: np.roll(a[::-1, ::-1, ::-1], 1, axis=(0, 1, 2))
    g = g + neg(g)
    return np.fft.rfftn(g).real


def close(got, ref, rms_bar=2e-6, max_bar=2e-5):
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    err = np.abs(got - ref)
    assert np.sqrt(np.mean(err ** 2)) <= rms_bar * rms
    assert np.max(err) <= max_bar * rms


@pytest.mark.parametrize("n,Lu", SIZES, ids=[f"L{n * (Lu - 1)}" for n, Lu in SIZES])
def test_fft_matches_numpy(api, n, Lu):
    import torch
    L = n * (Lu - 1)
    m = api.Ankh(4.0 * n, 8, n_cells=n, Lu=Lu, Lc=Lu, mixed=False)
    assert m.info["nf"] == L
    rng = np.random.default_rng(L)
    rho = rng.normal(size=(L, L, L)).astype(np.float32)
    D = random_even_spectrum(rng, L).astype(np.float32)
    rho_d = torch.from_numpy(rho).cuda()
    D_d = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    # forward transform
    spec = torch.empty((L, L, L // 2 + 1), dtype=torch.complex64, device="cuda")
    api.ankh_debug_fft(m.h, rho_d, None, 0, spec)
    ref = np.fft.rfftn(rho.astype(np.float64))
    close(spec.cpu().numpy().astype(np.complex128), ref)
    # far-field step: energy over the full spectrum and phi = ifft(D rho^) unnormalised
    phi = torch.empty((L, L, L), dtype=torch.float32, device="cuda")
    E = api.ankh_debug_fft(m.h, rho_d, D_d, 1, phi)
    M = L ** 3
    Dfull = np.fft.fftn(np.fft.irfftn(D.astype(np.float64), s=(L, L, L), axes=(0, 1, 2))).real
    rh = np.fft.fftn(rho.astype(np.float64))
    E_ref = np.sum(Dfull * np.abs(rh) ** 2) / (2.0 * M)
    scale = np.sum(np.abs(Dfull) * np.abs(rh) ** 2) / (2.0 * M)
    assert abs(E - E_ref) <= 1e-6 * scale
    phi_ref = np.fft.irfftn(D.astype(np.float64) * ref, s=(L, L, L), axes=(0, 1, 2)) * M
    close(phi.cpu().numpy().astype(np.float64), phi_ref)
    m.close()
