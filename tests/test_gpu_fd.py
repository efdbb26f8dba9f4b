"""The library's analytic forces and torques against central finite
differences of the FP64 ANKH energy (the oracle's literal ANKH-FFT at the
same n, L_u, L_c, xi) on 32 atoms of the 96,000-atom water workload.

The stored differences (tests/golden/fd_water_96000_qmuTheta.json) come from
tests/golden/make_fd.py, which calls the oracle only: h_FD = 1e-4 A for
positions (atoms at least 10 h_FD from every leaf face, where the energy is
smooth), rigid rotations of mu and Theta by +-1e-4 rad for torques.  Their
own error is ~1e-8 relative (h^2 truncation, FP64 cancellation).

Bar: RMS error <= 1e-4 of the RMS value (the force target of the method);
the FP32 arithmetic of the GPU path gives ~1e-5.  Forces go through the
autograd wrapper (backward = the adjoint computed in the same call).
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_2212_08284_gb300 import synth   # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "fd_water_96000_qmuTheta.json")


@pytest.fixture(scope="module")
def api(gpu):
    from paper_2212_08284_gb300 import api as A, build
    build.build()
    A.load_library()
    return A


@pytest.fixture(scope="module")
def fd_case(api):
    import torch
    g = json.load(open(GOLD))
    b = synth.config_box(3)
    assert b.name == g["workload"]
    m = api.Ankh(b.box, b.n, xi=g["xi"], n_cells=g["n_cells"], Lu=g["Lu"], Lc=g["Lc"])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return g, b, m, t(b.x), t(b.q), t(b.mu), t(b.theta)


def rel_rms(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.sqrt(np.mean((got - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))


def test_forces_match_finite_differences(api, fd_case):
    g, b, m, x, q, mu, th = fd_case
    x = x.clone().requires_grad_(True)
    E = api.ankh_energy_autograd(m, x, q, mu, th)
    E.backward()
    got = x.grad[g["atoms"]].cpu().numpy()
    err = rel_rms(got, g["fd_dEdx"])
    assert err <= 1e-4, err
    # no single component far off either
    ref = np.asarray(g["fd_dEdx"])
    assert np.max(np.abs(got - ref)) <= 1e-3 * np.sqrt(np.mean(ref ** 2))


def test_torques_match_rotational_finite_differences(api, fd_case):
    g, b, m, x, q, mu, th = fd_case
    _, out = m.energy_forces(x, q, mu, th, torques=True)
    got = out["torque"][g["torque_atoms"]].cpu().numpy()
    err = rel_rms(got, g["fd_torque"])
    assert err <= 1e-4, err
