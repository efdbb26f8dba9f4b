"""ankh_energy and ankh_energy_forces run the evaluation as a CUDA graph that
is captured at the first call and replayed while the call's pointers stay the
same: a replay reads the data the pointers hold at replay time, a new pointer
recaptures, the stage timing works through the graph's event nodes, and a
call made while the caller's stream is itself being captured runs the
kernels directly.  Every result is compared bit for bit with a fresh
handle's first (captured) call on the same data."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_2212_08284_gb300 import synth   # noqa: E402


@pytest.fixture(scope="module")
def api(gpu):
    from paper_2212_08284_gb300 import api as A, build
    build.build()
    A.load_library()
    return A


def dev(b):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return t(b.x), t(b.q), t(b.mu), t(b.theta)


def outputs(n):
    import torch
    return {"dEdx": torch.empty((n, 3), device="cuda"), "dEdq": torch.empty(n, device="cuda"),
            "dEdmu": torch.empty((n, 3), device="cuda"), "dEdtheta": torch.empty((n, 6), device="cuda"),
            "torque": torch.empty((n, 3), device="cuda")}


def fresh(api, b, x, q, mu, th):
    """The first call of a new handle on copies (new pointers: a capture)."""
    m = api.Ankh(b.box, b.n, n_cells=6, Lu=5)
    out = outputs(b.n)
    E = api.ankh_energy_forces(m.h, x.clone(), q.clone(), mu.clone(), th.clone(), **out)
    m.close()
    return E, out


def test_replay_reads_the_data_in_place(api):
    import torch
    b = synth.small_box(600, 21, box=26.0)
    x, q, mu, th = dev(b)
    m = api.Ankh(b.box, b.n, n_cells=6, Lu=5)
    out = outputs(b.n)
    api.ankh_energy_forces(m.h, x, q, mu, th, **out)            # capture
    # new positions and charges written into the same buffers: the replay reads them
    gen = torch.Generator(device="cuda").manual_seed(5)
    x.add_(0.05 * torch.randn(x.shape, device="cuda", generator=gen)).clamp_(-12.9, 12.9)
    q.mul_(1.1)
    E = api.ankh_energy_forces(m.h, x, q, mu, th, **out)        # replay
    E_ref, out_ref = fresh(api, b, x, q, mu, th)
    assert E == E_ref
    for k in out:
        assert torch.equal(out[k], out_ref[k])
    # a new output buffer recaptures; the energy-only variant has its own graph
    out2 = outputs(b.n)
    assert api.ankh_energy_forces(m.h, x, q, mu, th, **out2) == E
    for k in out:
        assert torch.equal(out2[k], out_ref[k])
    # energy alone (its own correction variant: the same energy to rounding)
    E1 = api.ankh_energy(m.h, x, q, mu, th)
    assert api.ankh_energy(m.h, x, q, mu, th) == E1
    assert E1 == pytest.approx(E, rel=1e-6)
    m.close()


def test_stage_times_through_the_graph(api):
    import torch
    b = synth.small_box(600, 22, box=26.0)
    x, q, mu, th = dev(b)
    m = api.Ankh(b.box, b.n, n_cells=6, Lu=5)
    out = outputs(b.n)
    E0 = api.ankh_energy_forces(m.h, x, q, mu, th, **out)
    api.ankh_set_timing(m.h, True)                              # recapture with the event nodes
    s = torch.cuda.current_stream()
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        E = api.ankh_energy_forces(m.h, x, q, mu, th, stream=s, **out)
        e1.record(s)
        e1.synchronize()
        st = api.ankh_stage_times(m.h)
        assert E == E0
        assert st["near"] > 0 and st["corr"] > 0 and st["l2p"] > 0
        assert sum(st.values()) <= e0.elapsed_time(e1) * 1.01
    api.ankh_set_timing(m.h, False)
    assert api.ankh_energy_forces(m.h, x, q, mu, th, **out) == E0
    m.close()


def test_call_inside_a_callers_capture(api):
    """The caller captures the call into its own graph: the library launches
    the kernels directly into that capture; replaying the caller's graph
    gives the same result."""
    import torch
    b = synth.small_box(600, 23, box=26.0)
    x, q, mu, th = dev(b)
    m = api.Ankh(b.box, b.n, n_cells=6, Lu=5)
    out = outputs(b.n)
    E0 = api.ankh_energy_forces(m.h, x, q, mu, th, **out)
    ref = {k: v.clone() for k, v in out.items()}
    for v in out.values():
        v.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        api.ankh_energy_forces(m.h, x, q, mu, th, stream=s, sync=False, **out)
    g.replay()
    torch.cuda.synchronize()
    for k in out:
        assert torch.equal(out[k], ref[k])
    m.close()


def test_stage_times_without_a_graph(api):
    """The host-buffer call launches the kernels directly (no graph): the
    stage events are plain records there, and the call still succeeds with
    timing on."""
    b = synth.small_box(600, 24, box=26.0)
    m = api.Ankh(b.box, b.n, n_cells=6, Lu=5)
    api.ankh_set_timing(m.h, True)
    host = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    outs = {k: np.zeros(s, np.float32) for k, s in (("dEdx", (b.n, 3)), ("dEdq", (b.n,)), ("dEdmu", (b.n, 3)),
                                                      ("dEdtheta", (b.n, 6)), ("torque", (b.n, 3)))}
    for _ in range(2):
        api.ankh_energy_forces_host(m.h, host(b.x), host(b.q), host(b.mu), host(b.theta), outs["dEdx"],
                                    outs["dEdq"], outs["dEdmu"], outs["dEdtheta"], outs["torque"])
        st = api.ankh_stage_times(m.h)
        assert st["near"] > 0 and st["l2p"] > 0
    api.ankh_set_timing(m.h, False)
    m.close()
