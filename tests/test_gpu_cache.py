"""Per-box table cache (ankh_create_cached): a handle whose tables (kernel
spectrum with its k = 0 value, correction blocks) are read from the cache
file gives bit-identical energies and gradients to one that computes them;
the file is keyed by everything the tables depend on."""
import os

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


def evaluate(api, b, **kw):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    m = api.Ankh(b.box, b.n, **kw)
    E, g = m.energy_forces(t(b.x), t(b.q), t(b.mu), t(b.theta), torques=True)
    info = m.info
    m.close()
    return E, {k: v.cpu().numpy() for k, v in g.items()}, info


@pytest.mark.parametrize("kw", [dict(n_cells=7, Lu=5, mixed=True), dict(n_cells=6, Lu=6, mixed=False),
                                dict(n_cells=5, Lu=5, nonperiodic=True)], ids=["mixed", "plain_Lu6", "nonperiodic"])
def test_cached_tables_give_identical_results(api, tmp_path, kw):
    b = synth.small_box(1000, 31, box=31.1)
    if kw.get("nonperiodic"):
        b.x = np.clip(b.x, -b.box / 2 + 1e-3, b.box / 2 - 1e-3).astype(np.float32)
    E0, g0, _ = evaluate(api, b, **kw)
    d = str(tmp_path)
    E1, g1, i1 = evaluate(api, b, cache_dir=d, **kw)      # computed, file written
    files = [f for f in os.listdir(d) if f.startswith("ankh_tables_")]
    assert len(files) == 1 and i1["tables_from_cache"] == 0
    E2, g2, i2 = evaluate(api, b, cache_dir=d, **kw)      # read from the file
    assert i2["tables_from_cache"] == 1
    assert E0 == E1 == E2
    for k in g0:
        assert np.array_equal(g0[k], g1[k]) and np.array_equal(g0[k], g2[k])
    # another key (xi) is another file -- except without images, where the
    # bare kernel ignores xi; a truncated file is recomputed
    npr = bool(kw.get("nonperiodic"))
    _, _, i3 = evaluate(api, b, cache_dir=d, xi=0.012, **kw)
    assert i3["tables_from_cache"] == (1 if npr else 0)
    assert len([f for f in os.listdir(d) if f.startswith("ankh_tables_")]) == (1 if npr else 2)
    path = os.path.join(d, files[0])
    with open(path, "r+b") as f:
        f.truncate(os.path.getsize(path) // 2)
    E4, g4, i4 = evaluate(api, b, cache_dir=d, **kw)
    assert i4["tables_from_cache"] == 0 and E4 == E0
    assert np.array_equal(g4["dEdx"], g0["dEdx"])
