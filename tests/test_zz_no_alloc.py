"""The allocation-free binning/sort entry point gives exactly the result of
the allocating path.

ankh_bin_sort_noalloc serves callers that cannot call cudaMalloc (an engine
that plans all device memory at start-up, code running inside CUDA-graph
stream capture, a host whose allocator belongs to another runtime); its
scratch is a static device array of the library.  Binning and sorting are
integer work, so the comparison is bit-exact.  Two calls in a row check that
the shared static scratch is reset correctly between calls.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_no_alloc_bin_sort_matches_allocating_path(gpu):
    import torch

    from paper_2212_08284_gb300 import api, build, synth
    build.build()
    lib = api.load_library()
    dev = torch.device("cuda", 0)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    boxes = [(synth.small_box(4000, 77, box=49.4), 11), (synth.small_box(1500, 78, box=35.6), 7)]
    for b, n in boxes:
        f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        x, q, mu, th = f32(b.x), f32(b.q), f32(b.mu), f32(b.theta)
        # the existing (allocating) entry point and its sort-stage outputs
        m = api.Ankh(b.box, b.n, n_cells=n, Lu=5)
        m.energy(x, q, mu, th)
        ref_perm = api.ankh_debug_copy(m.h, api.BUF_PERM)
        ref_start = api.ankh_debug_copy(m.h, api.BUF_START)
        for _ in range(2):
            perm = torch.full((b.n,), -1, dtype=torch.int32, device=dev)
            start = torch.full((n ** 3 + 1,), -1, dtype=torch.int32, device=dev)
            rc = lib.ankh_bin_sort_noalloc(ptr(x), b.n, b.box, n, ptr(perm), ptr(start), stream)
            assert rc == api.ANKH_OK, lib.ankh_last_error().decode()
            torch.cuda.synchronize()
            assert torch.equal(perm, ref_perm)
            assert torch.equal(start, ref_start)
        m.close()

    # sizes beyond the static array are rejected with a clear error
    x = torch.zeros((8, 3), dtype=torch.float32, device=dev)
    perm = torch.zeros(8, dtype=torch.int32, device=dev)
    start = torch.zeros(65 ** 3 + 1, dtype=torch.int32, device=dev)
    rc = lib.ankh_bin_sort_noalloc(ptr(x), (1 << 20) + 1, 10.0, 4, ptr(perm), ptr(start), stream)
    assert rc == api.ANKH_EINVAL
    assert b"static scratch" in lib.ankh_last_error()
    rc = lib.ankh_bin_sort_noalloc(ptr(x), 8, 10.0, 65, ptr(perm), ptr(start), stream)
    assert rc == api.ANKH_EINVAL
    assert b"static scratch" in lib.ankh_last_error()
