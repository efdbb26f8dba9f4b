"""The allocation-free binning/sort entry point gives exactly the result of
the allocating path.

ankh_bin_sort_noalloc serves callers that cannot call cudaMalloc (an engine
that plans all device memory at start-up, a host whose allocator belongs to
another runtime); its
scratch is a static device array of the library.  Binning and sorting are
integer work, so the comparison is bit-exact.  Two calls in a row check that
the shared static scratch is reset correctly between calls.  The cases cover
two random water boxes, coordinates on and next to leaf faces (where the
allocating path's FP32 screen hands over to the FP64 chain, which the
allocation-free path uses alone), every atom in one leaf, and half the atoms
in eight leaves.
"""
import ctypes

import numpy as np
import pytest

from cases import clustered_half_in_eight, clustered_one_leaf, face_box

pytestmark = pytest.mark.gpu


def test_no_alloc_bin_sort_matches_allocating_path(gpu):
    import torch

    from oracle import ankh_ref as ar
    from paper_2212_08284_gb300 import api, build, synth
    build.build()
    lib = api.load_library()
    dev = torch.device("cuda", 0)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    boxes = [(synth.small_box(4000, 77, box=49.4), 12), (synth.small_box(1500, 78, box=35.6), 7),
             face_box(False), clustered_one_leaf(), clustered_half_in_eight()]
    for b, n in boxes:
        f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        x, q = f32(b.x), f32(b.q)
        # the existing (allocating) entry point and its sort-stage outputs
        m = api.Ankh(b.box, b.n, n_cells=n, Lu=5, max_order=0)
        m.energy(x, q, None, None)
        ref_perm = api.ankh_debug_copy(m.h, api.BUF_PERM)
        ref_start = api.ankh_debug_copy(m.h, api.BUF_START)
        m.close()
        for _ in range(2):
            perm = torch.full((b.n,), -1, dtype=torch.int32, device=dev)
            start = torch.full((n ** 3 + 1,), -1, dtype=torch.int32, device=dev)
            rc = lib.ankh_bin_sort_noalloc(ptr(x), b.n, b.box, n, ptr(perm), ptr(start), stream)
            assert rc == api.ANKH_OK, lib.ankh_last_error().decode()
            torch.cuda.synchronize()
            assert torch.equal(perm, ref_perm)
            assert torch.equal(start, ref_start)
        # and both equal the FP64 leaf definition with the stable order
        cell, _, _, operm = ar.bin_atoms(b.x, b.box, n)
        assert np.array_equal(perm.cpu().numpy(), operm)

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
