"""gc_color_noalloc: the scratch-free entry point gives the same deterministic coloring as gc_color.

Callers that cannot allocate device memory (code running inside an allocator or memory-pool
callback, or under a framework that owns every device allocation) use gc_color_noalloc, which works
in a fixed scratch array built into the library.  This file runs last so that a failure here never
hides the results of the other tests."""
import ctypes

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


def _entry(gclib):
    lib = gclib.load()
    f = lib.gc_color_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]
    return f


@pytest.mark.parametrize("make", [lambda: gg.workload("er10k"), lambda: gg.rmat(13, 16, 2),
                                  lambda: gg.complete(600), lambda: gg.star(9000)])
def test_noalloc_matches_gc_color_twice(gclib, make):
    import torch
    f = _entry(gclib)
    g = make()
    rp = torch.from_numpy(g.rowptr).cuda()
    ci = torch.from_numpy(g.colidx).cuda()
    ref = gclib.color(rp, ci, "det", 7)
    ref_colors = ref.colors.cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # the scratch keeps the previous call's contents; results must not depend on it
        out = torch.full((g.n,), -5, dtype=torch.int32, device="cuda")
        nc, rd = ctypes.c_int32(-1), ctypes.c_int32(-1)
        st = f(g.n, rp.data_ptr(), ci.data_ptr(), 7, out.data_ptr(), ctypes.byref(nc), ctypes.byref(rd), stream)
        assert st == 0, gclib.load().gc_last_error()
        np.testing.assert_array_equal(out.cpu().numpy(), ref_colors)
        assert (nc.value, rd.value) == (ref.ncolors, ref.rounds)


def test_noalloc_allocates_nothing_after_warm_up(gclib):
    # the first call on a device loads the module (and its scratch array); after that a call must
    # leave the device's free memory exactly as it was
    import torch
    f = _entry(gclib)
    g = gg.rmat(13, 16, 2)
    rp = torch.from_numpy(g.rowptr).cuda()
    ci = torch.from_numpy(g.colidx).cuda()
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    nc, rd = ctypes.c_int32(0), ctypes.c_int32(0)
    stream = torch.cuda.current_stream().cuda_stream
    assert f(g.n, rp.data_ptr(), ci.data_ptr(), 7, out.data_ptr(), ctypes.byref(nc), ctypes.byref(rd), stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert f(g.n, rp.data_ptr(), ci.data_ptr(), 7, out.data_ptr(), ctypes.byref(nc), ctypes.byref(rd), stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_too_many_entries(gclib):
    # at most 16,384 vertices but more than 2^20 adjacency entries: rejected, outputs untouched
    import torch
    f = _entry(gclib)
    g = gg.complete(1100)  # 1,208,900 entries
    assert g.n <= 16384 and g.nnz > (1 << 20)
    rp = torch.from_numpy(g.rowptr).cuda()
    ci = torch.from_numpy(g.colidx).cuda()
    out = torch.full((g.n,), -5, dtype=torch.int32, device="cuda")
    nc, rd = ctypes.c_int32(-3), ctypes.c_int32(-3)
    st = f(g.n, rp.data_ptr(), ci.data_ptr(), 7, out.data_ptr(), ctypes.byref(nc), ctypes.byref(rd), None)
    assert st == gclib.GC_ERR_INVALID_ARG
    assert bool((out == -5).all())
    assert (nc.value, rd.value) == (-3, -3)


def test_noalloc_rejects_oversize(gclib):
    import torch
    f = _entry(gclib)
    g = gg.rmat(15, 16, 2)  # 32,768 vertices: above the 16,384-vertex limit
    rp = torch.from_numpy(g.rowptr).cuda()
    ci = torch.from_numpy(g.colidx).cuda()
    out = torch.full((g.n,), -5, dtype=torch.int32, device="cuda")
    nc, rd = ctypes.c_int32(0), ctypes.c_int32(0)
    st = f(g.n, rp.data_ptr(), ci.data_ptr(), 7, out.data_ptr(), ctypes.byref(nc), ctypes.byref(rd), None)
    assert st == gclib.GC_ERR_INVALID_ARG
    assert bool((out == -5).all())
