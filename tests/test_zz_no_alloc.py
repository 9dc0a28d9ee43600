"""The no-allocation entry point, tvs_total_viewshed_device_noalloc.

It serves callers that cannot allocate device memory themselves (a framework
whose caching allocator owns the GPU's memory budget, or a latency-bound loop
that must not pay the device-wide synchronisation of cudaMalloc/cudaFree).
Its scratch is one fixed 64 MiB device array shared by every call, so these
tests check that two calls in a row, through the C ABI, give what the
allocating entry point gives (up to the order of FP64 additions across
direction chunks, which the smaller scratch changes), and that a job too large
for the array is refused with an error instead of running.

This file is collected last on purpose: it also passes alone, in a fresh
process, where its first call resolves the array's address.
"""
import numpy as np
import pytest

import paper_2003_02200_gb300 as tvs
from paper_2003_02200_gb300 import terrain

pytestmark = pytest.mark.gpu

# Chunks of the no-allocation path are cut on 8-direction group boundaries
# when 8 directions fit its array, and the per-cell totals are exact sums of
# FP32 group sums: the result is then bit for bit the allocating path's.  A
# job whose 8 directions do not fit is cut inside groups, which moves results
# by FP32 rounding of the group sums only.
RTOL_INSIDE_GROUPS = 1e-6


def _reference(dem_t, step, h0, n, rng):
    import torch
    out = torch.empty_like(dem_t)
    with tvs.Context(0) as ctx:
        ctx.total_viewshed_device(dem_t, step, h0, n, rng, out=out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _noalloc(lib, dem_t, step, h0, n, rng):
    import torch
    out = torch.full_like(dem_t, -1.0)
    stream = torch.cuda.current_stream()
    rc = lib.tvs_total_viewshed_device_noalloc(dem_t.data_ptr(), dem_t.shape[0], dem_t.shape[1], step, h0, n,
                                               rng, out.data_ptr(), stream.cuda_stream)
    assert rc == 0, lib.tvs_last_error(None).decode()
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("rows,cols,n,rng,exact", [(300, 260, 96, 0.0, True), (640, 480, 45, 1500.0, False)])
def test_noalloc_matches_allocating_entry_point_twice(rows, cols, n, rng, exact):
    import torch
    lib = tvs.load()
    dem = terrain.fractal_dem(rows, cols, 0.8, 800.0, seed=rows + cols)
    d = torch.from_numpy(dem).cuda()
    want = _reference(d, 10.0, 1.5, n, rng)
    for _ in range(2):
        got = _noalloc(lib, d, 10.0, 1.5, n, rng)
        if exact:
            np.testing.assert_array_equal(got, want)
        else:
            np.testing.assert_allclose(got, want, rtol=RTOL_INSIDE_GROUPS, atol=0)


def test_noalloc_refuses_a_job_larger_than_its_array():
    import torch
    lib = tvs.load()
    d = torch.zeros(2000, 2000, device="cuda")
    out = torch.empty_like(d)
    rc = lib.tvs_total_viewshed_device_noalloc(d.data_ptr(), 2000, 2000, 10.0, 1.5, 180, 0.0, out.data_ptr(),
                                               torch.cuda.current_stream().cuda_stream)
    assert rc == tvs._binding.TVS_ERR_OOM
    assert b"64 MiB" in lib.tvs_last_error(None)


@pytest.mark.parametrize("rows,cols,n", [(2000, 100, 180), (2000, 100, 360), (100, 2000, 360), (128, 2048, 180)])
def test_noalloc_elongated_dems_stay_inside_the_array(rows, cols, n):
    """Elongated DEMs: the chunks with the most skewed rows and the chunk with
    the largest slab are different chunks, and the layout sized by both must
    still fit the array (the entry point checks the layout it really uses)."""
    import torch
    lib = tvs.load()
    dem = terrain.fractal_dem(rows, cols, 0.8, 600.0, seed=rows * 7 + cols)
    d = torch.from_numpy(dem).cuda()
    want = _reference(d, 10.0, 1.5, n, 0.0)
    for _ in range(2):
        got = _noalloc(lib, d, 10.0, 1.5, n, 0.0)
        np.testing.assert_allclose(got, want, rtol=RTOL_INSIDE_GROUPS, atol=0)


def test_noalloc_from_a_thread_with_a_small_stack():
    """A worker thread with a 256 KB stack, at the 1024-direction limit: the
    entry point keeps its planning tables off the caller's stack."""
    import threading
    import torch
    lib = tvs.load()
    dem = terrain.fractal_dem(48, 40, 0.8, 300.0, seed=11)
    d = torch.from_numpy(dem).cuda()
    want = _reference(d, 10.0, 1.5, 1024, 0.0)
    box = {}

    def work():
        try:
            torch.cuda.set_device(0)
            box["got"] = _noalloc(lib, d, 10.0, 1.5, 1024, 0.0)
        except BaseException as e:   # reported on the main thread
            box["err"] = e

    old = threading.stack_size(256 * 1024)
    try:
        t = threading.Thread(target=work)
        t.start()
        t.join()
    finally:
        threading.stack_size(old)
    assert "err" not in box, box.get("err")
    np.testing.assert_array_equal(box["got"], want)


def test_noalloc_refuses_stream_capture():
    import torch
    lib = tvs.load()
    d = torch.rand(32, 32, device="cuda")
    out = torch.empty_like(d)
    x = torch.zeros(4, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        x.add_(1.0)
        rc = lib.tvs_total_viewshed_device_noalloc(d.data_ptr(), 32, 32, 10.0, 1.5, 8, 0.0, out.data_ptr(),
                                                   s.cuda_stream)
        g.capture_end()
    torch.cuda.current_stream().wait_stream(s)
    assert rc == tvs._binding.TVS_ERR_ARG
    assert b"captured" in lib.tvs_last_error(None)
