"""gs_scan_noalloc: the tile-count scan for callers that cannot allocate device memory.

It must give exactly (integers: bit-exact) what the rasterizer's own scan gives inside
gs_raster_forward, on two calls in a row, so the scratch it shares between calls is cleared
correctly.  Collected last so a failure here stops a -x run only after every other test.
"""
import ctypes

import numpy as np
import pytest

import gsinputs as gi
from helpers import gpu_forward

pytestmark = pytest.mark.gpu


def test_scan_noalloc_matches_forward_scan():
    import torch

    import paper_2503_13086_gb300 as gs
    lib = gs.load()
    ras = gs.Raster()
    scenes = [(gi.cube_scene(5000, seed=3, stride=5024), 5000, [gi.identity_camera(300, 200, 260.0)]),
              (gi.cube_scene(1500, seed=4, stride=1504), 1500,
               [gi.identity_camera(96, 64, 90.0), gi.identity_camera(50, 41, 40.0)])]
    for p, n, cams in scenes:  # two calls in a row, the second one smaller
        g = gpu_forward(ras, p, n, cams)
        counts = g["count"]
        ref_offsets = g["offsets"]
        ref_total = len(g["keys"])
        assert ref_total > 0
        c_dev = torch.from_numpy(counts.view(np.int32).copy()).cuda()
        out = torch.full_like(c_dev, -1)
        total = torch.zeros(1, dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()
        st = lib.gs_scan_noalloc(ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(c_dev.data_ptr()),
                                 counts.shape[0], ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(total.data_ptr()))
        assert st == 0, lib.gs_last_error().decode()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref_offsets)
        assert int(total.item()) == ref_total
    ras.close()


def _scan(lib, counts_dev, n, out_dev, total_dev):
    import torch
    stream = torch.cuda.current_stream()
    return lib.gs_scan_noalloc(ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(counts_dev.data_ptr()), n,
                               ctypes.c_void_p(out_dev.data_ptr()),
                               ctypes.c_void_p(total_dev.data_ptr()) if total_dev is not None else None)


def test_scan_noalloc_against_cumsum_up_to_its_limit():
    """Hundreds to thousands of chained look-back tiles (2^20, 2^22 and the 2^24 limit, 2 048 counts
    per tile): the offsets equal numpy's exclusive cumulative sum bit for bit and the total its sum,
    on calls in a row (largest first, so a smaller call after it reuses scratch a larger one left);
    n = 0 gives a total of 0, and one count past the limit is refused on the host."""
    import torch
    import paper_2503_13086_gb300 as gs
    lib = gs.load()
    rng = np.random.default_rng(5)
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    for n in (1 << 24, 1 << 22, (1 << 20) + 777):
        counts = rng.integers(0, 16, size=n, dtype=np.uint32)
        ref = np.concatenate([[0], np.cumsum(counts, dtype=np.uint64)[:-1]]).astype(np.uint32)
        c_dev = torch.from_numpy(counts.view(np.int32)).cuda()
        out = torch.full_like(c_dev, -1)
        total.fill_(-5)
        assert _scan(lib, c_dev, n, out, total) == 0, lib.gs_last_error().decode()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref), n
        assert int(total.item()) == int(counts.sum(dtype=np.uint64)), n
        del c_dev, out
    empty = torch.zeros(4, dtype=torch.int32, device="cuda")
    total.fill_(-5)
    assert _scan(lib, empty, 0, empty, total) == 0
    torch.cuda.synchronize()
    assert int(total.item()) == 0
    assert _scan(lib, empty, (1 << 24) + 1, empty, total) == 4  # GS_ERR_CAPACITY
    assert b"n must be in" in lib.gs_last_error()
