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
