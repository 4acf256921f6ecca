"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI binding and
convert its workspace buffers to the oracle's conventions."""
import numpy as np

import gsinputs as gi
import oracle
from oracle import Camera


def ocam(d):
    return Camera(d["R"], d["t"], d["fx"], d["fy"], d["cx"], d["cy"], d["width"], d["height"])


def gpu_forward(ras, params_np, n, cams, bg=(0.0, 0.0, 0.0)):
    import torch
    P = torch.tensor(params_np, device="cuda")
    out = ras.forward(P, n, cams, bg)
    torch.cuda.synchronize()
    V = len(cams)
    stride = params_np.shape[1]
    recs = V * stride
    xyo = ras.read(0, np.float32).reshape(recs, 4)
    con = ras.read(1, np.float32).reshape(recs, 4)
    rgb = ras.read(2, np.float32).reshape(recs, 4)
    rec = dict(mean2d=np.ascontiguousarray(xyo[:, :2]), opacity=np.ascontiguousarray(rgb[:, 3]),
               conic=np.ascontiguousarray(np.stack([-2 * con[:, 0], -con[:, 1], -2 * con[:, 2]], 1)),
               rgb=np.ascontiguousarray(rgb[:, :3]))
    radius = ras.read(4, np.int32)
    count = ras.read(6, np.uint32)
    radius = np.where(count > 0, radius, 0).astype(np.int32)
    depth = ras.read(3, np.float32)
    keys = ras.read(8, np.uint64)
    vals = ras.read(9, np.uint32)
    ranges = ras.read(10, np.uint32).reshape(-1, 2)
    offsets = ras.read(7, np.uint32)
    clamp = ras.read(11, np.uint8)
    return dict(P=P, out=out, rec=rec, radius=radius, count=count, depth=depth, keys=keys, vals=vals, ranges=ranges,
                offsets=offsets, clamp=clamp)


def split_views(flat, sizes, planes):
    res, off = [], 0
    for w, h in sizes:
        k = planes * w * h
        res.append(flat[off:off + k].reshape((planes, h, w) if planes > 1 else (h, w)))
        off += k
    return res


def grad_close(g, ref, rel=1e-3, floor=1e-2):
    """Elementwise |g - ref| <= rel * max(|ref|, floor * max|ref over the row|), per row."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    rowmax = np.abs(ref).max(axis=-1, keepdims=True)
    bound = rel * np.maximum(np.abs(ref), floor * rowmax) + 1e-30
    bad = np.abs(g - ref) > bound
    return bad


def config1(seed=0):
    p = gi.cube_scene(4096, seed=seed, stride=4096)
    cam = gi.identity_camera(256, 256, 256.0)
    tgt = gi.uniform_target(256, 256, seed + 100)
    return p, [cam], [tgt]
