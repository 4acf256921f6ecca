"""The oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU restatement of the On-the-Fly GS hot path (the 3DGS rasterizer of Sec. III,
Eq. 1-2, its L1 + D-SSIM loss of Eq. 10, the analytic gradients and Adam) in ``gs_oracle.cpp``,
and of the progressive schedule (Eq. 3-8) in :mod:`oracle.schedule`.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this package.
It shares no code with the CUDA library and never imports it.

Arrays are numpy; parameters are component-major ``(59, stride)`` (see ``gs_oracle.cpp``).
``prec`` selects the instantiation: ``"f32"`` takes every threshold decision in fp32 (the
precision of the kernels), ``"f64"`` is for finite differences and closed forms.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libgs_oracle.so")
_lock = threading.Lock()
_lib = None

NPARAM = 59


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (plain IEEE arithmetic, no contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
        return _lib


P = ctypes.c_void_p
I32 = ctypes.c_int
I64 = ctypes.c_int64
F64 = ctypes.c_double


def _declare(L):
    for suf in ("f32", "f64"):
        getattr(L, f"orc_project_{suf}").argtypes = [P, I64, I64, P, I32, I32, I32, I32] + [P] * 9
        getattr(L, f"orc_blend_forward_{suf}").argtypes = [I32, I32, I32, I32, I64] + [P] * 12
        getattr(L, f"orc_blend_backward_{suf}").argtypes = [I32, I32, I32, I32, I64] + [P] * 10
        getattr(L, f"orc_blend_soft_count_{suf}").argtypes = [I32, I32, I32, I32, I64] + [P] * 7
        getattr(L, f"orc_blend_backward_magnitude_{suf}").argtypes = [I32, I32, I32, I32, I64] + [P] * 11
        getattr(L, f"orc_project_backward_{suf}").argtypes = [P, I64, I64, P, I32, I32, I32, I32, P, P]
        f = getattr(L, f"orc_loss_{suf}")
        f.argtypes = [I32, I32, P, P, F64, P, F64, P, P]
        f.restype = F64
        getattr(L, f"orc_adam_{suf}").argtypes = [P, P, P, P, I64, I64, P, F64, F64, F64, I64]
        getattr(L, f"orc_sh_eval_{suf}").argtypes = [P, I64, P]
    L.orc_project_backward_magnitude.argtypes = [P, I64, I64, P, I32, I32, I32, I32, P, P]
    L.orc_build_lists.argtypes = [I32, I64, P, P, I32, I32, P, P, P, I64, P, P, P]
    L.orc_build_lists.restype = I64


def _dt(prec):
    return np.float32 if prec == "f32" else np.float64


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Camera:
    """Pinhole view: world->camera R (3x3), t (3), focal lengths, principal point, size."""

    def __init__(self, R, t, fx, fy, cx, cy, width, height):
        self.R = np.asarray(R, dtype=np.float64).reshape(3, 3)
        self.t = np.asarray(t, dtype=np.float64).reshape(3)
        self.fx, self.fy, self.cx, self.cy = float(fx), float(fy), float(cx), float(cy)
        self.width, self.height = int(width), int(height)

    def packed(self):
        return np.concatenate([self.R.reshape(9), self.t, [self.fx, self.fy, self.cx, self.cy]]).astype(np.float64)

    def grid(self, tw=16, th=16):
        return (self.width + tw - 1) // tw, (self.height + th - 1) // th


def sh_eval(dirs, prec="f64"):
    dt = _dt(prec)
    d = _c(dirs, dt).reshape(-1, 3)
    out = np.zeros((d.shape[0], 16), dt)
    getattr(lib(), f"orc_sh_eval_{prec}")(_ptr(d), d.shape[0], _ptr(out))
    return out


def project(params, cam: Camera, tile=(16, 16), prec="f32", n=None):
    """Per-Gaussian projection (mean2d, depth, conic, opacity, rgb, radius, rect, clamp bits)."""
    dt = _dt(prec)
    params = _c(params, dt)
    stride = params.shape[1]
    n = stride if n is None else n
    out = dict(mean2d=np.zeros((n, 2), dt), depth=np.zeros(n, dt), conic=np.zeros((n, 3), dt),
               opacity=np.zeros(n, dt), rgb=np.zeros((n, 3), dt), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), clamp=np.zeros(n, np.uint8), margin=np.zeros(n, dt))
    camp = cam.packed()
    getattr(lib(), f"orc_project_{prec}")(
        _ptr(params), n, stride, _ptr(camp), cam.width, cam.height, tile[0], tile[1],
        _ptr(out["mean2d"]), _ptr(out["depth"]), _ptr(out["conic"]), _ptr(out["opacity"]),
        _ptr(out["rgb"]), _ptr(out["radius"]), _ptr(out["rect"]), _ptr(out["clamp"]), _ptr(out["margin"]))
    return out


def build_lists(sizes, mean2d, radius, depth, tile=(16, 16)):
    """Keys, record indices and per-tile ranges of all views in canonical order.

    ``sizes`` = [(W, H)] per view; ``mean2d`` (V*n, 2) fp32, ``radius`` (V*n,), ``depth`` (V*n,).
    Record index = view * n + Gaussian id; global tile = view tile base + ty * gx + tx.
    """
    V = len(sizes)
    mean2d = _c(mean2d, np.float32).reshape(-1, 2)
    radius = _c(radius, np.int32).reshape(-1)
    depth = _c(depth, np.float32).reshape(-1)
    n = radius.shape[0] // V
    Ws = np.array([s[0] for s in sizes], np.int32)
    Hs = np.array([s[1] for s in sizes], np.int32)
    tiles = [((w + tile[0] - 1) // tile[0]) * ((h + tile[1] - 1) // tile[1]) for w, h in sizes]
    ranges = np.zeros((sum(tiles), 2), np.uint32)
    L = lib()
    m = L.orc_build_lists(V, n, _ptr(Ws), _ptr(Hs), tile[0], tile[1], _ptr(mean2d), _ptr(radius),
                          _ptr(depth), 0, None, None, _ptr(ranges))
    keys = np.zeros(max(m, 1), np.uint64)
    vals = np.zeros(max(m, 1), np.uint32)
    L.orc_build_lists(V, n, _ptr(Ws), _ptr(Hs), tile[0], tile[1], _ptr(mean2d), _ptr(radius),
                      _ptr(depth), m, _ptr(keys), _ptr(vals), _ptr(ranges))
    base = np.concatenate([[0], np.cumsum(tiles)]).astype(np.int64)
    return dict(keys=keys[:m], vals=vals[:m], ranges=ranges, tile_base=base, n=n)


def blend_forward(cam_size, tile_base, ranges, vals, rec, bg=(0, 0, 0), tile=(16, 16), prec="f32"):
    """Eq. 2 per pixel.  ``rec`` holds mean2d/conic/opacity/rgb indexed by record index."""
    dt = _dt(prec)
    W, H = cam_size
    img = np.zeros((3, H, W), dt)
    T = np.zeros((H, W), dt)
    last = np.zeros((H, W), np.uint32)
    neval = np.zeros((H, W), np.uint32)
    gp = np.zeros((H, W), np.uint32)
    margin = np.zeros((H, W), dt)
    m2, co, op, rgb = (_c(rec[k], dt) for k in ("mean2d", "conic", "opacity", "rgb"))
    bgv = np.asarray(bg, dt)
    ranges = _c(ranges, np.uint32)
    vals = _c(vals, np.uint32) if len(vals) else np.zeros(1, np.uint32)
    getattr(lib(), f"orc_blend_forward_{prec}")(
        W, H, tile[0], tile[1], int(tile_base), _ptr(ranges), _ptr(vals), _ptr(m2), _ptr(co), _ptr(op),
        _ptr(rgb), _ptr(bgv), _ptr(img), _ptr(T), _ptr(last), _ptr(neval), _ptr(gp), _ptr(margin))
    return dict(image=img, T=T, last=last, neval=neval, gp=gp, margin=margin)


def blend_backward(cam_size, tile_base, ranges, vals, rec, dimg, grad2d, bg=(0, 0, 0), tile=(16, 16),
                   prec="f32", load_w=None):
    """Accumulate the per-record 2D gradients (9 per record) of one view into ``grad2d``.  load_w
    (H, W), optional: dL/dG_p per pixel of the load term (Eq. 9-10, see ``load_weights``)."""
    dt = _dt(prec)
    W, H = cam_size
    m2, co, op, rgb = (_c(rec[k], dt) for k in ("mean2d", "conic", "opacity", "rgb"))
    bgv = np.asarray(bg, dt)
    d = _c(dimg, dt)
    assert grad2d.dtype == dt and grad2d.flags.c_contiguous
    ranges = _c(ranges, np.uint32)
    vals = _c(vals, np.uint32) if len(vals) else np.zeros(1, np.uint32)
    lw = None if load_w is None else _c(load_w, dt)
    getattr(lib(), f"orc_blend_backward_{prec}")(
        W, H, tile[0], tile[1], int(tile_base), _ptr(ranges), _ptr(vals), _ptr(m2), _ptr(co), _ptr(op),
        _ptr(rgb), _ptr(bgv), _ptr(d), _ptr(lw), _ptr(grad2d))
    return grad2d


def blend_soft_count(cam_size, tile_base, ranges, vals, rec, tile=(16, 16), prec="f64"):
    """Per pixel, the soft count of Eq. 9's G_p: the sum of the alphas of its blended Gaussians."""
    dt = _dt(prec)
    W, H = cam_size
    m2, co, op, rgb = (_c(rec[k], dt) for k in ("mean2d", "conic", "opacity", "rgb"))
    out = np.zeros((H, W), dt)
    ranges = _c(ranges, np.uint32)
    vals = _c(vals, np.uint32) if len(vals) else np.zeros(1, np.uint32)
    getattr(lib(), f"orc_blend_soft_count_{prec}")(
        W, H, tile[0], tile[1], int(tile_base), _ptr(ranges), _ptr(vals), _ptr(m2), _ptr(co), _ptr(op),
        _ptr(rgb), _ptr(out))
    return out


def load_std(gps):
    """The spread of G_p over the pixels with G_p > 0 (the image's visible range), pooled over the
    views of a step (``gps``: per-view integer arrays): its population standard deviation."""
    g = np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in gps])
    g = g[g > 0]
    return float(np.std(g)) if g.size else 0.0


def load_term(gps):
    """Eq. 9's L_load: the population standard deviation of G_p over the pixels with G_p > 0 (the
    image's visible range), pooled over the views of a step; 0 without visible pixels."""
    return load_std(gps)


def load_weights(gps, lam):
    """dL/dG_p of lam x L_load per view (float64 arrays shaped like ``gps``): the derivative of the
    population standard deviation over the N pixels with G_p > 0, lam (G_p - mean) / (N std); zero
    at pixels with G_p = 0 and everywhere when std = 0."""
    g = np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in gps])
    vis = g > 0
    out = [np.zeros(np.shape(x), np.float64) for x in gps]
    if vis.sum() == 0:
        return out
    mean = g[vis].mean()
    std = np.sqrt(max(np.mean(g[vis] ** 2) - mean * mean, 0.0))
    if std == 0:
        return out
    for k, x in enumerate(gps):
        xv = np.asarray(x, np.float64)
        out[k] = np.where(xv > 0, lam * (xv - mean) / (vis.sum() * std), 0.0)
    return out


def blend_backward_magnitude(cam_size, tile_base, ranges, vals, rec, dimg, grad2d_mag, terms, bg=(0, 0, 0),
                             tile=(16, 16), prec="f32", load_w=None):
    """The rounding scale of blend_backward's sums: accumulates into ``grad2d_mag`` (9 per record) the
    sum of the magnitudes of every product that enters each 2D gradient, and into ``terms`` (uint32 per
    record) the number of (pixel, contributor) terms.  |fl(g) - g| <= gamma_k * grad2d_mag for k
    roundings in sequence (the componentwise bound of a floating-point sum)."""
    dt = _dt(prec)
    W, H = cam_size
    m2, co, op, rgb = (_c(rec[k], dt) for k in ("mean2d", "conic", "opacity", "rgb"))
    bgv = np.asarray(bg, dt)
    d = _c(dimg, dt)
    assert grad2d_mag.dtype == dt and grad2d_mag.flags.c_contiguous
    assert terms.dtype == np.uint32 and terms.flags.c_contiguous
    ranges = _c(ranges, np.uint32)
    vals = _c(vals, np.uint32) if len(vals) else np.zeros(1, np.uint32)
    lw = None if load_w is None else _c(load_w, dt)
    getattr(lib(), f"orc_blend_backward_magnitude_{prec}")(
        W, H, tile[0], tile[1], int(tile_base), _ptr(ranges), _ptr(vals), _ptr(m2), _ptr(co), _ptr(op),
        _ptr(rgb), _ptr(bgv), _ptr(d), _ptr(lw), _ptr(grad2d_mag), _ptr(terms))
    return grad2d_mag, terms


def project_backward(params, cam: Camera, grad2d, grads, tile=(16, 16), prec="f32", n=None):
    """Accumulate into ``grads`` (59, stride) the chain rule of one view's 2D gradients."""
    dt = _dt(prec)
    params = _c(params, dt)
    stride = params.shape[1]
    n = stride if n is None else n
    g2 = _c(grad2d, dt)
    assert grads.dtype == dt and grads.flags.c_contiguous and grads.shape == params.shape
    camp = cam.packed()
    getattr(lib(), f"orc_project_backward_{prec}")(
        _ptr(params), n, stride, _ptr(camp), cam.width, cam.height, tile[0], tile[1], _ptr(g2), _ptr(grads))
    return grads


def project_backward_magnitude(params, cam: Camera, grad2d, grads_mag, tile=(16, 16), n=None):
    """The rounding scale of project_backward's chain rule: accumulates into ``grads_mag`` (59, stride)
    float64 the sum of the magnitudes of the products that make up each parameter gradient (fp64
    evaluation of the same chain; see ``Mag`` in gs_oracle.cpp)."""
    params = _c(params, np.float64)
    stride = params.shape[1]
    n = stride if n is None else n
    g2 = _c(grad2d, np.float64)
    assert grads_mag.dtype == np.float64 and grads_mag.flags.c_contiguous and grads_mag.shape == params.shape
    camp = cam.packed()
    lib().orc_project_backward_magnitude(_ptr(params), n, stride, _ptr(camp), cam.width, cam.height, tile[0],
                                         tile[1], _ptr(g2), _ptr(grads_mag))
    return grads_mag


def loss(img, target, lam=0.2, want_grad=True, grad_scale=1.0, prec="f32"):
    """(loss, dL/dimg, l1, ssim) of L = (1-lam) L1 + lam (1 - SSIM) for one (3, H, W) view."""
    dt = _dt(prec)
    x = _c(img, dt)
    y = _c(target, dt)
    _, H, W = x.shape
    d = np.zeros_like(x) if want_grad else None
    l1 = ctypes.c_double()
    ss = ctypes.c_double()
    val = getattr(lib(), f"orc_loss_{prec}")(W, H, _ptr(x), _ptr(y), float(lam), _ptr(d), float(grad_scale),
                                           ctypes.byref(l1), ctypes.byref(ss))
    return val, d, l1.value, ss.value


def adam(params, grads, m, v, lrs, step, b1=0.9, b2=0.999, eps=1e-15, n=None, prec="f32"):
    """In-place Adam over the 59 component rows; ``lrs`` = 6 group learning rates."""
    dt = _dt(prec)
    for a in (params, grads, m, v):
        assert a.dtype == dt and a.flags.c_contiguous
    stride = params.shape[1]
    n = stride if n is None else n
    lr = np.asarray(lrs, np.float64)
    getattr(lib(), f"orc_adam_{prec}")(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), n, stride, _ptr(lr),
                                       b1, b2, eps, int(step))


def render(params, cams, tile=(16, 16), bg=(0, 0, 0), prec="f32", n=None):
    """K1-K6 for a batch of views.  Returns the per-view projections, the lists and the images."""
    dt = _dt(prec)
    params = _c(params, dt)
    n = params.shape[1] if n is None else n
    projs = [project(params, c, tile, prec, n=n) for c in cams]
    mean2d = np.concatenate([p["mean2d"] for p in projs]).astype(np.float32)
    radius = np.concatenate([p["radius"] for p in projs])
    depth = np.concatenate([p["depth"] for p in projs]).astype(np.float32)
    lists = build_lists([(c.width, c.height) for c in cams], mean2d, radius, depth, tile)
    rec = {k: np.concatenate([p[k] for p in projs]) for k in ("mean2d", "conic", "opacity", "rgb")}
    outs = [blend_forward((c.width, c.height), lists["tile_base"][v], lists["ranges"], lists["vals"], rec,
                          bg, tile, prec) for v, c in enumerate(cams)]
    return dict(projs=projs, lists=lists, rec=rec, outs=outs, n=n)


def loss_and_grad(params, cams, targets, lam=0.2, tile=(16, 16), bg=(0, 0, 0), prec="f32", n=None, lambda_l1=None,
                  lambda_load=0.0):
    """Batched step semantics: loss = mean over views of lambda_l1 L1 + lam D-SSIM (lambda_l1 defaults
    to 1 - lam), plus lambda_load L_load over all the views' pixels (Eq. 9-10); returns
    (loss, grads (59, stride), render)."""
    dt = _dt(prec)
    params = _c(params, dt)
    r = render(params, cams, tile, bg, prec, n)
    n = r["n"]
    V = len(cams)
    l1w = 1.0 - lam if lambda_l1 is None else lambda_l1
    grad2d = np.zeros((V * n, 9), dt)
    lws = load_weights([o["gp"] for o in r["outs"]], lambda_load) if lambda_load else [None] * V
    total = lambda_load * load_term([o["gp"] for o in r["outs"]]) if lambda_load else 0.0
    for v, c in enumerate(cams):
        # lambda_l1 L1 + lam D-SSIM = (lambda_l1 + lam) ((1 - lam') L1 + lam' D-SSIM), lam' = lam / (lambda_l1 + lam)
        wsum = l1w + lam
        lam_n = lam / wsum if wsum > 0 else 0.0
        val, d, _, _ = loss(r["outs"][v]["image"], targets[v], lam_n, True, wsum / V, prec)
        total += wsum * val / V
        blend_backward((c.width, c.height), r["lists"]["tile_base"][v], r["lists"]["ranges"], r["lists"]["vals"],
                       r["rec"], d, grad2d, bg, tile, prec, load_w=lws[v])
    grads = np.zeros_like(params)
    for v, c in enumerate(cams):
        project_backward(params, c, grad2d[v * n:(v + 1) * n], grads, tile, prec, n)
    r["grad2d"] = grad2d
    return total, grads, r


def pairs(r):
    """Gaussian-pixel pairs of one forward: per pixel, entries evaluated up to termination."""
    return int(sum(int(o["neval"].astype(np.int64).sum()) for o in r["outs"]))
