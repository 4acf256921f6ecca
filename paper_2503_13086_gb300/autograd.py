"""torch.autograd wrapper of the CUDA rasterizer (the hand-written backward behind autograd).

``rasterize(params, n, cams, raster)`` renders the views (K1-K6) and returns their images packed
back to back (3 x H x W per view); calling ``backward`` on anything computed from them runs K8 + K9
through the C ABI.  The gradient flows to ``params`` (59 x stride, component-major).

A Raster keeps only its latest forward's workspace, so a graph built with one Raster must be
differentiated before that Raster renders again; this is checked and raises otherwise.
"""
from __future__ import annotations

import torch

from . import Raster


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, n, cams, raster, bg):
        out = raster.forward(params.detach(), n, cams, bg)
        ctx.save_for_backward(params, out["image"], out["last"])
        ctx.raster = raster
        ctx.generation = raster.generation
        ctx.mark_non_differentiable(out["last"])
        return out["image"], out["last"]

    @staticmethod
    def backward(ctx, dimage, _dlast):
        params, image, last = ctx.saved_tensors
        if ctx.raster.generation != ctx.generation:
            raise RuntimeError("the Raster rendered again before this backward; use one Raster per pending graph")
        grads, _ = ctx.raster.backward(params.detach(), image, last, dimage.contiguous())
        return grads, None, None, None, None


def rasterize(params: torch.Tensor, n: int, cams, raster: Raster, bg=(0.0, 0.0, 0.0)):
    """Differentiable render of ``cams``; returns the packed images (3 H W floats per view)."""
    image, _ = _Rasterize.apply(params, n, list(cams), raster, tuple(float(x) for x in bg))
    return image


def unpack(images: torch.Tensor, cams):
    """Split packed images into a list of (3, H, W) views."""
    out, off = [], 0
    for c in cams:
        w, h = int(c["width"]), int(c["height"])
        out.append(images[off:off + 3 * w * h].view(3, h, w))
        off += 3 * w * h
    return out
