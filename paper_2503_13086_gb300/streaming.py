"""Streaming session: each arriving image is integrated into the resident field.

Per arrival (Sec. IV-B and IV-C): ``gs_add_image`` extends the field with the image's new sparse
points and records the overlap relations, then ``gs_integrate`` runs the Local & Semi-Global
optimisation (Eq. 3-5 schedule, T_I view-iterations, Eq. 6-8 learning rate) in steps of
``batch_views`` views.  The new-image integration latency is the wall time from the arrival to
the end of its T_I iterations, field update included.
"""
from __future__ import annotations

import time

import numpy as np

from . import Field, _torch


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, np.float64), q)) if len(xs) else float("nan")


class StreamingSession:
    """One scene: a Field on its own CUDA stream, fed one image at a time."""

    def __init__(self, stream=None, prune_opacity=None, **config):
        """config: gs_field_config fields.  prune_opacity: after each arrival's iterations, remove the
        Gaussians whose opacity fell below it (3DGS's opacity pruning, gs_field_densify with no
        clone or split), as the load-balancing term of Eq. 10 intends for redundant Gaussians."""
        torch = _torch()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.field = Field(stream=self.stream, **config)
        self.prune_opacity = prune_opacity
        self.results = []

    def close(self):
        self.field.close()

    def arrive(self, cam, target, pts_xyz=None, pts_rgb=None, tracks=None, arrival_time=None):
        """Integrate one image; returns its record (latency, steps, loss, new Gaussians, pairs)."""
        t0 = time.perf_counter() if arrival_time is None else arrival_time
        ta = time.perf_counter()
        n0 = self.field.stats()["n_gaussians"]
        img = self.field.add_image(cam, target, pts_xyz, pts_rgb, tracks)
        n1 = self.field.stats()["n_gaussians"]
        tb = time.perf_counter()
        st = self.field.integrate(img) if n1 > 0 else dict(iterations=0, steps=0, key_images=0, mean_loss=0.0,
                                                              pairs=0)
        pruned = 0
        if self.prune_opacity is not None and n1 > 0:
            pruned = self.field.densify(grad_thresh=3.0e38, percent_dense=1.0, min_opacity=self.prune_opacity,
                                        max_scale=1.0e30)["pruned"]
        t1 = time.perf_counter()
        rec = dict(image_id=img, latency_s=t1 - t0, add_image_s=tb - ta, integrate_s=t1 - tb, new_gaussians=n1 - n0,
                   n_gaussians=n1 - pruned, pruned=pruned, **st)
        self.results.append(rec)
        return rec

    def latency(self):
        lat = [r["latency_s"] for r in self.results]
        return dict(p50=percentile(lat, 50), p99=percentile(lat, 99), n=len(lat))

    def psnr(self, cams, targets):
        """Mean PSNR of the field's renders against targets (device tensors or arrays)."""
        torch = _torch()
        vals = []
        with torch.cuda.stream(self.stream):
            for c, t in zip(cams, targets):
                img = self.field.render(c)
                tt = t if hasattr(t, "is_cuda") else torch.as_tensor(np.asarray(t), device="cuda")
                mse = torch.mean((img.clamp(0.0, 1.0) - tt) ** 2).item()
                vals.append(10.0 * np.log10(1.0 / max(mse, 1e-12)))
        return float(np.mean(vals))
