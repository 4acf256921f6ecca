"""The batched local & semi-global workload at full size -- 500k Gaussians, the new view and 8
neighbours at mixed sizes from 960 x 540 to 1600 x 1060 -- differentiated through the
torch.autograd wrapper, against central finite differences of the same CUDA forward on a
64-Gaussian subset.

The loss is a seeded random linear functional of all nine images, so a perturbation changes it
only through the pixels the perturbed Gaussian reaches; the forward is deterministic, so every
other pixel cancels exactly in the difference.  Perturbations that change a discrete decision
anywhere (the set of Gaussians a pixel blends, or where it stops) are skipped and printed; every
other entry must agree within the per-entry bound of tests/parity.py (fd_check)."""
import numpy as np
import pytest

import gsinputs as gi
from parity import fd_check

pytestmark = pytest.mark.gpu


def test_batched_views_gradient_matches_finite_differences():
    import torch
    import paper_2503_13086_gb300 as gs
    from paper_2503_13086_gb300.autograd import rasterize
    n = 500_000
    p = gi.ring_scene(n, seed=5, stride=n)
    cams = gi.batched_views(9, seed=2)
    sizes = [(c["width"], c["height"]) for c in cams]
    assert len(set(sizes)) >= 3
    ras = gs.Raster()
    gen = torch.Generator(device="cuda").manual_seed(0)
    npix3 = sum(3 * w * h for w, h in sizes)
    weights = torch.randn(npix3, device="cuda", generator=gen, dtype=torch.float32)
    P = torch.tensor(p, device="cuda", requires_grad=True)
    img = rasterize(P, n, cams, ras)
    (img * weights).sum().backward()
    g = P.grad.detach().cpu().numpy()
    count = ras.read(6, np.uint32).reshape(len(cams), n)
    visible = np.nonzero((count > 0).any(0))[0]
    rng = np.random.default_rng(1)
    # 64 visible Gaussians with a gradient well above the noise of the opacity row
    op = np.abs(g[10, visible])
    cand = visible[op > 1e-2 * op.max()]
    subset = rng.choice(cand, 64, replace=False)
    fd_check("batched 9 views", ras, P, n, cams, weights, g, subset, [0, 1, 2, 3, 6, 10, 11], min_discriminating=90)
    ras.close()
