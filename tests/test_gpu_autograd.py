"""The hand-written backward behind torch.autograd: batched views at mixed sizes, gradients of a
64-Gaussian subset against central finite differences of the same CUDA forward, and agreement
with the oracle's gradient (bounds and exemptions: tests/parity.py)."""
import numpy as np
import pytest

import gsinputs as gi
from helpers import gpu_forward
from parity import backward_parity, fd_check

pytestmark = pytest.mark.gpu


def test_autograd_matches_finite_differences_and_oracle():
    import torch
    import paper_2503_13086_gb300 as gs
    from paper_2503_13086_gb300.autograd import rasterize
    n = 600
    p = gi.cube_scene(n, seed=11, stride=608, logscale=(-2.6, 0.3))
    cams = [gi.identity_camera(72, 56, 70.0), gi.identity_camera(48, 40, 45.0)]
    R, t = gi.look_at([0.4, -0.2, -0.3], [0.0, 0.0, 3.0])
    cams.append(gi.camera_dict(R, t, 60.0, 60.0, 30.0, 26.0, 61, 53))
    ras = gs.Raster()
    rng = np.random.default_rng(0)
    weights = torch.tensor(rng.normal(size=sum(3 * c["width"] * c["height"] for c in cams)).astype(np.float32),
                           device="cuda")
    P = torch.tensor(p, device="cuda", requires_grad=True)
    img = rasterize(P, n, cams, ras)
    loss = (img * weights).sum()
    loss.backward()
    g = P.grad.detach().cpu().numpy()

    # the same linear loss through the stateless raster: each backward stage against the oracle
    # on the same inputs (tests/parity.py), and the autograd result equal to it
    gg = gpu_forward(ras, p, n, cams)
    grads, _ = backward_parity("autograd three views", ras, gg, p, n, cams, weights)
    assert np.array_equal(g[:, :n], grads[:, :n])

    # central differences of the CUDA forward on a 64-Gaussian subset (tests/parity.py: fd_check)
    subset = rng.choice(n, 64, replace=False)
    fd_check("autograd three views", ras, P, n, cams, weights, g, subset, [0, 1, 2, 3, 6, 10, 11],
             min_discriminating=100)
    ras.close()
