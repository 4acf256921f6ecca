"""Every compiled tile shape and blend batch against the oracle run with the same tile shape, and
the autotuner of the session.

The tile shape is part of the result (the 3DGS rect rule bins by tile, and a Gaussian whose 1/255
footprint reaches past its 3-sigma square can enter or miss a pixel's list depending on the grid),
so each shape is compared with the oracle binning by the same shape: keys, order and ranges
bit-exact, pixels <= 1e-4 (ties printed), gradients within 1e-3 relative plus their rounding scale
(tests/parity.py).  The blend
batch only changes how many sorted Gaussians K6 stages per round: results are bitwise the same.
"""
import numpy as np
import pytest

import gsinputs as gi
import oracle
from helpers import gpu_forward, ocam, split_views
from parity import Exemptions, backward_parity

pytestmark = pytest.mark.gpu

TIE = 1e-5


def _candidates():
    import paper_2503_13086_gb300 as gs
    return gs.tiling_candidates()


def case_ragged():
    p = gi.cube_scene(3000, seed=5, stride=3008)
    cams = [gi.identity_camera(83, 61, 70.0), gi.identity_camera(50, 37, 45.0)]
    R, t = gi.look_at([0.5, -0.3, -0.5], [0.0, 0.0, 3.0])
    cams.append(gi.camera_dict(R, t, 60.0, 60.0, 40.0, 24.0, 79, 47))
    tg = [gi.uniform_target(c["width"], c["height"], 7 + k) for k, c in enumerate(cams)]
    return p, 3000, cams, tg


def case_dense():
    p = gi.cube_scene(2500, seed=8, stride=2528, half=0.15, logscale=(-3.5, 0.3))
    p[10, :2500] = -2.5
    return p, 2500, [gi.identity_camera(64, 48, 200.0)], [gi.uniform_target(64, 48, 3)]


def _run(ras, tl, case, check=False):
    """One forward, loss and backward with tiling tl; with check, the backward's two stages against
    the oracle run with the same tile shape (tests/parity.py)."""
    import torch
    p, n, cams, tg = case()
    ras.set_tiling(*tl)
    g = gpu_forward(ras, p, n, cams)
    sizes = [(c["width"], c["height"]) for c in cams]
    tgt = torch.tensor(np.concatenate([t.reshape(-1) for t in tg]).astype(np.float32), device="cuda")
    loss, dimg = ras.loss(g["out"]["image"], tgt, 0.2)
    if check:
        grads, grad2d = backward_parity(f"{case.__name__} {tl}", ras, g, p, n, cams, dimg, tile=(tl[0], tl[1]))
    else:
        grads, grad2d = ras.backward(g["P"], g["out"]["image"], g["out"]["last"], dimg, want_grad2d=True)
        grads, grad2d = grads.cpu().numpy(), grad2d.cpu().numpy().reshape(-1, 9)
    return dict(g=g, p=p, n=n, cams=cams, sizes=sizes, dimg=dimg.cpu().numpy(), loss=loss,
                grads=grads, grad2d=grad2d, image=g["out"]["image"].cpu().numpy())


@pytest.fixture(scope="module")
def ras():
    import paper_2503_13086_gb300 as gs
    r = gs.Raster()
    yield r
    r.close()


@pytest.mark.parametrize("case", [case_ragged, case_dense], ids=["ragged_multiview", "dense_tile"])
def test_every_tiling_matches_the_oracle(ras, case):
    for tl in _candidates():
        r = _run(ras, tl, case, check=True)  # the backward's stages are checked inside
        g, tile = r["g"], (tl[0], tl[1])
        # binning: bit-exact against the oracle's enumeration with the same tile shape
        L = oracle.build_lists(r["sizes"], g["rec"]["mean2d"], g["radius"], g["depth"], tile)
        assert np.array_equal(g["keys"], L["keys"]), tl
        assert np.array_equal(g["vals"], L["vals"]), tl
        assert np.array_equal(g["ranges"], L["ranges"]), tl
        # blending
        imgs = split_views(r["image"], r["sizes"], 3)
        lasts = split_views(g["out"]["last"].cpu().numpy().view(np.uint32), r["sizes"], 1)
        ex = Exemptions(f"{case.__name__} {tl} blend forward")
        for v, s in enumerate(r["sizes"]):
            o = oracle.blend_forward(s, L["tile_base"][v], L["ranges"], L["vals"], g["rec"], tile=tile, prec="f32")
            clean = o["margin"] > TIE
            for py, px in np.argwhere(~clean):
                ex.add(f"view {v} pixel ({py}, {px})", "threshold tie")
            assert np.abs(imgs[v] - o["image"])[:, clean].max() <= 1e-4, tl
            assert np.array_equal(lasts[v][clean], o["last"][clean]), tl
        ex.report()


def test_blend_batch_does_not_change_results(ras):
    by_shape = {}
    for tl in _candidates():
        by_shape.setdefault(tl[:2], []).append(tl)
    checked = 0
    for shape, tls in by_shape.items():
        if len(tls) < 2:
            continue
        ref = _run(ras, tls[0], case_dense)
        for tl in tls[1:]:
            r = _run(ras, tl, case_dense)
            assert np.array_equal(r["image"], ref["image"]), tl
            assert np.array_equal(r["grads"], ref["grads"]), tl
            assert r["loss"] == ref["loss"]
            checked += 1
    assert checked > 0


def test_unsupported_tiling_is_rejected(ras):
    import paper_2503_13086_gb300 as gs
    for bad in [(12, 12, 256), (16, 16, 100), (64, 64, 256), (0, 0, 0)]:
        with pytest.raises(gs.GSError):
            ras.set_tiling(*bad)
    with pytest.raises(gs.GSError):
        gs.Field(tiling=(12, 12, 256))


def _field_with_image(tiling):
    import paper_2503_13086_gb300 as gs
    p = gi.ring_scene(30000, seed=2, stride=30016)
    cams = [gi.ring_camera(0.3 + 0.1 * k, W=320, H=208, f=250.0) for k in range(3)]
    f = gs.Field(scene_extent=7.0, tiling=tiling)
    f.set_gaussians(p[:, :30000])
    ids = [f.add_image(c, gi.uniform_target(320, 208, 11 + k)) for k, c in enumerate(cams)]
    return f, ids, p, cams


def test_autotune_reports_every_candidate_and_leaves_the_field_unchanged():
    f, ids, _, _ = _field_with_image(None)
    before = f.get_gaussians(with_adam=True)
    res = f.autotune(ids, reps=2)
    cands = _candidates()
    assert [c for c, _ in res["candidates"]] == cands
    assert all(np.isfinite(ms) and ms > 0 for _, ms in res["candidates"])
    assert res["chosen"] == min(res["candidates"], key=lambda x: x[1])[0]
    after = f.get_gaussians(with_adam=True)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert f.stats()["adam_step"] == 0
    # the next step over a view set of that class runs the chosen tiling
    f.optimize_step(ids)
    assert f.stats()["last_tiling"] == res["chosen"]
    f.close()


def test_auto_tiled_step_equals_the_fixed_step_with_the_chosen_tiling():
    f, ids, _, _ = _field_with_image(None)
    losses = [f.optimize_step([ids[0]]) for _ in range(3)]  # the first step tunes this class
    chosen = f.stats()["last_tiling"]
    assert chosen in _candidates()
    got = f.get_gaussians(with_adam=True)
    f.close()
    g, ids2, _, _ = _field_with_image(chosen)
    ref_losses = [g.optimize_step([ids2[0]]) for _ in range(3)]
    ref = g.get_gaussians(with_adam=True)
    g.close()
    assert losses == ref_losses
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_field_step_matches_oracle_for_each_tile_shape():
    """One session step (forward, loss, backward, Adam) per compiled tile shape against the oracle's
    loss and gradient with that tile shape."""
    shapes = sorted({tl[:2] for tl in _candidates()})
    p = gi.cube_scene(4096, seed=4, stride=4096)
    cam = gi.identity_camera(200, 136, 200.0)
    tgt = gi.uniform_target(200, 136, 5)
    for tw, th in shapes:
        tl = next(t for t in _candidates() if t[:2] == (tw, th))
        import paper_2503_13086_gb300 as gs
        f = gs.Field(scene_extent=1.0, tiling=tl, use_graph=0)
        f.set_gaussians(p)
        img = f.add_image(cam, tgt)
        loss = f.optimize_step([img])
        L, _, _ = oracle.loss_and_grad(p, [ocam(cam)], [tgt], lam=0.2, tile=(tw, th), prec="f32")
        assert abs(loss - L) <= 1e-5 * max(1.0, abs(L)), (tl, loss, L)
        assert f.stats()["last_tiling"] == tl
        f.close()
