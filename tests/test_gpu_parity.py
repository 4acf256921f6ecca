"""Parity of the CUDA path (through the C ABI) with the oracle, kernel by kernel.

Bars: tile keys, sort order and per-tile ranges bit-exact (the oracle's binning is fed the
kernel's projected positions, radii and depths, so both decide from the same fp32 values);
pixels <= 1e-4 absolute; gradients elementwise <= 1e-3 relative with a floor of 1 % of the
row's largest magnitude (float summation order differs).  Per-pixel integers (last index, G_p,
entries evaluated) are exact except at recorded threshold ties: pixels where the oracle saw an
alpha within 1e-5 (relative) of 1/255 or a transmittance within 1e-5 of 1e-4.
"""
import numpy as np
import pytest

import gsinputs as gi
import oracle
from helpers import config1, gpu_forward, grad_close, ocam, split_views

pytestmark = pytest.mark.gpu

TIE = 1e-5


@pytest.fixture(scope="module")
def ras():
    import paper_2503_13086_gb300 as gs
    r = gs.Raster()
    yield r
    r.close()


def case_config1():
    p, cams, tg = config1()
    return p, 4096, cams, tg


def case_ragged_multiview():
    p = gi.cube_scene(3000, seed=5, stride=3008)
    cams = [gi.identity_camera(83, 61, 70.0), gi.identity_camera(50, 37, 45.0)]
    R, t = gi.look_at([0.5, -0.3, -0.5], [0.0, 0.0, 3.0])
    cams.append(gi.camera_dict(R, t, 60.0, 60.0, 40.0, 24.0, 79, 47))
    tg = [gi.uniform_target(c["width"], c["height"], 7 + k) for k, c in enumerate(cams)]
    return p, 3000, cams, tg


def case_dense_tile():
    # thousands of faint Gaussians over a few tiles: lists of > 256 entries (several blend
    # batches, many backward chunks) and late termination
    p = gi.cube_scene(2500, seed=8, stride=2528, half=0.15, logscale=(-3.5, 0.3))
    p[10, :2500] = -2.5
    cams = [gi.identity_camera(64, 48, 200.0)]
    tg = [gi.uniform_target(64, 48, 3)]
    return p, 2500, cams, tg


CASES = {"config1": case_config1, "ragged_multiview": case_ragged_multiview, "dense_tile": case_dense_tile}


@pytest.fixture(scope="module", params=list(CASES))
def run(request, ras):
    p, n, cams, tg = CASES[request.param]()
    g = gpu_forward(ras, p, n, cams)
    g["params"] = p
    g["n"] = n
    g["cams"] = cams
    g["targets"] = tg
    g["sizes"] = [(c["width"], c["height"]) for c in cams]
    g["name"] = request.param
    return g


def test_projection(run):
    p, n, cams = run["params"], run["n"], run["cams"]
    stride = p.shape[1]
    for v, c in enumerate(cams):
        o = oracle.project(p, ocam(c), prec="f32", n=n)
        sl = slice(v * stride, v * stride + n)
        vis_g = run["count"][sl] > 0
        vis_o = o["radius"] > 0
        border = o["margin"] < 1e-3
        assert ((vis_g == vis_o) | border).all()
        both = vis_g & vis_o & ~border
        assert both.sum() > 0
        assert (run["radius"][sl][both] == o["radius"][both]).all()
        assert np.allclose(run["rec"]["mean2d"][sl][both], o["mean2d"][both], rtol=1e-5, atol=1e-3)
        assert np.allclose(run["depth"][sl][both], o["depth"][both], rtol=1e-6)
        assert np.allclose(run["rec"]["conic"][sl][both], o["conic"][both], rtol=1e-4, atol=1e-6)
        assert np.allclose(run["rec"]["opacity"][sl][both], o["opacity"][both], rtol=1e-6, atol=1e-7)
        assert np.allclose(run["rec"]["rgb"][sl][both], o["rgb"][both], atol=1e-5)
        assert (run["clamp"][sl][both] == o["clamp"][both]).all()


def test_binning_bit_exact(run):
    L = oracle.build_lists(run["sizes"], run["rec"]["mean2d"], run["radius"], run["depth"])
    assert len(run["keys"]) == len(L["keys"])
    assert np.array_equal(run["keys"], L["keys"])
    assert np.array_equal(run["vals"], L["vals"])
    assert np.array_equal(run["ranges"], L["ranges"])
    cnt = run["count"].astype(np.int64)
    assert np.array_equal(run["offsets"].astype(np.int64), np.concatenate([[0], np.cumsum(cnt)[:-1]]))
    run["lists"] = L


def _oracle_forward_on_gpu_records(run):
    L = oracle.build_lists(run["sizes"], run["rec"]["mean2d"], run["radius"], run["depth"])
    outs = [oracle.blend_forward(s, L["tile_base"][v], L["ranges"], L["vals"], run["rec"], prec="f32")
            for v, s in enumerate(run["sizes"])]
    return L, outs


def test_blend_forward(run):
    L, outs = _oracle_forward_on_gpu_records(run)
    out = run["out"]
    imgs = split_views(out["image"].cpu().numpy(), run["sizes"], 3)
    Ts = split_views(out["T"].cpu().numpy(), run["sizes"], 1)
    lasts = split_views(out["last"].cpu().numpy().view(np.uint32), run["sizes"], 1)
    gps = split_views(out["gp"].cpu().numpy().view(np.uint32), run["sizes"], 1)
    pairs_ref = 0
    ties = 0
    for v, o in enumerate(outs):
        clean = o["margin"] > TIE
        ties += int((~clean).sum())
        assert np.abs(imgs[v] - o["image"])[:, clean].max() <= 1e-4
        assert np.abs(Ts[v] - o["T"])[clean].max() <= 1e-4
        assert np.array_equal(lasts[v][clean], o["last"][clean])
        assert np.array_equal(gps[v][clean], o["gp"][clean])
        pairs_ref += int(o["neval"].astype(np.int64).sum())
    if ties == 0:
        assert out["pairs"] == pairs_ref
    else:
        assert abs(out["pairs"] - pairs_ref) <= 64 * ties


def test_forward_against_oracle_end_to_end(run):
    r = oracle.render(run["params"], [ocam(c) for c in run["cams"]], prec="f32", n=run["n"])
    imgs = split_views(run["out"]["image"].cpu().numpy(), run["sizes"], 3)
    for v, o in enumerate(r["outs"]):
        d = np.abs(imgs[v] - o["image"]).max(0)
        good = (d <= 1e-4) | (o["margin"] <= TIE)
        assert good.mean() >= 0.999, (run["name"], v, good.mean(), d.max())


def test_loss(run, ras):
    import torch
    out = run["out"]
    tg = np.concatenate([t.reshape(-1) for t in run["targets"]]).astype(np.float32)
    T = torch.tensor(tg, device="cuda")
    loss, dimg = ras.loss(out["image"], T, 0.2)
    imgs = split_views(out["image"].cpu().numpy(), run["sizes"], 3)
    ds = split_views(dimg.cpu().numpy(), run["sizes"], 3)
    V = len(imgs)
    ref = 0.0
    for v in range(V):
        val, d, _, _ = oracle.loss(imgs[v], run["targets"][v], 0.2, True, 1.0 / V, prec="f32")
        ref += val / V
        bad = grad_close(ds[v].reshape(1, -1), d.reshape(1, -1), rel=1e-3, floor=1e-2)
        assert not bad.any(), (v, np.abs(ds[v] - d).max(), np.abs(d).max())
    assert abs(loss - ref) <= 1e-5 * max(1.0, abs(ref))
    run["dimage"] = dimg


def test_backward(run, ras):
    import torch
    out = run["out"]
    if "dimage" not in run:
        tg = np.concatenate([t.reshape(-1) for t in run["targets"]]).astype(np.float32)
        ras.loss(out["image"], torch.tensor(tg, device="cuda"), 0.2)
    # re-run the forward so this test stands alone, then take a fresh dL/dimage
    g = gpu_forward(ras, run["params"], run["n"], run["cams"])
    tg = np.concatenate([t.reshape(-1) for t in run["targets"]]).astype(np.float32)
    _, dimg = ras.loss(g["out"]["image"], torch.tensor(tg, device="cuda"), 0.2)
    grads, grad2d = ras.backward(g["P"], g["out"]["image"], g["out"]["last"], dimg, want_grad2d=True)
    grads = grads.cpu().numpy()
    grad2d = grad2d.cpu().numpy().reshape(-1, 9)
    n, stride = run["n"], run["params"].shape[1]
    L = oracle.build_lists(run["sizes"], g["rec"]["mean2d"], g["radius"], g["depth"])
    ds = split_views(dimg.cpu().numpy(), run["sizes"], 3)
    g2_ref = np.zeros((len(run["sizes"]) * stride, 9), np.float32)
    for v, s in enumerate(run["sizes"]):
        oracle.blend_backward(s, L["tile_base"][v], L["ranges"], L["vals"], g["rec"], ds[v], g2_ref, prec="f32")
    vis = g["count"] > 0
    bad2 = grad_close(grad2d[vis].T, g2_ref[vis].T)
    assert bad2.mean() < 1e-3, (run["name"], bad2.sum(axis=1))
    g_ref = np.zeros_like(run["params"])
    for v, c in enumerate(run["cams"]):
        oracle.project_backward(run["params"], ocam(c), g2_ref[v * stride:(v + 1) * stride], g_ref, prec="f32", n=n)
    bad = grad_close(grads[:, :n], g_ref[:, :n])
    assert bad.mean() < 1e-3, (run["name"], bad.sum(axis=1))


def test_adam_kernel():
    import torch
    import paper_2503_13086_gb300 as gs
    rng = np.random.default_rng(1)
    n, stride = 1000, 1024
    p = rng.normal(size=(59, stride)).astype(np.float32)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    lrs = [8e-4, 5e-3, 1e-3, 0.05, 2.5e-3, 1.25e-4]
    P, Mt, Vt = (torch.tensor(a, device="cuda") for a in (p, m, v))
    for step in (1, 2, 3):
        gr = rng.normal(size=(59, stride)).astype(np.float32)
        gs.adam_step(P, torch.tensor(gr, device="cuda"), Mt, Vt, n, lrs, step)
        oracle.adam(p, gr, m, v, lrs, step, n=n, prec="f32")
    torch.cuda.synchronize()
    assert np.allclose(P.cpu().numpy()[:, :n], p[:, :n], rtol=1e-5, atol=1e-6)
    assert np.allclose(Mt.cpu().numpy()[:, :n], m[:, :n], rtol=1e-5, atol=1e-7)
    # rows beyond n are untouched
    assert np.array_equal(P.cpu().numpy()[:, n:], p[:, n:])


def test_backward_is_deterministic(ras):
    import torch
    p, cams, tg = config1(seed=3)
    T = torch.tensor(tg[0].reshape(-1), device="cuda")
    res = []
    for _ in range(2):
        g = gpu_forward(ras, p, 4096, cams)
        _, d = ras.loss(g["out"]["image"], T, 0.2)
        gr, _ = ras.backward(g["P"], g["out"]["image"], g["out"]["last"], d)
        res.append(gr.cpu().numpy())
    assert np.array_equal(res[0], res[1])


def test_empty_and_fully_culled(ras):
    import torch
    for kind in ("empty", "behind"):
        p = gi.cube_scene(64, seed=2, stride=64)
        n = 0 if kind == "empty" else 64
        if kind == "behind":
            p[2, :] = -3.0
        cams = [gi.identity_camera(40, 24, 40.0)]
        g = gpu_forward(ras, p, n, cams, bg=(0.25, 0.5, 0.75))
        img = g["out"]["image"].cpu().numpy().reshape(3, 24, 40)
        for ch, b in enumerate((0.25, 0.5, 0.75)):
            assert np.all(img[ch] == b)
        assert g["out"]["pairs"] == 0 and len(g["keys"]) == 0
        tg = torch.rand(3 * 24 * 40, device="cuda")
        _, d = ras.loss(g["out"]["image"], tg, 0.2)
        gr, _ = ras.backward(g["P"], g["out"]["image"], g["out"]["last"], d)
        assert float(gr.abs().max()) == 0.0
