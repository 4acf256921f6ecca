"""Parity of the CUDA path (through the C ABI) with the oracle, kernel by kernel.

Bars: tile keys, sort order and per-tile ranges bit-exact (the oracle's binning is fed the
kernel's projected positions, radii and depths, so both decide from the same fp32 values);
pixels <= 1e-4 absolute; the projection's mean within 4 u of its rounding scale and the conic
within its conditioning; gradients elementwise within 1e-3 relative plus the rounding scale of
their products (tests/parity.py).  Per-pixel integers (last index, G_p, entries evaluated) are
exact except at recorded threshold ties: pixels where the oracle saw an alpha within 1e-5
(relative) of 1/255 or a transmittance within 1e-5 of 1e-4.  Every exemption is printed.
"""
import numpy as np
import pytest

import gsinputs as gi
import oracle
from helpers import config1, gpu_forward, grad_close, ocam, split_views
from parity import U32, Exemptions, backward_parity

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
        ex = Exemptions(f"{run['name']} view {v} projection")
        for i in np.nonzero((vis_g != vis_o) & border)[0]:
            ex.add(f"Gaussian {i}", f"visibility differs at a cull/rect threshold (margin {o['margin'][i]:.2e})")
        ex.report()
        assert (run["radius"][sl][both] == o["radius"][both]).all()
        # mean2d = f x/z + c: fp32 rounding of the camera transform (3-term dot products), the
        # division and the affine map, each side within 2 u of the scale below
        R = np.asarray(c["R"], np.float64).reshape(3, 3)
        t = np.asarray(c["t"], np.float64)
        mu = p[0:3, :n].astype(np.float64)
        pc = R @ mu + t[:, None]
        ax = np.abs(R) @ np.abs(mu) + np.abs(t)[:, None]
        for k, (f, cc) in enumerate(((c["fx"], c["cx"]), (c["fy"], c["cy"]))):
            uu = f * pc[k] / pc[2] + cc
            scale = f * (ax[k] + np.abs(pc[k] / pc[2]) * ax[2]) / np.abs(pc[2]) + np.abs(uu)
            err = np.abs(run["rec"]["mean2d"][sl][:, k].astype(np.float64) - o["mean2d"][:, k])
            assert (err[both] <= 4 * U32 * scale[both]).all(), (k, float((err / scale)[both].max() / U32))
        assert np.allclose(run["depth"][sl][both], o["depth"][both], rtol=1e-6)
        # the conic is the inverse of the 2D covariance: its fp32 error grows with the condition
        # number kappa of that 2 x 2 matrix; bound 64 u kappa |conic| (+1e-5 |conic|)
        co = o["conic"].astype(np.float64)
        tr = co[:, 0] + co[:, 2]
        disc = np.sqrt(np.maximum((co[:, 0] - co[:, 2]) ** 2 + 4 * co[:, 1] ** 2, 0))
        lmax, lmin = 0.5 * (tr + disc), np.maximum(0.5 * (tr - disc), 1e-30)
        nrm = np.abs(co).max(1)
        cb = (64 * U32 * lmax / lmin + 1e-5) * nrm
        cerr = np.abs(run["rec"]["conic"][sl].astype(np.float64) - co).max(1)
        assert (cerr[both] <= cb[both]).all(), float((cerr / cb)[both].max())
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
    ex = Exemptions(f"{run['name']} blend forward")
    for v, o in enumerate(outs):
        clean = o["margin"] > TIE
        ties += int((~clean).sum())
        for py, px in np.argwhere(~clean):
            ex.add(f"view {v} pixel ({py}, {px})", f"threshold tie (margin {o['margin'][py, px]:.1e})")
        assert np.abs(imgs[v] - o["image"])[:, clean].max() <= 1e-4
        assert np.abs(Ts[v] - o["T"])[clean].max() <= 1e-4
        assert np.array_equal(lasts[v][clean], o["last"][clean])
        assert np.array_equal(gps[v][clean], o["gp"][clean])
        pairs_ref += int(o["neval"].astype(np.int64).sum())
    ex.report()
    if ties == 0:
        assert out["pairs"] == pairs_ref
    else:
        assert abs(out["pairs"] - pairs_ref) <= 64 * ties


def test_forward_against_oracle_end_to_end(run):
    """The GPU's pixels against the oracle's whole forward (its own projection and binning).  A pixel
    may differ only where the oracle itself, walking the GPU's projected records instead of its own,
    takes another decision (blend set, stop) or sits at a threshold tie: there the projection's
    rounding decides the branch.  Each such pixel is printed; every other pixel is within 1e-4."""
    r = oracle.render(run["params"], [ocam(c) for c in run["cams"]], prec="f32", n=run["n"])
    L, outs_g = _oracle_forward_on_gpu_records(run)
    imgs = split_views(run["out"]["image"].cpu().numpy(), run["sizes"], 3)
    for v, o in enumerate(r["outs"]):
        og = outs_g[v]
        flip = (o["last"] != og["last"]) | (o["gp"] != og["gp"]) | (o["neval"] != og["neval"])
        tie = (o["margin"] <= TIE) | (og["margin"] <= TIE)
        d = np.abs(imgs[v] - o["image"]).max(0)
        ex = Exemptions(f"{run['name']} view {v} end-to-end forward")
        for py, px in np.argwhere((d > 1e-4) & (flip | tie)):
            ex.add(f"pixel ({py}, {px}) |d| {d[py, px]:.1e}",
                   "decision differs on the GPU's records" if flip[py, px] else "threshold tie")
        ex.report()
        bad = (d > 1e-4) & ~flip & ~tie
        assert not bad.any(), (run["name"], v, np.argwhere(bad)[:10].tolist(), float(d[bad].max()))


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
    # a fresh forward and dL/dimage so this test stands alone
    g = gpu_forward(ras, run["params"], run["n"], run["cams"])
    tg = np.concatenate([t.reshape(-1) for t in run["targets"]]).astype(np.float32)
    _, dimg = ras.loss(g["out"]["image"], torch.tensor(tg, device="cuda"), 0.2)
    backward_parity(run["name"], ras, g, run["params"], run["n"], run["cams"], dimg)


def test_backward_with_the_load_term(run, ras):
    """Eq. 9-10 with the paper's weight 0.41: the raster's loss adds lambda_load std(G_p) and the
    backward the load term's gradient through the soft count; both stages against the oracle on the
    same records, and the loss value against the oracle's."""
    import torch
    g = gpu_forward(ras, run["params"], run["n"], run["cams"])
    tg = np.concatenate([t.reshape(-1) for t in run["targets"]]).astype(np.float32)
    loss, dimg = ras.loss(g["out"]["image"], torch.tensor(tg, device="cuda"), 0.12, lambda_l1=0.47, lambda_load=0.41)
    L, outs = _oracle_forward_on_gpu_records(run)
    imgs = split_views(g["out"]["image"].cpu().numpy(), run["sizes"], 3)
    V = len(imgs)
    ref = 0.41 * oracle.load_term([o["gp"] for o in outs])
    for v in range(V):
        val, _, _, _ = oracle.loss(imgs[v], run["targets"][v], 0.12 / 0.59, False, 1.0, prec="f32")
        ref += 0.59 * val / V
    assert abs(loss - ref) <= 1e-5 * max(1.0, abs(ref)), (loss, ref)
    with_load, _ = backward_parity(run["name"] + " with L_load", ras, g, run["params"], run["n"], run["cams"], dimg,
                                   lambda_load=0.41)
    # the load term changes the gradient (it is not only in the reported loss); the loss and the
    # backward may run again on the same forward
    loss_wo, dimg2 = ras.loss(g["out"]["image"], torch.tensor(tg, device="cuda"), 0.12, lambda_l1=0.47,
                              lambda_load=0.0)
    ref_wo = ref - 0.41 * oracle.load_term([o["gp"] for o in outs])
    assert abs(loss_wo - ref_wo) <= 1e-5 * max(1.0, abs(ref_wo)), (loss_wo, ref_wo)
    without, _ = backward_parity(run["name"] + " without L_load", ras, g, run["params"], run["n"], run["cams"], dimg2)
    assert np.abs(with_load - without).max() > 0


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
