"""3DGS adaptive density control through the C ABI (kept among the 3DGS settings, Sec. V-A):
the per-step view-space gradient statistics against oracle.densify on the step's own 2D gradients, and
clone / split / prune against oracle.densify on the same float32 state."""
import numpy as np
import pytest

import gsinputs as gi
import oracle
from helpers import gpu_forward
from parity import backward_parity
from oracle import densify as od

pytestmark = pytest.mark.gpu


def make_field(**kw):
    import paper_2503_13086_gb300 as gs
    kw.setdefault("scene_extent", 1.0)
    kw.setdefault("tiling", (16, 16, 256))
    kw.setdefault("densify_stats", 1)
    kw.setdefault("use_graph", 0)
    return gs.Field(**kw)


def scene3(n=3000, seed=12):
    p = gi.cube_scene(n, seed=seed, stride=n)
    cams = [gi.identity_camera(96, 64, 90.0), gi.identity_camera(70, 52, 60.0)]
    R, t = gi.look_at([0.4, -0.3, -0.4], [0.0, 0.0, 3.0])
    cams.append(gi.camera_dict(R, t, 70.0, 70.0, 40.0, 30.0, 81, 61))
    tg = [gi.uniform_target(c["width"], c["height"], 20 + k) for k, c in enumerate(cams)]
    return p, cams, tg


def oracle_stats(p, cams, tg, n):
    """Norm sums and counts of one step over `cams`, computed by oracle.densify from the step's own 2D
    gradients (the raster's, each stage of which is checked against the oracle on the same inputs)."""
    import torch
    import paper_2503_13086_gb300 as gs
    stride = -(-n // 32) * 32  # the raster takes a row stride that is a multiple of 32
    pp = np.zeros((59, stride), np.float32)
    pp[:, :n] = p[:, :n]
    p = pp
    ras = gs.Raster()
    ras.set_tiling(16, 16, 256)
    g = gpu_forward(ras, p, n, cams)
    tgt = np.concatenate([t.reshape(-1) for t in tg]).astype(np.float32)
    _, dimg = ras.loss(g["out"]["image"], torch.tensor(tgt, device="cuda"), 0.2)
    _, g2 = backward_parity("densify statistics step", ras, g, p, n, cams, dimg)
    ras.close()
    acc = np.zeros(n, np.float32)
    cnt = np.zeros(n, np.float32)
    for v, c in enumerate(cams):
        has = g["count"][v * stride:v * stride + n] > 0
        nv = od.view_space_norm(g2[v * stride:v * stride + n, 0], g2[v * stride:v * stride + n, 1], c["width"],
                                c["height"])
        acc[has] += nv[has]
        cnt[has] += 1
    return acc, cnt


def test_statistics_of_one_step_match_the_oracle():
    p, cams, tg = scene3()
    n = p.shape[1]
    f = make_field()
    f.set_gaussians(p)
    ids = [f.add_image(c, t) for c, t in zip(cams, tg)]
    a0, c0 = f.densify_stats()
    assert not a0.any() and not c0.any()
    f.optimize_step(ids)
    acc, cnt = f.densify_stats()
    ref_acc, ref_cnt = oracle_stats(p, cams, tg, n)
    assert np.array_equal(cnt, ref_cnt)
    assert (ref_cnt > 0).sum() > n // 2
    # a norm (4 roundings) per view, summed over up to three views
    assert (np.abs(acc - ref_acc) <= 16 * 2.0 ** -24 * ref_acc + 1e-30).all(), float(np.abs(acc - ref_acc).max())
    f.close()


def test_statistics_off_by_default_and_accumulate_over_steps():
    p, cams, tg = scene3()
    f = make_field(densify_stats=0)
    f.set_gaussians(p)
    ids = [f.add_image(c, t) for c, t in zip(cams, tg)]
    f.optimize_step(ids)
    a, c = f.densify_stats()
    assert not a.any() and not c.any()
    f.close()
    f = make_field()
    f.set_gaussians(p)
    ids = [f.add_image(c, t) for c, t in zip(cams, tg)]
    for k in range(3):
        f.optimize_step([ids[k]])
    _, c = f.densify_stats()
    # each single-view step adds 1 to every Gaussian with instances in that view
    assert c.max() <= 3 and (c == 3).sum() > 0
    f.close()


def run_densify(seed=7, steps=2, **over):
    p, cams, tg = scene3(seed=seed)
    f = make_field(seed=seed)
    f.set_gaussians(p)
    ids = [f.add_image(c, t) for c, t in zip(cams, tg)]
    for _ in range(steps):
        f.optimize_step(ids)
    P, M, V = f.get_gaussians(with_adam=True)
    acc, cnt = f.densify_stats()
    n = P.shape[1]
    g = np.where(cnt > 0, acc / np.maximum(cnt, 1), 0).astype(np.float32)
    maxls = P[3:6].max(0)
    opac = 1.0 / (1.0 + np.exp(-P[10].astype(np.float64)))
    # thresholds from the state so that every branch is taken by many Gaussians
    kw = dict(grad_thresh=float(np.quantile(g[g > 0], 0.6)), percent_dense=float(np.exp(np.median(maxls))),
              min_opacity=float(np.quantile(opac, 0.08)), max_scale=float(np.exp(np.quantile(maxls, 0.93))))
    kw.update(over)
    res = f.densify(**kw)
    P2, M2, V2 = f.get_gaussians(with_adam=True)
    RP, RM, RV, info = od.densify(P, M, V, n, acc, cnt, 1.0, seed=seed, rnd=0, **kw)
    return f, (P2, M2, V2, res), (RP, RM, RV, info), n, ids


def test_densify_matches_the_oracle():
    f, (P2, M2, V2, res), (RP, RM, RV, info), n, ids = run_densify()
    assert res["n_before"] == n
    assert res["n_after"] == info["n"] == P2.shape[1]
    assert res["cloned"] == info["cloned"] and res["split"] == info["split"] and res["pruned"] == info["pruned"]
    assert info["cloned"] > 50 and info["split"] > 50 and info["pruned"] > 50
    # moments: kept originals copied, new ones zero -- exact
    assert np.array_equal(M2, RM) and np.array_equal(V2, RV)
    nk = info["kept"]
    nc = info["cloned"]
    # kept originals and clones are copies; children: everything but the mean is exact
    assert np.array_equal(P2[:, :nk + nc], RP[:, :nk + nc])
    assert np.array_equal(P2[3:, nk + nc:], RP[3:, nk + nc:])
    d = np.abs(P2[:3, nk + nc:] - RP[:3, nk + nc:])
    scale = np.exp(RP[3:6, nk + nc:].astype(np.float64) + float(np.log(1.6))).max(0)
    assert (d <= 1e-5 * (1.0 + np.abs(RP[:3, nk + nc:])) + 1e-5 * scale).all()
    # the statistics start over and the session goes on at the new size
    a, c = f.densify_stats()
    assert a.shape == (P2.shape[1],) and not a.any() and not c.any()
    loss = f.optimize_step(ids)
    assert np.isfinite(loss)
    assert f.stats()["n_gaussians"] == P2.shape[1]
    f.close()


def test_densify_with_the_3dgs_settings_and_without_statistics():
    """Default settings: nothing reaches the gradient threshold without statistics, so only the
    opacity / size prune acts."""
    p, cams, tg = scene3(seed=9)
    p = p.copy()
    p[10, ::17] = -8.0  # sigmoid < 0.005: pruned
    f = make_field(densify_stats=0, seed=9)
    f.set_gaussians(p)
    P, M, V = f.get_gaussians(with_adam=True)
    res = f.densify()
    RP, RM, RV, info = od.densify(P, M, V, P.shape[1], np.zeros(P.shape[1], np.float32),
                                  np.zeros(P.shape[1], np.float32), 1.0, seed=9)
    assert res["cloned"] == 0 and res["split"] == 0
    assert res["pruned"] == info["pruned"] >= len(range(0, p.shape[1], 17))
    assert np.array_equal(f.get_gaussians(), RP)
    f.close()


def test_graph_session_densifies_and_replays():
    """With graph capture on, a densification drops the captured steps; the next ones are
    captured again at the new size and equal eager launches bit for bit."""
    res = []
    for use_graph in (1, 0):
        p, cams, tg = scene3(seed=5)
        f = make_field(use_graph=use_graph, seed=5)
        f.set_gaussians(p)
        ids = [f.add_image(c, t) for c, t in zip(cams, tg)]
        for _ in range(3):
            f.optimize_step(ids)
        f.densify(grad_thresh=1e-7, percent_dense=0.02, min_opacity=0.01, max_scale=0.5)
        losses = [f.optimize_step(ids) for _ in range(3)]
        res.append((losses, f.get_gaussians(with_adam=True)))
        f.close()
    assert res[0][0] == res[1][0]
    for a, b in zip(res[0][1], res[1][1]):
        assert np.array_equal(a, b)


def test_checkpoint_keeps_statistics_and_the_split_round(tmp_path):
    import paper_2503_13086_gb300 as gs
    p, cams, tg = scene3(seed=6)
    f = make_field(seed=6)
    f.set_gaussians(p)
    ids = [f.add_image(c, t) for c, t in zip(cams, tg)]
    kw = dict(grad_thresh=1e-6, percent_dense=0.02, min_opacity=0.01, max_scale=0.5)
    f.optimize_step(ids)
    f.densify(**kw)  # the first densification (split counter 0)
    f.optimize_step(ids)
    f.save(tmp_path / "s.gsf")
    g = gs.Field.load(tmp_path / "s.gsf")
    for x in (f, g):
        x.optimize_step(ids)
    sa, sb = f.densify_stats(), g.densify_stats()
    assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
    ra, rb = f.densify(**kw), g.densify(**kw)  # the second one (counter 1) on both
    assert ra == rb
    for a, b in zip(f.get_gaussians(with_adam=True), g.get_gaussians(with_adam=True)):
        assert np.array_equal(a, b)
    f.close()
    g.close()
