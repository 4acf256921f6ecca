"""Session layer through the C ABI: optimisation step vs the oracle's step, graph replay vs
eager launch, snapshot/restore, the schedule (Eq. 3-8) vs the oracle's schedule, and the field
update of Sec. IV-B (new-point test and 3DGS initialisation)."""
import math

import numpy as np
import pytest

import gsinputs as gi
import oracle
from helpers import config1, ocam
from parity import check_adam, raster_gradients
from oracle import schedule as sch

pytestmark = pytest.mark.gpu

LRS_REST = [5e-3, 1e-3, 0.05, 2.5e-3, 2.5e-3 / 20]
C0 = 0.5 * math.sqrt(1.0 / math.pi)


def make_field(**kw):
    import paper_2503_13086_gb300 as gs
    kw.setdefault("scene_extent", 1.0)
    kw.setdefault("tiling", (16, 16, 256))  # the oracle's default binning; bitwise comparisons
    return gs.Field(**kw)


def test_step_matches_oracle_step():
    p, cams, tg = config1(seed=4)
    f = make_field(use_graph=0)
    f.set_gaussians(p)
    img = f.add_image(cams[0], tg[0])
    lr = f.image_lr(img)
    assert lr == pytest.approx(1.6e-4, rel=1e-6)  # Eq. 6-8: T = 0, no overlapping image
    loss = f.optimize_step([img])
    got = f.get_gaussians()
    f.close()
    L, _, _ = oracle.loss_and_grad(p, [ocam(cams[0])], tg, lam=0.2, prec="f32")
    assert abs(loss - L) <= 1e-5 * max(1.0, abs(L))
    # the step's gradients (each stage against the oracle) and its Adam update on them
    _, grads = raster_gradients(p, 4096, cams, tg, label="session step")
    check_adam("session step", got, p, grads, [lr * 1.0] + LRS_REST, 1)


def test_graph_replay_equals_eager():
    p, cams, tg = config1(seed=5)
    res = []
    for use_graph in (1, 0):
        f = make_field(use_graph=use_graph)
        f.set_gaussians(p)
        img = f.add_image(cams[0], tg[0])
        losses = [f.optimize_step([img]) for _ in range(4)]
        res.append((losses, f.get_gaussians(with_adam=True)))
        f.close()
    assert res[0][0] == res[1][0]
    for a, b in zip(res[0][1], res[1][1]):
        assert np.array_equal(a, b)


def test_snapshot_restore():
    p, cams, tg = config1(seed=6)
    f = make_field()
    f.set_gaussians(p)
    img = f.add_image(cams[0], tg[0])
    f.optimize_step([img])
    f.snapshot()
    s0 = f.get_gaussians(with_adam=True)
    T0, _ = f.image_info(img, 1)
    l1 = [f.optimize_step([img]) for _ in range(2)]
    assert not np.array_equal(f.get_gaussians(), s0[0])
    f.restore()
    s1 = f.get_gaussians(with_adam=True)
    for a, b in zip(s0, s1):
        assert np.array_equal(a, b)
    assert f.image_info(img, 1)[0] == T0
    l2 = [f.optimize_step([img]) for _ in range(2)]
    assert l1 == l2  # deterministic replay from the snapshot
    f.close()


def test_schedule_matches_oracle():
    """Golden 5-image overlap example: weights (Eq. 3-4), allocation (Eq. 5 + semi-global) and the
    per-image learning rate (Eq. 6-8) of the C++ session against the oracle's schedule."""
    T_I, N_m, seed = 21, 3, 11  # odd: the semi-global remainder exercises the seeded draw
    f = make_field(T_I=T_I, N_m=N_m, T_a=200, seed=seed, use_graph=0)
    p = gi.cube_scene(512, seed=1, stride=512)
    f.set_gaussians(p)
    tracks = [np.arange(1, 11), np.arange(6, 16), np.arange(11, 21), np.arange(16, 26), np.arange(30, 36)]
    W, H = 64, 48
    for k, tr in enumerate(tracks):
        cam = gi.identity_camera(W, H, 64.0)
        cam["t"] = np.array([0.05 * k, 0.0, 0.0])
        f.add_image(cam, gi.uniform_target(W, H, k), pts_xyz=np.zeros((len(tr), 3)) + 100.0 + k,
                    pts_rgb=np.full((len(tr), 3), 0.5), tracks=tr)
    M = sch.overlap_matrix(tracks)
    for i in range(5):
        assert np.allclose(f.image_info(i, 5)[1], M[i], atol=1e-7)
    ids, w = f.select_neighbors(3, 4)
    wref, _ = sch.hierarchical_weights(M, 3)
    assert ids == [3, 2, 1, 0]
    assert np.allclose(w, [wref[i] for i in ids], atol=1e-7)
    # integrate image 3 and compare T_j with the oracle's allocation
    n_before = f.stats()["n_gaussians"]
    st = f.integrate(3)
    keys, iters, slots = sch.allocate(wref, N_m, T_I, list(range(5)), 3, seed)
    assert st["iterations"] == T_I and st["key_images"] == len(keys)
    Ts = [f.image_info(i, 5)[0] for i in range(5)]
    assert Ts == [iters[i] for i in range(5)]
    for i in range(5):
        ref = sch.lr_image(i, M, Ts, 200, 1.6e-4, 1.6e-6)
        assert f.image_lr(i) == pytest.approx(ref, rel=1e-5)
    assert f.stats()["n_gaussians"] == n_before
    f.close()


def test_field_update_adds_far_points_with_3dgs_init():
    thr = 0.05
    f = make_field(add_dist_thresh=thr, use_graph=0)
    rng = np.random.default_rng(3)
    W, H = 48, 32
    cam = gi.identity_camera(W, H, 48.0)
    pts1 = rng.uniform(-0.5, 0.5, (200, 3)) + [0, 0, 3]
    col1 = rng.uniform(0, 1, (200, 3))
    f.add_image(cam, gi.uniform_target(W, H, 1), pts1, col1, np.arange(200))
    n1 = f.stats()["n_gaussians"]
    # first image: no existing points, every point becomes a Gaussian
    assert n1 == 200
    near = pts1[:50] + rng.normal(0, 0.005, (50, 3))        # within thr of an existing point
    far = rng.uniform(-0.5, 0.5, (80, 3)) + [0, 0, 6]        # far from everything
    pts2 = np.concatenate([near, far])
    col2 = rng.uniform(0, 1, (130, 3))
    f.add_image(cam, gi.uniform_target(W, H, 2), pts2, col2, np.arange(100, 230))
    d_exist = np.sqrt(((pts2[:, None, :] - pts1[None, :, :]) ** 2).sum(-1)).min(1)
    is_new = d_exist > thr
    got = f.get_gaussians()
    assert got.shape[1] == 200 + is_new.sum()
    new = got[:, 200:]
    allp = np.concatenate([pts1, pts2]).astype(np.float32)
    idx = np.nonzero(is_new)[0]
    assert np.allclose(new[0:3].T, pts2[idx], atol=1e-6)
    for q, k in enumerate(idx):
        d2 = ((allp - pts2[k].astype(np.float32)) ** 2).sum(1)
        d2[200 + k] = np.inf
        mean3 = np.sort(d2)[:3].mean()
        assert new[3, q] == pytest.approx(math.log(math.sqrt(max(mean3, 1e-7))), abs=1e-4)
    assert np.allclose(new[6], 1.0) and np.allclose(new[7:10], 0.0)
    assert np.allclose(new[10], math.log(0.1 / 0.9), atol=1e-6)
    assert np.allclose(new[11:14].T, (col2[idx] - 0.5) / C0, atol=1e-5)
    assert np.allclose(new[14:59], 0.0)
    # overlap from shared tracks: 100 of 200 tracks of image 0 are in image 1 (130 tracks)
    assert f.image_info(0, 2)[1][1] == pytest.approx(100 / 130, rel=1e-6)
    f.close()


def test_budget_and_bad_arguments():
    import paper_2503_13086_gb300 as gs
    f = make_field(hbm_budget_bytes=1 << 20)
    with pytest.raises(gs.GSError) as e:
        f.set_gaussians(gi.cube_scene(100000, seed=0, stride=100000))
    assert e.value.status == 3  # GS_ERR_BUDGET
    f.close()
    f = make_field()
    with pytest.raises(gs.GSError) as e:
        f.optimize_step([0])
    assert e.value.status in (1, 7)
    f.close()


@pytest.mark.parametrize("scaling", [0, 1])
def test_multi_view_step_matches_oracle(scaling):
    """A step over three views at mixed sizes (R13: mean loss, one Adam step at the mean of the
    views' Eq. 8 rates); with batch_scaling every rate is x sqrt(3) and the betas are cubed."""
    p = gi.cube_scene(3000, seed=12, stride=3008)
    cams = [gi.identity_camera(96, 64, 90.0), gi.identity_camera(70, 52, 60.0)]
    R, t = gi.look_at([0.4, -0.3, -0.4], [0.0, 0.0, 3.0])
    cams.append(gi.camera_dict(R, t, 70.0, 70.0, 40.0, 30.0, 81, 61))
    tg = [gi.uniform_target(c["width"], c["height"], 20 + k) for k, c in enumerate(cams)]
    f = make_field(use_graph=0, batch_scaling=scaling)
    f.set_gaussians(p[:, :3000])
    ids = [f.add_image(c, t) for c, t in zip(cams, tg)]
    lr = float(np.mean([f.image_lr(i) for i in ids]))
    loss = f.optimize_step(ids)
    got = f.get_gaussians()
    L, _, _ = oracle.loss_and_grad(p, [ocam(c) for c in cams], tg, lam=0.2, prec="f32", n=3000)
    assert abs(loss - L) <= 1e-5 * max(1.0, abs(L))
    s = math.sqrt(3.0) if scaling else 1.0
    b1, b2 = (0.9 ** 3, 0.999 ** 3) if scaling else (0.9, 0.999)
    lrs = [s * lr] + [s * x for x in LRS_REST]
    _, grads = raster_gradients(p, 3000, cams, tg, label="three-view step")
    check_adam("three-view step", got, p, grads, lrs, 1, b1=b1, b2=b2, n=3000)
    f.close()


def test_field_update_at_scale_matches_brute_force():
    """Four images of 30 000 sparse points each (the point arrays and the hash table grow and are
    rebuilt on the way): the far test against every earlier point and the 3-nearest initial scale
    against a k-d tree in float64, away from distances within 1e-5 of the threshold."""
    from scipy.spatial import cKDTree
    thr = 0.02
    f = make_field(add_dist_thresh=thr, use_graph=0)
    rng = np.random.default_rng(7)
    cam = gi.identity_camera(48, 32, 48.0)
    allp = np.zeros((0, 3), np.float32)
    n_g = 0
    for k in range(4):
        pts = rng.uniform(-1.0, 1.0, (30000, 3)).astype(np.float32) + np.float32([0, 0, 3])
        col = rng.uniform(0, 1, (30000, 3)).astype(np.float32)
        if len(allp):
            d, _ = cKDTree(allp.astype(np.float64)).query(pts.astype(np.float64), k=1)
        else:
            d = np.full(len(pts), np.inf)
        far = d > thr
        tie = np.abs(d - thr) <= 1e-5 * thr
        f.add_image(cam, gi.uniform_target(48, 32, k), pts, col, np.arange(30000) + 30000 * k)
        got = f.get_gaussians()
        added = got.shape[1] - n_g
        assert abs(added - int(far.sum())) <= int(tie.sum()), (k, added, int(far.sum()))
        allp = np.concatenate([allp, pts])
        if not tie.any():
            new = got[:, n_g:]
            idx = np.nonzero(far)[0]
            assert np.allclose(new[0:3].T, pts[idx])
            dd, _ = cKDTree(allp.astype(np.float64)).query(pts[idx].astype(np.float64), k=4)
            ref = np.log(np.sqrt(np.maximum((dd[:, 1:] ** 2).mean(1), 1e-7)))
            assert np.allclose(new[3], ref, atol=1e-4), np.abs(new[3] - ref).max()
            assert np.allclose(new[11:14].T, (col[idx] - 0.5) / C0, atol=1e-5)
        n_g = got.shape[1]
    f.close()


def test_new_gaussians_start_with_zero_adam_moments_after_restore():
    thr = 0.05
    f = make_field(add_dist_thresh=thr, use_graph=0)
    rng = np.random.default_rng(4)
    cam = gi.identity_camera(64, 48, 64.0)
    pts1 = rng.uniform(-0.5, 0.5, (300, 3)).astype(np.float32) + np.float32([0, 0, 3])
    img = f.add_image(cam, gi.uniform_target(64, 48, 1), pts1, rng.uniform(0, 1, (300, 3)), np.arange(300))
    f.snapshot()
    pts2 = rng.uniform(-0.5, 0.5, (200, 3)).astype(np.float32) + np.float32([0, 0, 5])
    f.add_image(cam, gi.uniform_target(64, 48, 2), pts2, rng.uniform(0, 1, (200, 3)), np.arange(300, 500))
    for _ in range(3):
        f.optimize_step([img])
    _, m, v = f.get_gaussians(with_adam=True)
    assert np.abs(m[:, 300:]).max() > 0  # the Gaussians past the snapshot have moments now
    f.restore()
    pts3 = rng.uniform(-0.5, 0.5, (150, 3)).astype(np.float32) + np.float32([0, 0, 8])
    f.add_image(cam, gi.uniform_target(64, 48, 3), pts3, rng.uniform(0, 1, (150, 3)), np.arange(500, 650))
    p, m, v = f.get_gaussians(with_adam=True)
    assert p.shape[1] == 450
    assert np.all(m[:, 300:] == 0) and np.all(v[:, 300:] == 0)
    f.close()


def test_paper_loss_preset_with_the_load_term():
    """Eq. 10 with the paper's weights: 0.47 L1 + 0.12 D-SSIM + 0.41 L_load, L_load = std of G_p
    over the pixels some Gaussian reaches (Eq. 9), its gradient through the soft count: the session
    step's loss against the oracle's, its Adam update on the step's gradients (each stage of which
    is checked against the oracle with the load term)."""
    p, cams, tg = config1(seed=7)
    f = make_field(use_graph=0, lambda_l1=0.47, lambda_ssim=0.12, lambda_load=0.41)
    f.set_gaussians(p)
    img = f.add_image(cams[0], tg[0])
    lr = f.image_lr(img)
    loss = f.optimize_step([img])
    got = f.get_gaussians()
    ref_loss, _, _ = oracle.loss_and_grad(p, [ocam(cams[0])], tg, lam=0.12, lambda_l1=0.47, lambda_load=0.41,
                                          prec="f32")
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss)), (loss, ref_loss)
    _, grads = raster_gradients(p, 4096, cams, tg, lam=0.12, lambda_l1=0.47, lambda_load=0.41,
                                label="paper-weights step")
    check_adam("paper-weights step", got, p, grads, [lr] + LRS_REST, 1)
    f.close()


def test_session_checkpoint_and_resume_continue_bit_for_bit(tmp_path):
    """A session saved to a file after three arrivals and resumed in a new field integrates the next
    arrivals exactly as the uninterrupted session (fixed tiling)."""
    import paper_2503_13086_gb300 as gs
    gt = gi.ring_scene(20000, seed=3, stride=20000)
    cams = gi.random_walk_cameras(5, seed=4, W=160, H=104, f=125.0)
    rng = np.random.default_rng(0)
    tgt = [gi.uniform_target(160, 104, 40 + k) for k in range(5)]
    pts = [gi.sparse_points(gt, 20000, c, 1500, seed=k) for k, c in enumerate(cams)]
    f = make_field(T_I=16, N_m=3, scene_extent=7.0, seed=3, add_dist_thresh=0.05)

    def arrive(field, k):
        xyz, rgb, tr = pts[k]
        img = field.add_image(cams[k], tgt[k], xyz, rgb, tr)
        field.integrate(img)

    for k in range(3):
        arrive(f, k)
    path = str(tmp_path / "session.gsf")
    f.save(path)
    g = gs.Field.load(path)
    a0 = f.get_gaussians(with_adam=True)
    b0 = g.get_gaussians(with_adam=True)
    for x, y in zip(a0, b0):
        assert np.array_equal(x, y)
    for k in (3, 4):
        arrive(f, k)
        arrive(g, k)
    for x, y in zip(f.get_gaussians(with_adam=True), g.get_gaussians(with_adam=True)):
        assert np.array_equal(x, y)
    sf, sg = f.stats(), g.stats()
    assert sf["adam_step"] == sg["adam_step"] and sf["n_images"] == sg["n_images"] == 5
    assert [f.image_info(i, 5) for i in range(5)] == [g.image_info(i, 5) for i in range(5)]
    f.close()
    g.close()


def test_initial_training_draws_views_and_follows_the_3dgs_rate():
    """Phase 1 (Sec. IV-A): the views come from SplitMix64 (seed ^ 0x5048415345310000, next() mod n)
    and the position rate from 3DGS's exponential schedule, not from Eq. 8: after one ordinary step
    has made every image 'trained' (T_j >= T_a = 1, Eq. 8 would give eta_f), the first phase-1 step
    still uses eta_0 x extent."""
    p = gi.cube_scene(3000, seed=13, stride=3008)
    cams = [gi.identity_camera(64, 48, 60.0) for _ in range(3)]
    for k, c in enumerate(cams):
        c["t"] = np.array([0.03 * k, 0.0, 0.0])
    tg = [gi.uniform_target(64, 48, 50 + k) for k in range(3)]
    f = make_field(use_graph=0, T_a=1, seed=21)
    f.set_gaussians(p[:, :3000])
    ids = [f.add_image(c, t) for c, t in zip(cams, tg)]
    f.optimize_step(ids)  # T_j = 1 for all three
    assert f.image_lr(0) == pytest.approx(1.6e-6, rel=1e-5)
    p1, m1, v1 = f.get_gaussians(with_adam=True)
    rng = sch.SplitMix64(21 ^ 0x5048415345310000)
    draws = [rng.below(3) for _ in range(5)]
    st = f.initial_training(1, max_steps=30000)
    assert st["iterations"] == 1 and st["steps"] == 1
    got = f.get_gaussians()
    P1 = np.zeros((59, 3008), np.float32)
    P1[:, :3000] = p1
    M1 = np.zeros_like(P1)
    V1 = np.zeros_like(P1)
    M1[:, :3000] = m1
    V1[:, :3000] = v1
    _, grads = raster_gradients(P1, 3000, [cams[draws[0]]], [tg[draws[0]]], label="phase-1 step")
    check_adam("phase-1 step", got, P1, grads, [1.6e-4] + LRS_REST, 2, m0=M1, v0=V1, n=3000)
    # the rest of the phase: T_j counts follow the same draws
    f.initial_training(4, max_steps=30000)
    counts = [1 + draws[:5].count(i) for i in range(3)]
    assert [f.image_info(i, 3)[0] for i in range(3)] == counts
    assert f.stats()["adam_step"] == 6
    f.close()


def test_sparse_adam_updates_only_the_gaussians_a_step_sees():
    """sparse_adam: Gaussians without instances in the step's views keep parameters and moments
    bit for bit; the others take the dense step's update."""
    p, cams, tg = config1(seed=8)
    p = p.copy()
    p[0, ::5] += 3.0  # push a fifth of the cube out of the view
    f = make_field(use_graph=0, sparse_adam=1)
    f.set_gaussians(p)
    img = f.add_image(cams[0], tg[0])
    lr = f.image_lr(img)
    loss = f.optimize_step([img])
    got, gm, gv = f.get_gaussians(with_adam=True)
    L, g, r = oracle.loss_and_grad(p, [ocam(cams[0])], tg, lam=0.2, prec="f32")
    rect = r["projs"][0]["rect"]
    seen = ((rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1]) > 0) & (r["projs"][0]["radius"] > 0)
    assert 0.3 < seen.mean() < 0.95
    assert abs(loss - L) <= 1e-5 * max(1.0, abs(L))
    assert np.array_equal(got[:, ~seen], p[:, ~seen])
    assert not gm[:, ~seen].any() and not gv[:, ~seen].any()
    _, grads = raster_gradients(p, 4096, cams, tg, label="sparse-Adam step")
    check_adam("sparse-Adam step", got, p, grads, [lr] + LRS_REST, 1, cols=seen)
    f.optimize_step([img])  # the unseen ones stay put on later steps too
    assert np.array_equal(f.get_gaussians()[:, ~seen], p[:, ~seen])
    f.close()


def test_sparse_adam_over_several_views():
    """sparse_adam in a step over three views: a Gaussian seen by any of them takes the dense
    step's update, one seen by none keeps parameters and moments bit for bit."""
    p = gi.cube_scene(3000, seed=13, stride=3008)
    p[0, :3000:4] += 4.0  # a quarter far to the side: outside every view
    cams = [gi.identity_camera(96, 64, 90.0), gi.identity_camera(70, 52, 60.0)]
    R, t = gi.look_at([0.4, -0.3, -0.4], [0.0, 0.0, 3.0])
    cams.append(gi.camera_dict(R, t, 70.0, 70.0, 40.0, 30.0, 81, 61))
    tg = [gi.uniform_target(c["width"], c["height"], 30 + k) for k, c in enumerate(cams)]
    f = make_field(use_graph=0, sparse_adam=1)
    f.set_gaussians(p[:, :3000])
    ids = [f.add_image(c, t) for c, t in zip(cams, tg)]
    lr = float(np.mean([f.image_lr(i) for i in ids]))
    f.optimize_step(ids)
    got, gm, gv = f.get_gaussians(with_adam=True)
    L, g, r = oracle.loss_and_grad(p, [ocam(c) for c in cams], tg, lam=0.2, prec="f32", n=3000)
    seen = np.zeros(3000, bool)
    for v in range(3):
        rect = r["projs"][v]["rect"]
        seen |= ((rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1]) > 0) & (r["projs"][v]["radius"] > 0)
    assert 0.3 < seen.mean() < 0.9
    assert np.array_equal(got[:, ~seen], p[:, :3000][:, ~seen])
    assert not gm[:, ~seen].any() and not gv[:, ~seen].any()
    _, grads = raster_gradients(p, 3000, cams, tg, label="sparse-Adam three-view step")
    check_adam("sparse-Adam three-view step", got, p, grads, [lr] + LRS_REST, 1, n=3000, cols=seen)
    f.close()


def test_phase3_refinement_takes_updated_poses():
    """Phase 3 (Sec. IV-A) after the last arrival: a refined pose set with set_image is the one
    the next step renders (its loss equals the oracle's for that pose and the field's current
    state), and initial_training then runs the additional optimisation over the images."""
    p, cams, tg = config1(seed=14)
    f = make_field(use_graph=0)
    f.set_gaussians(p)
    img = f.add_image(cams[0], tg[0])
    f.optimize_step([img])
    refined = gi.camera_dict(cams[0]["R"], np.array([0.03, -0.02, 0.05]), cams[0]["fx"], cams[0]["fy"],
                             cams[0]["cx"], cams[0]["cy"], cams[0]["width"], cams[0]["height"])
    f.set_image(img, cam=refined)
    state = f.get_gaussians()
    loss = f.optimize_step([img])
    L, _, _ = oracle.loss_and_grad(state, [ocam(refined)], tg, lam=0.2, prec="f32")
    assert abs(loss - L) <= 1e-5 * max(1.0, abs(L))
    L_old, _, _ = oracle.loss_and_grad(state, [ocam(cams[0])], tg, lam=0.2, prec="f32")
    assert abs(L - L_old) > 1e-4  # the pose change is visible in the loss
    st = f.initial_training(6, max_steps=30000)
    assert st["iterations"] == 6 and np.isfinite(st["mean_loss"])
    f.close()


def test_interleaved_and_planar_targets_give_the_same_step():
    """gs_add_image takes the interleaved H x W x 3 image decoders produce (host or device) and
    transposes it on the device; the planar entry point takes 3 x H x W.  All three register the same
    target: the steps after them are bitwise equal.  A page-locked host image is read by the layout
    kernel directly (16-byte aligned, and at a 4-byte offset, which takes the per-pixel kernel).
    gs_field_stats reports the field's size and memory like gs_field_info_get, and gs_set_image
    replaces a target in either layout."""
    import torch
    p, cams, tg = config1(seed=9)
    hwc = np.ascontiguousarray(np.transpose(tg[0], (1, 2, 0)))
    pinned = torch.tensor(hwc).pin_memory()
    assert pinned.is_pinned() and pinned.data_ptr() % 16 == 0
    spare = torch.empty(hwc.size + 1, dtype=torch.float32).pin_memory()  # the same image 4 bytes in
    spare[1:] = torch.from_numpy(hwc.reshape(-1))
    pinned_off = spare[1:].view(hwc.shape)
    assert pinned_off.is_pinned() and pinned_off.data_ptr() % 16 == 4
    res = []
    for kind in ("chw", "hwc_host", "hwc_device", "hwc_pinned", "hwc_pinned_offset"):
        f = make_field(use_graph=0)
        f.set_gaussians(p)
        src = {"chw": tg[0], "hwc_host": hwc, "hwc_device": torch.tensor(hwc, device="cuda"), "hwc_pinned": pinned,
               "hwc_pinned_offset": pinned_off}[kind]
        img = f.add_image(cams[0], src)
        loss = f.optimize_step([img])
        n, b = f.footprint()
        st = f.stats()
        assert n == st["n_gaussians"] == 4096 and b == st["bytes_in_use"] > 0
        assert st["last_run_steps"] == 1 and st["last_run_ms"] > 0 and st["last_d2h_bytes"] > 0
        res.append((loss, f.get_gaussians()))
        # replacing the target with a zero image in the other layout changes the next loss
        zero = np.zeros((3, 256, 256), np.float32) if kind != "chw" else np.zeros((256, 256, 3), np.float32)
        f.set_image(img, zero)
        assert f.optimize_step([img]) != loss
        f.close()
    for loss, g in res[1:]:
        assert loss == res[0][0] and np.array_equal(g, res[0][1])
