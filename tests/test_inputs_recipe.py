"""The seeded synthetic inputs match the recipe they stand in for (the scene-scale ring volume, the
tiny cube view, the trajectories): proportions, ranges and distributions, and determinism per seed.
The generators hold no arithmetic of the method; these checks keep the workloads' shapes honest."""
import numpy as np

import gsinputs as gi


def test_ring_scene_recipe():
    n = 200_000
    p = gi.ring_scene(n, seed=0, stride=n)
    assert p.shape == (59, n) and p.dtype == np.float32
    x, y, z = p[0].astype(np.float64), p[1].astype(np.float64), p[2].astype(np.float64)
    r = np.hypot(x, z)
    ground = slice(0, int(round(0.6 * n)))
    # 60 % on the ground plane: y ~ N(0, 0.05), uniform over the annulus 4 <= r <= 10
    assert abs(np.std(y[ground]) - 0.05) < 0.002 and abs(np.mean(y[ground])) < 0.002
    assert r[ground].min() >= 4.0 - 1e-4 and r[ground].max() <= 10.0 + 1e-4
    # uniform over the area: half the points inside r^2 = (16 + 100) / 2
    assert abs(np.mean(r[ground] ** 2 < 58.0) - 0.5) < 0.01
    # 40 % in boxes standing on the ground (up = -y), inside the ring
    boxes = slice(int(round(0.6 * n)), n)
    assert (y[boxes] <= 1e-6).all() and (r[boxes] > 2.0).all() and (r[boxes] < 12.0).all()
    # log-scales N(-4.5, 0.7); unit quaternions; opacity logits N(0, 1); SH N(0, 0.2)
    ls = p[3:6].astype(np.float64)
    assert abs(ls.mean() + 4.5) < 0.01 and abs(ls.std() - 0.7) < 0.01
    assert np.allclose(np.linalg.norm(p[6:10].astype(np.float64), axis=0), 1.0, atol=1e-6)
    assert abs(p[10].mean()) < 0.01 and abs(p[10].std() - 1.0) < 0.01
    assert abs(p[11:59].std() - 0.2) < 0.002
    # seeded: same seed, same scene; another seed, another one
    assert np.array_equal(p, gi.ring_scene(n, seed=0, stride=n))
    assert not np.array_equal(p, gi.ring_scene(n, seed=1, stride=n))


def test_cube_scene_and_tiny_view():
    p = gi.cube_scene(4096, seed=3)
    assert p.shape[1] % 32 == 0 and (p[:, 4096:] == 0).all()
    assert (np.abs(p[0, :4096]) <= 1.0).all() and (np.abs(p[2, :4096] - 3.0) <= 1.0).all()
    assert abs(p[3:6, :4096].mean() + 4.0) < 0.05
    cam = gi.identity_camera()
    assert cam["width"] == cam["height"] == 256 and cam["fx"] == 256.0 and cam["cx"] == 128.0
    t = gi.uniform_target(256, 256, 1)
    assert t.shape == (3, 256, 256) and t.min() >= 0.0 and t.max() <= 1.0


def test_ring_camera_looks_at_the_ring_centre():
    cam = gi.ring_camera(0.3)
    R, t = np.asarray(cam["R"]), np.asarray(cam["t"])
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and abs(np.linalg.det(R) - 1.0) < 1e-12
    eye = -R.T @ t
    assert abs(np.hypot(eye[0], eye[2]) - 7.0) < 1e-9 and abs(eye[1] + 1.5) < 1e-9
    # the target (0, -0.3, 0) projects to the image centre
    pc = R @ np.array([0.0, -0.3, 0.0]) + t
    assert pc[2] > 0
    u = cam["fx"] * pc[0] / pc[2] + cam["cx"]
    v = cam["fy"] * pc[1] / pc[2] + cam["cy"]
    assert abs(u - 1297 / 2) < 1e-6 and abs(v - 840 / 2) < 1e-6


def test_trajectories():
    cams = gi.batched_views(9, seed=2)
    assert len(cams) == 9 and all((c["width"], c["height"]) in gi.MIXED_SIZES for c in cams)
    walk = gi.random_walk_cameras(20, seed=7)
    fov = 2.0 * np.arctan(1297 / 2000.0)
    # consecutive headings move by (1 - overlap) x FOV with overlap in [0.6, 0.8] (jitter aside)
    heads = []
    for c in walk:
        eye = -np.asarray(c["R"]).T @ np.asarray(c["t"])
        heads.append(np.arctan2(eye[2], eye[0]))
    steps = np.abs(np.angle(np.exp(1j * np.diff(heads))))
    assert (steps > 0.15 * fov).all() and (steps < 0.45 * fov).all()
