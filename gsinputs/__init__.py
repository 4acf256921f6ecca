"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module only draws random numbers and builds cameras; it holds none of the method's
arithmetic (no projection, blending, loss or schedule).  Every workload of the paper (3DGS,
Mip-NeRF 360, UAV and Replica scenes) is absent here, so these generators stand in for them with
the shapes and statistics the workloads are specified by:

* ``cube_scene``  -- N Gaussians with means uniform in a 2 x 2 x 2 cube centred 3 units in front
  of the identity camera, log-scales N(-4, 0.5), random unit quaternions, opacity logits N(0, 1),
  SH N(0, 0.2) (the 256 x 256 single-view case);
* ``ring_scene``  -- an outdoor-like ring (radius 4..10 around the origin): 60 % of the means on a
  noisy ground plane y = 0 (noise 0.05), 40 % in 5 box-like clusters; log-scales N(-4.5, 0.7);
* ``ring_camera`` -- a camera on the ring looking inward (OpenCV axes, world up = -y);
* ``uniform_target`` -- a seeded uniform-random target image.

Parameters are returned component-major, shape (59, stride): rows 0-2 mean, 3-5 log-scale, 6-9
quaternion (w, x, y, z), 10 opacity logit, 11 + 3k + ch SH coefficient k of channel ch.
"""
from __future__ import annotations

import numpy as np

NPARAM = 59


def _stride(n, align=32):
    return max(align, (n + align - 1) // align * align)


def _empty(n, stride=None):
    stride = _stride(n) if stride is None else stride
    return np.zeros((NPARAM, stride), np.float32)


def cube_scene(n, seed=0, stride=None, center_z=3.0, half=1.0, logscale=(-4.0, 0.5), sh_sigma=0.2):
    rng = np.random.default_rng(seed)
    p = _empty(n, stride)
    p[0, :n] = rng.uniform(-half, half, n)
    p[1, :n] = rng.uniform(-half, half, n)
    p[2, :n] = rng.uniform(center_z - half, center_z + half, n)
    p[3:6, :n] = rng.normal(logscale[0], logscale[1], (3, n))
    q = rng.normal(0.0, 1.0, (4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    p[6:10, :n] = q
    p[10, :n] = rng.normal(0.0, 1.0, n)
    p[11:59, :n] = rng.normal(0.0, sh_sigma, (48, n))
    return p


def ring_scene(n, seed=0, stride=None, r_in=4.0, r_out=10.0, logscale=(-4.5, 0.7), sh_sigma=0.2):
    rng = np.random.default_rng(seed)
    p = _empty(n, stride)
    n_ground = int(round(0.6 * n))
    n_box = n - n_ground
    # ground: uniform over the annulus area, height noise 0.05
    r = np.sqrt(rng.uniform(r_in * r_in, r_out * r_out, n_ground))
    th = rng.uniform(0.0, 2.0 * np.pi, n_ground)
    gx, gz = r * np.cos(th), r * np.sin(th)
    gy = rng.normal(0.0, 0.05, n_ground)
    # 5 boxes standing on the ground inside the ring
    centers_r = rng.uniform(r_in + 1.0, r_out - 1.0, 5)
    centers_t = rng.uniform(0.0, 2.0 * np.pi, 5)
    sizes = rng.uniform(0.6, 1.6, (5, 3))
    which = rng.integers(0, 5, n_box)
    local = rng.uniform(-0.5, 0.5, (n_box, 3)) * sizes[which]
    bx = centers_r[which] * np.cos(centers_t[which]) + local[:, 0]
    bz = centers_r[which] * np.sin(centers_t[which]) + local[:, 2]
    by = -(local[:, 1] + 0.5 * sizes[which, 1])  # boxes rise above the ground (up = -y)
    p[0, :n] = np.concatenate([gx, bx])
    p[1, :n] = np.concatenate([gy, by])
    p[2, :n] = np.concatenate([gz, bz])
    p[3:6, :n] = rng.normal(logscale[0], logscale[1], (3, n))
    q = rng.normal(0.0, 1.0, (4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    p[6:10, :n] = q
    p[10, :n] = rng.normal(0.0, 1.0, n)
    p[11:59, :n] = rng.normal(0.0, sh_sigma, (48, n))
    return p


def look_at(eye, target, up=(0.0, -1.0, 0.0)):
    """World->camera (R, t) for a camera at ``eye`` looking at ``target`` (OpenCV: +z forward,
    +y down on the image, ``up`` is the world's up direction)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    x = np.cross(up, f)
    x /= np.linalg.norm(x)
    x = -x
    y = np.cross(f, x)
    R = np.stack([x, y, f])  # rows: camera axes in world coordinates
    t = -R @ eye
    return R, t


def camera_dict(R, t, fx, fy, cx, cy, W, H):
    return dict(R=np.asarray(R, np.float64), t=np.asarray(t, np.float64), fx=float(fx), fy=float(fy),
                cx=float(cx), cy=float(cy), width=int(W), height=int(H))


def identity_camera(W=256, H=256, f=256.0):
    return camera_dict(np.eye(3), np.zeros(3), f, f, W / 2.0, H / 2.0, W, H)


def ring_camera(theta, W=1297, H=840, f=1000.0, radius=7.0, height=1.5, target_height=0.3,
                jitter=0.0, rng=None):
    eye = np.array([radius * np.cos(theta), -height, radius * np.sin(theta)])
    tgt = np.array([0.0, -target_height, 0.0])
    if jitter and rng is not None:
        eye = eye + rng.normal(0.0, jitter, 3)
        tgt = tgt + rng.normal(0.0, jitter, 3)
    R, t = look_at(eye, tgt)
    return camera_dict(R, t, f, f, W / 2.0, H / 2.0, W, H)


def uniform_target(W, H, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (3, H, W)).astype(np.float32)


MIXED_SIZES = [(960, 540), (1280, 720), (1297, 840), (1600, 1060)]


def batched_views(n_views=9, seed=0, f=1000.0):
    """The new view plus neighbours on a seeded circular trajectory (radius 7) at mixed sizes."""
    rng = np.random.default_rng(seed)
    cams = []
    base = rng.uniform(0, 2 * np.pi)
    for k in range(n_views):
        W, H = MIXED_SIZES[int(rng.integers(0, len(MIXED_SIZES)))]
        theta = base + 0.12 * (k - n_views // 2)
        cams.append(ring_camera(theta, W, H, f, jitter=0.05, rng=rng))
    return cams


def random_walk_cameras(n, seed=0, W=1297, H=840, f=1000.0, radius=7.0, overlap=(0.6, 0.8), reverse_p=0.1):
    """Cameras on the ring looking inward; consecutive frames overlap 60-80 % of the horizontal
    field of view (the heading moves by (1 - overlap) x FOV), with occasional reversals."""
    rng = np.random.default_rng(seed)
    fov = 2.0 * np.arctan(W / (2.0 * f))
    theta = rng.uniform(0, 2 * np.pi)
    direction = 1.0
    cams = []
    for k in range(n):
        if k > 0:
            if rng.uniform() < reverse_p:
                direction = -direction
            theta += direction * (1.0 - rng.uniform(*overlap)) * fov
        cams.append(ring_camera(theta, W, H, f, radius=radius, jitter=0.03, rng=rng))
    return cams


def sparse_points(gt_params, n_gt, cam, n_pts, seed=0, noise=0.01):
    """Synthetic sparse points of one image (stand-in for an SfM front end): ground-truth means
    visible in the camera's frustum, n_pts of them at random, plus N(0, noise) jitter; colour is
    the ground-truth DC colour; the track id is the ground-truth index."""
    rng = np.random.default_rng(seed)
    mu = gt_params[0:3, :n_gt].T.astype(np.float64)
    pc = mu @ np.asarray(cam["R"]).T + np.asarray(cam["t"])
    z = pc[:, 2]
    ok = z > 0.2
    u = cam["fx"] * pc[:, 0] / np.where(ok, z, 1.0) + cam["cx"]
    v = cam["fy"] * pc[:, 1] / np.where(ok, z, 1.0) + cam["cy"]
    ok &= (u >= 0) & (u < cam["width"]) & (v >= 0) & (v < cam["height"])
    ids = np.nonzero(ok)[0]
    if len(ids) > n_pts:
        ids = np.sort(rng.choice(ids, n_pts, replace=False))
    xyz = (mu[ids] + rng.normal(0.0, noise, (len(ids), 3))).astype(np.float32)
    c0 = 0.5 * np.sqrt(1.0 / np.pi)
    rgb = np.clip(gt_params[11:14, ids].T * c0 + 0.5, 0.0, 1.0).astype(np.float32)
    return xyz, rgb, ids.astype(np.int64)
