"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test pins a part of the oracle to something other than itself: closed forms of a single
Gaussian's splat (Eq. 1-2 with the 3DGS EWA projection), hand-worked examples stored under
tests/golden/, exact binary termination, central finite differences of the whole forward, an
independent dense PyTorch formulation, torch.optim.Adam, a torch conv2d SSIM, and real
spherical harmonics from scipy.
"""
import math
import os

import numpy as np
import pytest

import gsinputs as gi
import oracle
from oracle import Camera
from oracle import schedule as sch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C0 = 0.5 * math.sqrt(1.0 / math.pi)


def blank(n, stride=32, dtype=np.float64):
    p = np.zeros((59, stride), dtype)
    p[6, :] = 1.0  # identity quaternion
    return p


def cam(W, H, f, cx=None, cy=None, R=None, t=None):
    return Camera(np.eye(3) if R is None else R, np.zeros(3) if t is None else t, f, f,
                  W / 2.0 if cx is None else cx, H / 2.0 if cy is None else cy, W, H)


# ------------------------------------------------------------------------------------------
# Spherical harmonics: degree <= 3 real SH in the convention of 3DGS, whose basis the paper keeps
# (Sec. V-A): Y_l^m of scipy carries the Condon-Shortley phase (-1)^m, and 3DGS's real basis is
# sqrt(2) Re Y_l^m (m > 0), sqrt(2) Im Y_l^|m| (m < 0), Y_l^0 (m = 0), ordered m = -l .. l.  Each of
# the oracle's 16 functions must equal that reference with its sign, and the set be orthonormal.
# ------------------------------------------------------------------------------------------
def _real_sh_3dgs(l, m, polar, azim):
    import scipy.special as sp
    if hasattr(sp, "sph_harm_y"):
        Y = sp.sph_harm_y(l, abs(m), polar, azim)
    else:  # older scipy
        Y = sp.sph_harm(abs(m), l, azim, polar)
    if m > 0:
        return math.sqrt(2.0) * Y.real
    if m < 0:
        return math.sqrt(2.0) * Y.imag
    return Y.real


def _sphere_quadrature():
    x, w = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phi = 2 * np.pi * np.arange(nphi) / nphi
    CT, PH = np.meshgrid(x, phi, indexing="ij")
    ST = np.sqrt(1 - CT ** 2)
    dirs = np.stack([ST * np.cos(PH), ST * np.sin(PH), CT], -1).reshape(-1, 3)
    wt = (w[:, None] * np.ones((1, nphi)) * (2 * np.pi / nphi)).reshape(-1)
    return dirs, wt


def test_sh_basis_matches_real_spherical_harmonics():
    dirs, wt = _sphere_quadrature()
    Y = oracle.sh_eval(dirs, "f64")
    G = (Y * wt[:, None]).T @ Y
    assert np.allclose(G, np.eye(16), atol=1e-12)
    polar = np.arccos(np.clip(dirs[:, 2], -1, 1))
    azim = np.arctan2(dirs[:, 1], dirs[:, 0])
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            ref = _real_sh_3dgs(l, m, polar, azim)
            # the projection onto the reference, sign included: +1 for the same function
            c = float(np.sum(wt * Y[:, k] * ref))
            assert abs(c - 1.0) < 1e-10, (l, m, c)
            assert np.allclose(Y[:, k], ref, atol=1e-12), (l, m)
            k += 1


def test_sh_basis_values_on_the_axes():
    """Hand-evaluated values on the coordinate axes (x, y, z = one of the unit vectors), from the
    normalisations sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) (times sqrt 2 for m != 0) and the
    Legendre functions of each (l, m); zero wherever a factor x, y or z of the function vanishes."""
    pi = math.pi
    k1 = math.sqrt(3 / (4 * pi))                  # l = 1
    k2 = 0.5 * math.sqrt(15 / pi)                 # l = 2, |m| = 1, 2 (xy, yz, xz)
    k20 = 0.25 * math.sqrt(5 / pi)                # l = 2, m = 0: (3 z^2 - 1)
    k22 = 0.25 * math.sqrt(15 / pi)               # l = 2, m = 2: (x^2 - y^2)
    k33 = 0.25 * math.sqrt(35 / (2 * pi))         # l = 3, |m| = 3
    k31 = 0.25 * math.sqrt(21 / (2 * pi))         # l = 3, |m| = 1
    k30 = 0.25 * math.sqrt(7 / pi)                # l = 3, m = 0: z (5 z^2 - 3)
    Y = oracle.sh_eval(np.eye(3), "f64")
    want = np.zeros((3, 16))
    want[:, 0] = 0.5 / math.sqrt(pi)
    # +x: Y_1^1 = -k1 x; Y_2^0 = -k20; Y_2^2 = +k22; Y_3^1 = -k31 x (4z^2 - x^2 - y^2) = +k31;
    #     Y_3^3 = -k33 x (x^2 - 3y^2) = -k33
    want[0, 3], want[0, 6], want[0, 8], want[0, 13], want[0, 15] = -k1, -k20, k22, k31, -k33
    # +y: Y_1^-1 = -k1 y; Y_2^0 = -k20; Y_2^2 = -k22; Y_3^-3 = -k33 y (3x^2 - y^2) = +k33;
    #     Y_3^-1 = -k31 y (4z^2 - x^2 - y^2) = +k31
    want[1, 1], want[1, 6], want[1, 8], want[1, 9], want[1, 11] = -k1, -k20, -k22, k33, k31
    # +z: Y_1^0 = k1 z; Y_2^0 = 2 k20; Y_3^0 = k30 z (2z^2 - 3x^2 - 3y^2) = 2 k30
    want[2, 2], want[2, 6], want[2, 12] = k1, 2 * k20, 2 * k30
    assert np.allclose(Y, want, atol=1e-14), np.argwhere(~np.isclose(Y, want, atol=1e-14))


# ------------------------------------------------------------------------------------------
# One isotropic Gaussian on the optical axis: J = (f/z) I, so Sigma_2D = ((f s / z)^2 + 0.3) I,
# alpha(d) = sigma exp(-d^2 / (2 v)), cut at 1/255, r = ceil(3 sqrt(v + sqrt(0.1))).
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_single_isotropic_gaussian_closed_form(prec, tol):
    W = H = 64
    f, z, s, sig, col = 64.0, 4.0, 0.05, 0.5, 0.9
    p = blank(1)
    p[2, 0] = z
    p[3:6, 0] = math.log(s)
    p[10, 0] = 0.0  # sigmoid(0) = 0.5
    p[11:14, 0] = (col - 0.5) / C0
    c = cam(W, H, f)
    r = oracle.render(p, [c], prec=prec, n=1)
    pr = r["projs"][0]
    v = (f * s / z) ** 2 + 0.3
    assert pr["radius"][0] == math.ceil(3 * math.sqrt(v + math.sqrt(0.1)))
    assert np.allclose(pr["conic"][0], [1 / v, 0.0, 1 / v], rtol=tol, atol=tol)
    assert np.allclose(pr["mean2d"][0], [32.0, 32.0])
    assert np.allclose(pr["rgb"][0], col, atol=tol)
    ys, xs = np.mgrid[0:H, 0:W]
    d2 = (xs - 32.0) ** 2 + (ys - 32.0) ** 2
    alpha = sig * np.exp(-d2 / (2 * v))
    alpha = np.where(alpha < 1 / 255, 0.0, alpha)
    img = r["outs"][0]["image"]
    for ch in range(3):
        assert np.allclose(img[ch], col * alpha, atol=tol)
    assert np.allclose(r["outs"][0]["T"], 1 - alpha, atol=tol)
    assert (r["outs"][0]["gp"] == (alpha > 0)).all()
    ring = (alpha == 0) & (d2 < 16)  # inside the radius but below the 1/255 cutoff
    assert ring.any()


def test_eq2_three_gaussians_by_hand():
    """Three Gaussians centred on one pixel at depths 5, 3, 4 (ids in a different order)."""
    W = H = 32
    ops = [0.3, 0.5, 0.6]
    depths = [5.0, 3.0, 4.0]
    cols = [(0.9, 0.1, 0.2), (0.2, 0.8, 0.1), (0.3, 0.3, 0.7)]
    p = blank(3)
    for i in range(3):
        p[2, i] = depths[i]
        p[3:6, i] = math.log(0.02)
        p[10, i] = math.log(ops[i] / (1 - ops[i]))
        p[11:14, i] = (np.array(cols[i]) - 0.5) / C0
    bg = (0.1, 0.2, 0.3)
    r = oracle.render(p, [cam(W, H, 32.0)], bg=bg, prec="f64", n=3)
    o = r["outs"][0]
    order = [1, 2, 0]  # by depth
    T = 1.0
    C = np.zeros(3)
    Ts = [T]
    for i in order:
        C += np.array(cols[i]) * ops[i] * T
        T *= 1 - ops[i]
        Ts.append(T)
    C += T * np.array(bg)
    assert np.allclose(o["image"][:, 16, 16], C, atol=1e-12)
    assert abs(o["T"][16, 16] - T) < 1e-12
    assert all(a >= b for a, b in zip(Ts, Ts[1:]))  # transmittance never increases
    assert o["gp"][16, 16] == 3 and o["last"][16, 16] == 3 and o["neval"][16, 16] == 3


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_termination_binary_exact(prec):
    """20 Gaussians with alpha exactly 0.5 at one pixel: T = 2^-13 >= 1e-4 after 13, the 14th would
    give 2^-14 < 1e-4, so exactly 13 are blended and the 14th entry is the last evaluated."""
    n = 20
    p = blank(n)
    for i in range(n):
        p[2, i] = 2.0 + 0.1 * i
        p[3:6, i] = math.log(0.01)
        p[10, i] = 0.0
        p[11:14, i] = (0.8 - 0.5) / C0
    r = oracle.render(p, [cam(16, 16, 16.0, cx=8.0, cy=8.0)], prec=prec, n=n)
    o = r["outs"][0]
    assert o["last"][8, 8] == 13 and o["gp"][8, 8] == 13 and o["neval"][8, 8] == 14
    assert o["T"][8, 8] == 2.0 ** -13
    assert abs(o["image"][0, 8, 8] - 0.8 * (1 - 2.0 ** -13)) < 1e-6


def test_alpha_clamp_and_zero_gradient_through_it():
    p = blank(1)
    p[2, 0] = 3.0
    p[3:6, 0] = math.log(0.5)
    p[10, 0] = 10.0  # sigmoid ~ 0.99995 -> alpha clamped at 0.99
    p[11:14, 0] = (0.6 - 0.5) / C0
    c = cam(1, 1, 10.0, cx=0.0, cy=0.0)
    bg = (0.25, 0.25, 0.25)
    tgt = np.zeros((3, 1, 1))
    L, g, r = oracle.loss_and_grad(p, [c], [tgt], lam=0.0, bg=bg, prec="f64", n=1)
    assert np.allclose(r["outs"][0]["image"][:, 0, 0], 0.6 * 0.99 + 0.25 * 0.01, atol=1e-12)
    assert g[10, 0] == 0.0  # no gradient to the opacity through the clamp
    assert np.all(g[0:10, 0] == 0.0)  # nor to the footprint
    assert g[11, 0] != 0.0  # the colour still receives gradient


def test_alpha_cutoff_skips():
    p = blank(1)
    p[2, 0] = 3.0
    p[3:6, 0] = math.log(0.5)
    sig = 0.9 / 255
    p[10, 0] = math.log(sig / (1 - sig))
    r = oracle.render(p, [cam(4, 4, 10.0, cx=2.0, cy=2.0)], bg=(0.3, 0.3, 0.3), prec="f64", n=1)
    o = r["outs"][0]
    assert (o["gp"] == 0).all() and np.allclose(o["image"], 0.3)


# ------------------------------------------------------------------------------------------
# Tile binning: a hand-worked example (golden) including a depth tie and two culled Gaussians.
# ------------------------------------------------------------------------------------------
def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *vals = line.split()
        out[k] = vals
    return out


def test_lists_hand_example():
    gd = _golden("lists_small.txt")
    g = [(8, 8, 2, 5.0), (16, 16, 4, 3.0), (40, 30, 3, 7.0), (20, 8, 1, 5.0), (0, 0, 0, 1.0), (-50, 8, 3, 2.0),
         (10, 6, 1, 5.0)]
    mean2d = np.array([[a[0], a[1]] for a in g], np.float32)
    radius = np.array([a[2] for a in g], np.int32)
    depth = np.array([a[3] for a in g], np.float32)
    L = oracle.build_lists([(48, 32)], mean2d, radius, depth)
    assert list(L["vals"]) == [int(x) for x in gd["sorted_ids"]]
    assert list((L["keys"] >> np.uint64(32)).astype(int)) == [int(x) for x in gd["sorted_tiles"]]
    assert list(L["ranges"].reshape(-1)) == [int(x) for x in gd["ranges"]]


def test_lists_invariants_random():
    rng = np.random.default_rng(5)
    V, n = 2, 300
    sizes = [(97, 61), (40, 33)]
    mean2d = np.concatenate([rng.uniform(-20, 120, (n, 2)) for _ in range(V)]).astype(np.float32)
    radius = rng.integers(0, 30, V * n).astype(np.int32)
    depth = rng.choice(np.array([1.0, 2.0, 3.5], np.float32), V * n)
    L = oracle.build_lists(sizes, mean2d, radius, depth)
    keys, vals = L["keys"], L["vals"]
    # sorted by (key, val) and each (record, tile) pair appears once
    order = np.lexsort((vals, keys))
    assert (order == np.arange(len(keys))).all()
    pairs = set(zip((keys >> np.uint64(32)).tolist(), vals.tolist()))
    assert len(pairs) == len(keys)
    # ranges partition the list
    r = L["ranges"]
    nonempty = r[:, 1] > r[:, 0]
    assert r[nonempty, 1].sum() - r[nonempty, 0].sum() == len(keys)


# ------------------------------------------------------------------------------------------
# Gradients: central finite differences in double of the full forward + loss, on tiny scenes
# that exercise the FOV clamp, the colour clamp and two views.  Perturbations that change any
# discrete decision (blend set, termination) are skipped.
# ------------------------------------------------------------------------------------------
def _scene(kind):
    if kind == "random":
        p = gi.cube_scene(6, seed=3, stride=32, logscale=(-1.5, 0.3)).astype(np.float64)
        cams = [cam(32, 32, 40.0)]
    elif kind == "fov_clamp":
        p = gi.cube_scene(5, seed=4, stride=32, logscale=(-1.5, 0.3)).astype(np.float64)
        # a large Gaussian whose mean lies outside 1.3 x the half-FOV tangent (0.52) but reaches in
        p[0:3, 0] = [0.6 * 3.0, 0.0, 3.0]
        p[3:6, 0] = math.log(0.6)
        cams = [cam(32, 32, 40.0)]
    elif kind == "colour_clamp":
        p = gi.cube_scene(5, seed=6, stride=32, logscale=(-1.5, 0.3)).astype(np.float64)
        p[11, 0] = -3.0  # red DC far below zero -> clamped channel
        cams = [cam(32, 32, 40.0)]
    else:  # two views
        p = gi.cube_scene(5, seed=7, stride=32, logscale=(-1.5, 0.3)).astype(np.float64)
        R, t = gi.look_at([0.6, -0.2, -0.3], [0.0, 0.0, 3.0])
        cams = [cam(32, 32, 40.0), cam(24, 28, 30.0, R=R, t=t)]
    return p, cams


@pytest.mark.parametrize("kind", ["random", "fov_clamp", "colour_clamp", "two_views"])
def test_gradients_match_central_differences(kind):
    p, cams = _scene(kind)
    n = 6 if kind == "random" else 5
    tgts = [gi.uniform_target(c.width, c.height, 11 + k).astype(np.float64) for k, c in enumerate(cams)]
    L, g, r = oracle.loss_and_grad(p, cams, tgts, lam=0.2, prec="f64", n=n)
    if kind == "fov_clamp":
        x_over_z = p[0, 0] / p[2, 0]
        assert x_over_z > 1.3 * 32 / (2 * 40.0)
        assert r["projs"][0]["radius"][0] > 0
    if kind == "colour_clamp":
        assert r["projs"][0]["clamp"][0] & 1
    eps = 1e-6
    keys = ("last", "gp", "neval")
    checked = 0
    for i in range(n):
        for c in range(59):
            lp_ = []
            same = True
            for sgn in (1, -1):
                q = p.copy()
                q[c, i] += sgn * eps
                l_, _, rq = oracle.loss_and_grad(q, cams, tgts, lam=0.2, prec="f64", n=n)
                lp_.append(l_)
                same &= all((rq["outs"][v][k] == r["outs"][v][k]).all() for v in range(len(cams)) for k in keys)
            if not same:
                continue
            fd = (lp_[0] - lp_[1]) / (2 * eps)
            an = g[c, i]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), abs(an)) + 2e-9, (kind, i, c, fd, an)
            checked += 1
    assert checked > 0.8 * n * 59


# ------------------------------------------------------------------------------------------
# An independent dense PyTorch (float64, autograd) restatement of the same forward and loss:
# every Gaussian is evaluated at every pixel; the tile rectangle, the cutoffs, the clamp and the
# early stop become masks computed without gradient.
# ------------------------------------------------------------------------------------------
def _dense_torch_loss(params, cam_, target, lam, n, bg=(0.0, 0.0, 0.0)):
    import torch
    P = params[:, :n]
    R = torch.tensor(cam_.R, dtype=torch.float64)
    t = torch.tensor(cam_.t, dtype=torch.float64)
    fx, fy, cx, cy, W, H = cam_.fx, cam_.fy, cam_.cx, cam_.cy, cam_.width, cam_.height
    mu = P[0:3].T
    pc = mu @ R.T + t
    x, y, z = pc[:, 0], pc[:, 1], pc[:, 2]
    q = P[6:10].T
    q = q / q.norm(dim=1, keepdim=True)
    w_, qx, qy, qz = q.unbind(1)
    Rq = torch.stack([
        1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - w_ * qz), 2 * (qx * qz + w_ * qy),
        2 * (qx * qy + w_ * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - w_ * qx),
        2 * (qx * qz - w_ * qy), 2 * (qy * qz + w_ * qx), 1 - 2 * (qx * qx + qy * qy)], 1).reshape(-1, 3, 3)
    S = torch.diag_embed(torch.exp(P[3:6].T))
    Mm = Rq @ S
    Sig = Mm @ Mm.transpose(1, 2)
    limx, limy = 1.3 * W / (2 * fx), 1.3 * H / (2 * fy)
    txz = torch.clamp(x / z, -limx, limx)
    tyz = torch.clamp(y / z, -limy, limy)
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([fx / z, zero, -fx * txz / z], 1), torch.stack([zero, fy / z, -fy * tyz / z], 1)], 1)
    Tm = J @ R
    cov = Tm @ Sig @ Tm.transpose(1, 2)
    a = cov[:, 0, 0] + 0.3
    b = cov[:, 0, 1]
    c = cov[:, 1, 1] + 0.3
    det = a * c - b * b
    ca, cb, cc = c / det, -b / det, a / det
    u = fx * x / z + cx
    v = fy * y / z + cy
    with torch.no_grad():
        mid = 0.5 * (a + c)
        lam_ = mid + torch.sqrt(torch.clamp(mid * mid - det, min=0.1))
        rad = torch.ceil(3 * torch.sqrt(lam_))
        gx, gy = (W + 15) // 16, (H + 15) // 16
        x0 = torch.clamp(torch.floor((u - rad) / 16), 0, gx)
        x1 = torch.clamp(torch.floor((u + rad + 15) / 16), 0, gx)
        y0 = torch.clamp(torch.floor((v - rad) / 16), 0, gy)
        y1 = torch.clamp(torch.floor((v + rad + 15) / 16), 0, gy)
        vis = (z > 0.2) & ((x1 - x0) * (y1 - y0) > 0)
    campos = -(R.T @ t)
    d = mu - campos
    d = d / d.norm(dim=1, keepdim=True)
    Y = torch.tensor(oracle.sh_eval(d.detach().numpy(), "f64"))
    # SH basis with gradient: evaluate the same polynomials in torch via the 16 monomial forms
    dx_, dy_, dz_ = d.unbind(1)
    k = [0.5 * math.sqrt(1 / math.pi), math.sqrt(3 / (4 * math.pi)), 0.5 * math.sqrt(15 / math.pi),
         0.25 * math.sqrt(5 / math.pi), 0.25 * math.sqrt(15 / math.pi), 0.25 * math.sqrt(35 / (2 * math.pi)),
         0.5 * math.sqrt(105 / math.pi), 0.25 * math.sqrt(21 / (2 * math.pi)), 0.25 * math.sqrt(7 / math.pi),
         0.25 * math.sqrt(105 / math.pi)]
    xx, yy, zz = dx_ * dx_, dy_ * dy_, dz_ * dz_
    Yt = torch.stack([
        torch.full_like(dx_, k[0]), -k[1] * dy_, k[1] * dz_, -k[1] * dx_,
        k[2] * dx_ * dy_, -k[2] * dy_ * dz_, k[3] * (2 * zz - xx - yy), -k[2] * dx_ * dz_, k[4] * (xx - yy),
        -k[5] * dy_ * (3 * xx - yy), k[6] * dx_ * dy_ * dz_, -k[7] * dy_ * (4 * zz - xx - yy),
        k[8] * dz_ * (2 * zz - 3 * xx - 3 * yy), -k[7] * dx_ * (4 * zz - xx - yy), k[9] * dz_ * (xx - yy),
        -k[5] * dx_ * (xx - 3 * yy)], 1)
    assert torch.allclose(Yt.detach(), Y, atol=1e-12)
    sh = P[11:59].T.reshape(-1, 16, 3)
    raw = (Yt[:, :, None] * sh).sum(1) + 0.5
    rgb = torch.clamp(raw, min=0.0)
    op = torch.sigmoid(P[10])
    # dense per-pixel blending in canonical order (depth, id)
    order = sorted(range(n), key=lambda i: (np.float32(z[i].item()).view(np.uint32), i))
    ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64), indexing="ij")
    tx_, ty_ = (xs // 16), (ys // 16)
    Tacc = torch.ones(H, W, dtype=torch.float64)
    C = torch.zeros(3, H, W, dtype=torch.float64)
    alive = torch.ones(H, W, dtype=torch.bool)
    for i in order:
        if not bool(vis[i]):
            continue
        inrect = (tx_ >= x0[i]) & (tx_ < x1[i]) & (ty_ >= y0[i]) & (ty_ < y1[i])
        ddx, ddy = u[i] - xs, v[i] - ys
        power = -0.5 * (ca[i] * ddx * ddx + cc[i] * ddy * ddy) - cb[i] * ddx * ddy
        al = torch.minimum(op[i] * torch.exp(power), torch.tensor(0.99, dtype=torch.float64))
        with torch.no_grad():
            m = inrect & alive & (power <= 0) & (al >= 1 / 255)
            stop = m & (Tacc * (1 - al) < 1e-4)
            m = m & ~stop
            alive = alive & ~stop
        mf = m.double()
        C = C + rgb[i][:, None, None] * (al * Tacc * mf)[None]
        Tacc = Tacc * (1 - al * mf)
    img = C + Tacc[None] * torch.tensor(bg, dtype=torch.float64)[:, None, None]
    # loss: L1 + SSIM with an 11x11 Gaussian window via conv2d (zero padding)
    g1 = torch.exp(-torch.arange(-5, 6, dtype=torch.float64) ** 2 / (2 * 1.5 ** 2))
    g1 = g1 / g1.sum()
    win = (g1[:, None] * g1[None, :])[None, None].repeat(3, 1, 1, 1)
    import torch.nn.functional as F
    X = img[None]
    Yg = torch.tensor(target, dtype=torch.float64)[None]
    mx = F.conv2d(X, win, padding=5, groups=3)
    my = F.conv2d(Yg, win, padding=5, groups=3)
    sxx = F.conv2d(X * X, win, padding=5, groups=3) - mx * mx
    syy = F.conv2d(Yg * Yg, win, padding=5, groups=3) - my * my
    sxy = F.conv2d(X * Yg, win, padding=5, groups=3) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ssim = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return (1 - lam) * (X - Yg).abs().mean() + lam * (1 - ssim.mean())


def test_gradients_match_dense_torch_autograd():
    import torch
    n = 40
    p = gi.cube_scene(n, seed=21, stride=64, logscale=(-2.5, 0.4)).astype(np.float64)
    c = cam(24, 20, 24.0)
    tgt = gi.uniform_target(24, 20, 3).astype(np.float64)
    L, g, r = oracle.loss_and_grad(p, [c], [tgt], lam=0.2, prec="f64", n=n)
    pt = torch.tensor(p, requires_grad=True)
    Lt = _dense_torch_loss(pt, c, tgt, 0.2, n)
    Lt.backward()
    assert abs(Lt.item() - L) < 1e-12
    gt = pt.grad.numpy()[:, :n]
    assert np.allclose(g[:, :n], gt, rtol=1e-8, atol=1e-12)


# ------------------------------------------------------------------------------------------
# Adam against torch.optim.Adam (per-group learning rates, three steps).
# ------------------------------------------------------------------------------------------
def test_adam_matches_torch():
    import torch
    rng = np.random.default_rng(2)
    n, stride = 50, 64
    p = rng.normal(size=(59, stride))
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    lrs = [1.6e-4 * 5, 5e-3, 1e-3, 0.05, 2.5e-3, 1.25e-4]
    groups = [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14), (14, 59)]
    tens = [torch.tensor(p[a:b, :n].copy(), requires_grad=True) for a, b in groups]
    opt = torch.optim.Adam([{"params": [t_], "lr": lr} for t_, lr in zip(tens, lrs)], betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 4):
        gr = rng.normal(size=(59, stride))
        oracle.adam(p, gr, m, v, lrs, step, n=n, prec="f64")
        for t_, (a, b) in zip(tens, groups):
            t_.grad = torch.tensor(gr[a:b, :n].copy())
        opt.step()
    ref = np.concatenate([t_.detach().numpy() for t_ in tens])
    assert np.allclose(p[:, :n], ref, rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------------------------------
# SSIM: identical images give SSIM 1 and zero gradient; values and gradients against torch.
# ------------------------------------------------------------------------------------------
def test_ssim_identical_images():
    x = gi.uniform_target(23, 17, 1).astype(np.float64)
    val, d, l1, ss = oracle.loss(x, x, lam=0.2, prec="f64")
    assert abs(ss - 1.0) < 1e-12 and l1 == 0.0 and abs(val) < 1e-12
    assert np.abs(d).max() < 1e-12


def test_loss_matches_torch_conv2d():
    import torch
    import torch.nn.functional as F
    x = gi.uniform_target(29, 19, 4).astype(np.float64)
    y = gi.uniform_target(29, 19, 5).astype(np.float64)
    val, d, _, _ = oracle.loss(x, y, lam=0.2, prec="f64")
    X = torch.tensor(x[None], requires_grad=True)
    Y = torch.tensor(y[None])
    g1 = torch.exp(-torch.arange(-5, 6, dtype=torch.float64) ** 2 / (2 * 1.5 ** 2))
    g1 = g1 / g1.sum()
    win = (g1[:, None] * g1[None, :])[None, None].repeat(3, 1, 1, 1)
    mx = F.conv2d(X, win, padding=5, groups=3)
    my = F.conv2d(Y, win, padding=5, groups=3)
    sxx = F.conv2d(X * X, win, padding=5, groups=3) - mx * mx
    syy = F.conv2d(Y * Y, win, padding=5, groups=3) - my * my
    sxy = F.conv2d(X * Y, win, padding=5, groups=3) - mx * my
    s = ((2 * mx * my + 1e-4) * (2 * sxy + 9e-4)) / ((mx * mx + my * my + 1e-4) * (sxx + syy + 9e-4))
    L = 0.8 * (X - Y).abs().mean() + 0.2 * (1 - s.mean())
    L.backward()
    assert abs(L.item() - val) < 1e-12
    assert np.allclose(d, X.grad.numpy()[0], atol=1e-12)


def test_float_and_double_oracles_agree():
    p = gi.cube_scene(300, seed=9, stride=320)
    c = Camera(**gi.identity_camera(96, 80, 96.0))
    tg = gi.uniform_target(96, 80, 2)
    L32, g32, r32 = oracle.loss_and_grad(p, [c], [tg], prec="f32", n=300)
    L64, g64, r64 = oracle.loss_and_grad(p.astype(np.float64), [c], [tg.astype(np.float64)], prec="f64", n=300)
    assert abs(L32 - L64) < 1e-5
    ok = r32["outs"][0]["margin"] > 1e-3
    assert np.abs(r32["outs"][0]["image"] - r64["outs"][0]["image"])[:, ok].max() < 1e-4


# ------------------------------------------------------------------------------------------
# The rounding scale of the blend backward (used by the GPU parity bounds): the sum of the
# magnitudes of every product entering each 2D gradient.  Pinned by a one-term case (closed form),
# by the triangle inequality and the term count, and by the rounding it bounds:
# the fp32 backward's error against the fp64 backward on the same records lies within
# gamma_k x magnitude (k = terms + the longest per-pixel chain + 16 roundings per term).
# ------------------------------------------------------------------------------------------
def test_backward_magnitude_single_term_equals_abs_gradient():
    p = blank(1)
    p[0:3, 0] = [0.0, 0.0, 3.0]  # on the optical axis: J diagonal, so the axis-aligned conic has b = 0
    p[3:6, 0] = [math.log(0.01), math.log(0.02), math.log(0.015)]
    p[10, 0] = 0.4
    p[11:14, 0] = [0.7, 0.2, 0.4]
    c = cam(1, 1, 100.0, cx=0.3, cy=-0.2)  # the one pixel (0, 0) sits off the mean: dx, dy != 0
    r = oracle.render(p, [c], prec="f64", n=1)
    assert r["outs"][0]["gp"][0, 0] == 1 and abs(r["rec"]["conic"][0, 1]) < 1e-15
    L = r["lists"]
    d = np.array([0.3, 0.1, 0.2]).reshape(3, 1, 1)  # positive: no sign mixing across channels
    g = np.zeros((1, 9))
    oracle.blend_backward((1, 1), 0, L["ranges"], L["vals"], r["rec"], d, g, prec="f64")
    mag = np.zeros((1, 9))
    terms = np.zeros(1, np.uint32)
    oracle.blend_backward_magnitude((1, 1), 0, L["ranges"], L["vals"], r["rec"], d, mag, terms, prec="f64")
    assert terms[0] == 1
    # colour entries: one product each, the magnitude is |gradient|; the entries through alpha also
    # carry the colour behind at the scale of the pixel's colour c alpha T (T = 1 in front), so
    # d alpha's magnitude is dC c (1 + alpha / (1 - alpha)) = |d alpha| / (1 - alpha)
    alpha = 1.0 - r["outs"][0]["T"][0, 0]
    assert np.allclose(mag[0, 6:], np.abs(g[0, 6:]), rtol=1e-14, atol=0)
    assert np.allclose(mag[0, :6], np.abs(g[0, :6]) / (1 - alpha), rtol=1e-13, atol=0) and (mag[0, :2] > 0).all()


def test_backward_magnitude_bounds_fp32_rounding():
    u = 2.0 ** -24
    p = gi.cube_scene(300, seed=10, stride=320)
    c = Camera(**gi.identity_camera(96, 80, 96.0))
    r = oracle.render(p, [c], prec="f32", n=300)
    o = r["outs"][0]
    assert o["margin"].min() > 1e-4  # no threshold tie: fp32 and fp64 blend the same pairs
    L = r["lists"]
    d = np.random.default_rng(10).normal(size=(3, 80, 96)).astype(np.float32) * 1e-4
    rec64 = {k: v.astype(np.float64) for k, v in r["rec"].items()}
    g32 = np.zeros((300, 9), np.float32)
    oracle.blend_backward((96, 80), 0, L["ranges"], L["vals"], r["rec"], d, g32, prec="f32")
    g64 = np.zeros((300, 9))
    oracle.blend_backward((96, 80), 0, L["ranges"], L["vals"], rec64, d.astype(np.float64), g64, prec="f64")
    mag = np.zeros((300, 9))
    terms = np.zeros(300, np.uint32)
    oracle.blend_backward_magnitude((96, 80), 0, L["ranges"], L["vals"], rec64, d.astype(np.float64), mag, terms,
                                    prec="f64")
    assert int(terms.sum()) == int(o["gp"].astype(np.int64).sum())
    assert (mag >= np.abs(g64) * (1 - 1e-12)).all()
    mag_neg = np.zeros((300, 9))
    oracle.blend_backward_magnitude((96, 80), 0, L["ranges"], L["vals"], rec64, -d.astype(np.float64), mag_neg,
                                    np.zeros(300, np.uint32), prec="f64")
    assert np.array_equal(mag, mag_neg)
    k = terms[:, None].astype(np.float64) + float(o["gp"].max()) + 16
    gamma = k * u / (1 - k * u)
    assert (np.abs(g32 - g64) <= gamma * mag).all()
    # and the bound is not vacuous: cancellation makes |g| much smaller than the scale somewhere
    assert (np.abs(g64) < 0.1 * mag).any()


def test_chain_magnitude_closed_forms():
    """One Gaussian on the optical axis, camera centre at the origin: the view direction is exactly
    +z, so the SH products are c0, c1 z, c2b (2 z z - x x - y y), c3d z (2 z z - 3 x x - 3 y y) with
    x = y = 0: the SH rows' magnitudes are |dcol| x (c0, c1, 2 c2b, 2 c3d) for k = 0, 2, 6, 12 and 0
    for the other coefficients; the opacity row g2[5] o (1 - o) has magnitude |g2[5]| o (1 + o)."""
    p = blank(1, dtype=np.float64)
    p[2, 0] = 3.0
    p[3:6, 0] = math.log(0.05)
    p[10, 0] = 0.3
    p[11:14, 0] = 0.2
    c = cam(32, 32, 40.0)
    g2 = np.array([[0.1, -0.2, 0.3, 0.05, -0.4, 0.7, 0.25, -0.5, 0.125]])
    mag = np.zeros((59, 32))
    oracle.project_backward_magnitude(p, c, g2, mag, n=1)
    pi = math.pi
    mY = np.zeros(16)
    mY[0] = 0.5 / math.sqrt(pi)
    mY[2] = math.sqrt(3 / (4 * pi))
    mY[6] = 2 * 0.25 * math.sqrt(5 / pi)
    mY[12] = 2 * 0.25 * math.sqrt(7 / pi)
    for k in range(16):
        for ch in range(3):
            assert mag[11 + 3 * k + ch, 0] == pytest.approx(abs(g2[0, 6 + ch]) * mY[k], rel=1e-14, abs=1e-300)
    o = 1 / (1 + math.exp(-0.3))
    assert mag[10, 0] == pytest.approx(0.7 * o * (1 + o), rel=1e-14)


def test_chain_magnitude_bounds_fp32_rounding():
    u = 2.0 ** -24
    p = gi.cube_scene(2000, seed=3, stride=2016, logscale=(-2.5, 0.5))
    p[11, ::7] = -3.0  # some clamped colour channels
    c = Camera(**gi.identity_camera(96, 80, 96.0))
    g2 = np.random.default_rng(0).normal(size=(2016, 9)).astype(np.float32)
    g32 = np.zeros((59, 2016), np.float32)
    oracle.project_backward(p, c, g2, g32, prec="f32", n=2000)
    g64 = np.zeros((59, 2016))
    oracle.project_backward(p.astype(np.float64), c, g2.astype(np.float64), g64, prec="f64", n=2000)
    mag = np.zeros((59, 2016))
    oracle.project_backward_magnitude(p, c, g2, mag, n=2000)
    assert (mag >= np.abs(g64) * (1 - 1e-12)).all()
    k = 64
    assert (np.abs(g32 - g64) <= k * u / (1 - k * u) * mag).all()
    assert (np.abs(g64) < 0.01 * mag).sum() > 1000  # cancellation: relative bounds alone would not hold


# ------------------------------------------------------------------------------------------
# Load balancing (Eq. 9-10).  L_load = std of G_p over the pixels with G_p > 0; the count's derivative
# is taken through the soft count, the sum of the blended Gaussians' alphas.  Pinned by finite differences: of the standard deviation (its weights dL/dG_p), and of
# the frozen-weight functional sum_p w_p soft_p(theta) through the whole projection, in fp64.
# ------------------------------------------------------------------------------------------
def test_load_weights_are_the_derivative_of_the_standard_deviation():
    rng = np.random.default_rng(3)
    gps = [rng.integers(0, 9, size=(5, 7)).astype(np.float64), rng.integers(0, 4, size=(3, 4)).astype(np.float64)]
    lam = 0.41
    w = oracle.load_weights(gps, lam)
    flat = np.concatenate([g.reshape(-1) for g in gps])
    vis = flat > 0

    def f(x):
        return lam * np.std(x[vis])

    wf = np.concatenate([x.reshape(-1) for x in w])
    h = 1e-6
    for i in np.nonzero(vis)[0][:20]:
        e = np.zeros_like(flat)
        e[i] = h
        assert (f(flat + e) - f(flat - e)) / (2 * h) == pytest.approx(wf[i], rel=1e-6, abs=1e-10)
    assert (wf[~vis] == 0).all()
    assert oracle.load_term(gps) * lam == pytest.approx(f(flat), rel=1e-15)
    assert oracle.load_std(gps) == pytest.approx(np.std(flat[vis]), rel=1e-15)
    # a uniform count has no spread and no gradient
    same = [np.where(g > 0, 3.0, 0.0) for g in gps]
    assert all((x == 0).all() for x in oracle.load_weights(same, lam)) and oracle.load_term(same) == 0.0


def test_load_gradient_matches_finite_differences_of_the_soft_count():
    p, cams = _scene("two_views")
    n = 5
    rng = np.random.default_rng(4)
    ws = [rng.normal(size=(c.height, c.width)) for c in cams]

    def phi(q):
        r = oracle.render(q, cams, prec="f64", n=n)
        L = r["lists"]
        return sum(float((ws[v] * oracle.blend_soft_count((c.width, c.height), L["tile_base"][v], L["ranges"],
                                                          L["vals"], r["rec"], prec="f64")).sum())
                   for v, c in enumerate(cams)), r

    _, r0 = phi(p)
    L = r0["lists"]
    g2 = np.zeros((len(cams) * n, 9))
    for v, c in enumerate(cams):
        oracle.blend_backward((c.width, c.height), L["tile_base"][v], L["ranges"], L["vals"], r0["rec"],
                              np.zeros((3, c.height, c.width)), g2, prec="f64", load_w=ws[v])
    g = np.zeros_like(p)
    for v, c in enumerate(cams):
        oracle.project_backward(p, c, g2[v * n:(v + 1) * n], g, prec="f64", n=n)
    assert np.abs(g[:, :n]).max() > 0
    eps = 1e-6
    keys = ("last", "gp", "neval")
    checked = 0
    for i in range(n):
        for c in list(range(11)) + [11, 12, 13]:
            vals, same = [], True
            for sgn in (1, -1):
                q = p.copy()
                q[c, i] += sgn * eps
                val, rq = phi(q)
                vals.append(val)
                same &= all((rq["outs"][v][k] == r0["outs"][v][k]).all() for v in range(len(cams)) for k in keys)
            if not same:
                continue
            fd = (vals[0] - vals[1]) / (2 * eps)
            assert abs(fd - g[c, i]) <= 1e-6 * max(abs(fd), abs(g[c, i])) + 1e-9, (i, c, fd, g[c, i])
            checked += 1
    assert checked > 40
    # the colour rows take no gradient from the count (s depends on alpha only)
    assert (g[11:, :n] == 0).all()


# ------------------------------------------------------------------------------------------
# Schedule (Eq. 3-8): a hand-computed example and invariants.
# ------------------------------------------------------------------------------------------
def test_schedule_hand_example():
    gd = _golden("schedule_small.txt")
    tracks = [range(1, 11), range(6, 16), range(11, 21), range(16, 26), range(30, 36)]
    M = sch.overlap_matrix(tracks)
    w, layer = sch.hierarchical_weights(M, 3)
    assert np.allclose(w, [float(x) for x in gd["weights"]], atol=1e-15)
    keys, iters, slots = sch.allocate(w, 3, 20, list(range(5)), 3, seed=0)
    assert keys == [3, 2, 1]
    assert [iters[i] for i in range(5)] == [int(x) for x in gd["iterations"]]
    assert sorted(slots) == sorted(sum(([i] * iters[i] for i in range(5)), []))
    T = [200, 100, 50, 0, 0]
    assert abs(sch.lr_image(3, M, T, 200, 1.6e-4, 1.6e-6) - float(gd["lr_image3"][0])) < 1e-11
    assert abs(sch.lr_image(1, M, T, 200, 1.6e-4, 1.6e-6) - float(gd["lr_image1"][0])) < 1e-11


def test_schedule_invariants():
    rng = np.random.default_rng(0)
    for trial in range(20):
        n = int(rng.integers(2, 15))
        tracks = [set(rng.integers(0, 60, int(rng.integers(5, 25))).tolist()) for _ in range(n)]
        M = sch.overlap_matrix(tracks)
        new = n - 1
        w, layer = sch.hierarchical_weights(M, new)
        assert w[new] == 1.0 and np.all(w <= 1.0 + 1e-12)
        keys, iters, slots = sch.allocate(w, 4, 200, list(range(n)), new, seed=trial)
        assert len(slots) == 200
        if len(keys) < n:
            assert sum(iters[i] for i in keys) == 100          # Eq. 5 sums to T_I / 2
            others = [i for i in range(n) if i not in keys]
            cnts = [iters[i] for i in others]
            assert max(cnts) - min(cnts) <= 1                    # evenly spread
        # more weight never means fewer Eq. 5 iterations
        ks = sorted(keys, key=lambda i: -w[i])
        if len(keys) < n:
            assert all(iters[a] >= iters[b] - 1 for a, b in zip(ks, ks[1:]))
    # t = 1 once T_j > T_a (Eq. 7) and the rate is then etaf
    assert sch.lr_current(201, 200, 1.6e-4, 1.6e-6) == pytest.approx(1.6e-6, rel=1e-12)
    assert sch.lr_current(0, 200, 1.6e-4, 1.6e-6) == pytest.approx(1.6e-4, rel=1e-12)
    # the rate falls as the image is trained (Sec. IV-C)
    rates = [sch.lr_current(t, 200, 1.6e-4, 1.6e-6) for t in range(0, 250, 10)]
    assert all(a >= b for a, b in zip(rates, rates[1:]))


# ---------------------------------------------------------------------------------------------
# 3DGS adaptive density control (oracle/densify.py)
# ---------------------------------------------------------------------------------------------
def test_splitmix64_published_vector():
    """SplitMix64 seeded with 1234567: the first five outputs of the published reference."""
    from oracle import densify as dn
    from oracle import schedule as sch
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
           16408922859458223821]
    assert [dn.splitmix64_hash((1234567 + k * dn.GOLDEN) % (1 << 64)) for k in range(5)] == ref
    r = sch.SplitMix64(1234567)
    assert [r.next() for _ in range(5)] == ref


def test_densify_normals_are_standard():
    from oracle import densify as dn
    z = np.array([dn.normal(3, 1, i, c, a) for i in range(2000) for c in range(2) for a in range(3)], np.float64)
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1.0) < 0.03
    assert abs(np.mean(z ** 4) - 3.0) < 0.2  # Gaussian kurtosis


def test_view_space_norm_closed_form():
    from oracle import densify as dn
    assert dn.view_space_norm(3.0 / 960.0, 4.0 / 540.0, 1920, 1080) == pytest.approx(5.0, rel=1e-6)


def test_densify_hand_example():
    """Four Gaussians, extent 10 (clone limit log 0.1, prune limit log 1.0): A hot and small (clone),
    B hot and large and rotated 90 degrees about z (split), C cold and transparent (pruned), D cold
    and huge (pruned).  Output: A, A's clone, B's two children; only A keeps its moments."""
    from oracle import densify as dn
    n = 4
    p = np.zeros((59, n), np.float32)
    p[0:3] = [[0, 1, 2, 3], [0, 0, 0, 0], [5, 5, 5, 5]]
    p[3:6, 0] = np.log(0.05)
    p[3:6, 1] = np.log([0.5, 0.2, 0.1])
    p[3:6, 2] = np.log(0.05)
    p[3:6, 3] = np.log(2.0)
    p[6, :] = 1.0
    c45 = np.float32(np.sqrt(0.5))
    p[6, 1], p[9, 1] = c45, c45  # 90 degrees about z: (x, y, z) -> (-y, x, z)
    p[10, :] = 2.0
    p[10, 2] = -8.0  # opacity 3.4e-4 < 0.005
    p[11:59] = 0.1
    m = np.full_like(p, 0.5)
    v = np.full_like(p, 0.25)
    accum = np.array([3e-3, 3e-3, 1e-5, 1e-5], np.float32)
    count = np.array([10, 10, 10, 10], np.float32)
    P, M, V, info = dn.densify(p, m, v, n, accum, count, extent=10.0, seed=7, rnd=2)
    assert info == dict(cloned=1, split=1, pruned=2, kept=1, n=4)
    assert np.array_equal(P[:, 0], p[:, 0]) and np.array_equal(P[:, 1], p[:, 0])
    assert np.all(M[:, 0] == 0.5) and np.all(V[:, 0] == 0.25)
    assert np.all(M[:, 1:] == 0) and np.all(V[:, 1:] == 0)
    s = np.array([0.5, 0.2, 0.1])
    for c in range(2):
        z = np.array([float(dn.normal(7, 2, 1, c, a)) for a in range(3)])
        local = s * z
        expect = np.array([1.0, 0.0, 5.0]) + np.array([-local[1], local[0], local[2]])
        assert np.allclose(P[0:3, 2 + c], expect, atol=1e-5)
        assert np.allclose(P[3:6, 2 + c], np.log(s / 1.6), atol=1e-6)
        assert np.array_equal(P[6:59, 2 + c], p[6:59, 1])
