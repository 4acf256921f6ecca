"""The oracle of the adaptive density control of the original 3DGS -- TEST INFRASTRUCTURE ONLY.

On-the-Fly GS keeps "all other settings" of 3DGS (Sec. V-A); the field grows by the update of
Sec. IV-B, and 3DGS's densification and pruning are the optional further step restated here
(3DGS, Kerbl et al. 2023, Sec. 5.2 "adaptive control of Gaussians").  Readings where that text is
silent (the kernels follow the same ones):

* statistics, per optimisation step and per view in which the Gaussian has instances: the norm of
  its view-space mean gradient, the pixel-space gradient scaled by (W / 2, H / 2) (the NDC
  derivative), accumulated with a count;
* a Gaussian whose mean accumulated norm (sum / count, 0 without views) is >= grad_thresh is
  cloned when its largest scale is <= percent_dense x extent, split otherwise; a split replaces
  it by 2 children at mean + R(q) (s * z), z standard normal, with every log-scale lowered by
  log(1.6) and everything else copied; clones copy everything;
* every resulting Gaussian (kept original, clone, child) with opacity < min_opacity or largest
  scale > max_scale x extent is pruned (3DGS resets its screen-space radii when it densifies, so
  no screen-size test applies);
* order: kept originals, then clones, then children (by original, child 0 before child 1); the
  Adam moments of clones and children are 0, the kept originals keep theirs;
* the decisions compare log-scales and opacity logits against thresholds taken to the log / logit
  domain in float64 from the float32 settings and extent, then rounded to float32, so both sides
  decide on the same float32 values;
* the normals z: for split round r, original i, child c, axis a: k = (2 i + c) 3 + a, two
  SplitMix64 outputs h(base + 2k), h(base + 2k + 1) with base = seed ^ (r * 0x9E3779B97F4A7C15)
  give u1 = ((h1 >> 11) + 1) / 2^53, u2 = (h2 >> 11) / 2^53 and z = sqrt(-2 ln u1) cos(2 pi u2)
  (Box-Muller), in float64, then float32.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64_hash(x: int) -> int:
    """One SplitMix64 output for state x (Vigna's published finaliser after the increment)."""
    z = (x + GOLDEN) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def normal(seed: int, rnd: int, i: int, c: int, a: int) -> np.float32:
    base = (seed ^ ((rnd * GOLDEN) & _M64)) & _M64
    k = (2 * i + c) * 3 + a
    h1 = splitmix64_hash((base + 2 * k) & _M64)
    h2 = splitmix64_hash((base + 2 * k + 1) & _M64)
    u1 = ((h1 >> 11) + 1) * 2.0 ** -53
    u2 = (h2 >> 11) * 2.0 ** -53
    return np.float32(math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2))


def view_space_norm(gx, gy, W, H):
    """float32 norm of the pixel-space mean gradient scaled to NDC (W / 2, H / 2)."""
    gx = np.float32(gx) * np.float32(0.5 * W)
    gy = np.float32(gy) * np.float32(0.5 * H)
    return np.sqrt(np.float32(gx * gx + gy * gy), dtype=np.float32)


def quat_to_rot(q):
    w, x, y, z = (float(v) for v in q)
    n = math.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / n, x / n, y / n, z / n
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def thresholds(extent, grad_thresh=2e-4, percent_dense=0.01, min_opacity=0.005, max_scale=0.1):
    # the settings and the extent are float32 values; the products and logs are taken in float64
    f = lambda x: float(np.float32(x))
    extent, percent_dense, min_opacity, max_scale = f(extent), f(percent_dense), f(min_opacity), f(max_scale)
    return dict(grad=np.float32(grad_thresh),
                ls_dense=np.float32(math.log(percent_dense * extent)),
                ls_big=np.float32(math.log(max_scale * extent)),
                logit_min=np.float32(math.log(min_opacity / (1.0 - min_opacity))),
                ls_shrink=np.float32(math.log(1.6)))


def densify(params, m, v, n, accum, count, extent, seed=0, rnd=0, **kw):
    """params, m, v: (59, >= n) float32; accum, count: (>= n,) float32.  Returns (params', m', v',
    info) with n' columns and info = dict(cloned, split, pruned, kept)."""
    th = thresholds(extent, **kw)
    P = np.asarray(params, np.float32)[:, :n]
    Mo = np.asarray(m, np.float32)[:, :n]
    Vo = np.asarray(v, np.float32)[:, :n]
    acc = np.asarray(accum, np.float32)[:n]
    cnt = np.asarray(count, np.float32)[:n]
    g = np.where(cnt > 0, acc / np.where(cnt > 0, cnt, np.float32(1)), np.float32(0)).astype(np.float32)
    maxls = P[3:6].max(axis=0)
    hot = g >= th["grad"]
    clone = hot & (maxls <= th["ls_dense"])
    split = hot & (maxls > th["ls_dense"])

    def pruned(col):
        return bool(col[10] < th["logit_min"]) or bool(col[3:6].max() > th["ls_big"])

    outP, outM, outV = [], [], []
    info = dict(cloned=0, split=int(split.sum()), pruned=0, kept=0)
    for i in range(n):  # kept originals
        if split[i]:
            continue
        if pruned(P[:, i]):
            info["pruned"] += 1
            continue
        outP.append(P[:, i].copy()); outM.append(Mo[:, i].copy()); outV.append(Vo[:, i].copy())
        info["kept"] += 1
    zero = np.zeros(59, np.float32)
    for i in range(n):  # clones
        if clone[i]:
            if pruned(P[:, i]):
                info["pruned"] += 1
                continue
            outP.append(P[:, i].copy()); outM.append(zero.copy()); outV.append(zero.copy())
            info["cloned"] += 1
    for i in range(n):  # children
        if not split[i]:
            continue
        R = quat_to_rot(P[6:10, i])
        s = np.exp(P[3:6, i].astype(np.float64))
        for c in range(2):
            z = np.array([normal(seed, rnd, i, c, a) for a in range(3)], np.float64)
            col = P[:, i].copy()
            col[0:3] = (P[0:3, i].astype(np.float64) + R @ (s * z)).astype(np.float32)
            col[3:6] = (P[3:6, i] - th["ls_shrink"]).astype(np.float32)
            if pruned(col):
                info["pruned"] += 1
                continue
            outP.append(col); outM.append(zero.copy()); outV.append(zero.copy())
    k = len(outP)
    stack = (lambda L: np.stack(L, axis=1) if L else np.zeros((59, 0), np.float32))
    return stack(outP), stack(outM), stack(outV), dict(info, n=k)
