"""The oracle of the progressive schedule -- TEST INFRASTRUCTURE ONLY.

Plain Python restatement of Sec. IV-C/IV-D of On-the-Fly GS: the overlap matrix, hierarchical
image weighting (Eq. 3-4), Local & Semi-Global iteration allocation (Eq. 5) and the per-image
adaptive learning rate (Eq. 6-8).  Where the paper is silent this module takes these readings:

* overlap M[i, j] = (sparse-point tracks shared by i and j) / min(tracks of i, tracks of j);
* layers are breadth-first depths over the graph M > 0 from the new image; images the new image
  cannot reach get weight 0; in Eq. 4, M_{(k-1)j,ki} is M between image j of layer k-1 and image
  i of layer k;
* the key images are the N_m highest-weight images with positive weight (the new image, weight
  1, first), ties broken by lower image id;
* Eq. 5 is rounded by largest remainder so the key images receive exactly T_I / 2 iterations,
  equal remainders going to the lower image id;
* the semi-global half is split evenly over the other registered images; the T_I/2 mod n left
  over go to distinct images drawn by a partial Fisher-Yates shuffle; with no other image the
  whole T_I is split over the key images by Eq. 5's proportions;
* the order of the T_I view slots is a Fisher-Yates shuffle;
* random draws come from SplitMix64 (Steele, Lea and Flood, 2014; Vigna's published
  reference), seeded per arrival with seed XOR ((new_id + 1) * 0x9E3779B97F4A7C15 mod 2^64),
  and a draw in [0, k) is next() mod k.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _M64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def below(self, k: int) -> int:
        return self.next() % k


def arrival_rng(seed: int, new_id: int) -> SplitMix64:
    return SplitMix64((seed ^ (((new_id + 1) * 0x9E3779B97F4A7C15) & _M64)) & _M64)


def overlap_matrix(tracks):
    """M[i, j] from the sets of sparse-point track ids seen by each image (diagonal 0)."""
    n = len(tracks)
    M = np.zeros((n, n), np.float64)
    sets = [set(int(t) for t in tr) for tr in tracks]
    for i in range(n):
        for j in range(n):
            if i == j or not sets[i] or not sets[j]:
                continue
            M[i, j] = len(sets[i] & sets[j]) / min(len(sets[i]), len(sets[j]))
    return M


def hierarchical_weights(M, new):
    """Eq. 3-4.  Returns (weights, layer index per image, 0 = unreachable; the new image is 1)."""
    n = M.shape[0]
    w = np.zeros(n, np.float64)
    layer = np.zeros(n, np.int64)
    w[new] = 1.0
    layer[new] = 1
    prev = [new]
    k = 1
    while prev:
        k += 1
        nxt = sorted({i for j in prev for i in range(n) if layer[i] == 0 and M[j, i] > 0})
        for i in nxt:
            layer[i] = k
        for i in nxt:
            if k == 2:
                w[i] = w[new] * M[i, new]                                   # Eq. 3
            else:
                w[i] = sum(w[j] * M[j, i] for j in prev) / len(prev)        # Eq. 4
        prev = nxt
    return w, layer


def select_key_images(w, n_m):
    """The N_m images of highest positive weight, ordered by (weight desc, id asc)."""
    cand = [i for i in range(len(w)) if w[i] > 0]
    cand.sort(key=lambda i: (-w[i], i))
    return cand[:n_m]


def largest_remainder(shares, ids, total):
    """Integer split of ``total`` proportional to ``shares`` (sum exact, ties to lower id)."""
    s = float(sum(shares))
    exact = [total * x / s for x in shares]
    base = [int(math.floor(e)) for e in exact]
    left = total - sum(base)
    order = sorted(range(len(ids)), key=lambda k: (-(exact[k] - base[k]), ids[k]))
    for k in order[:left]:
        base[k] += 1
    return base


def allocate(w, n_m, T_I, registered, new, seed):
    """Eq. 5 plus the semi-global half.  Returns (key ids, {image: iterations}, slot order)."""
    keys = select_key_images(w, n_m)
    shares = [1.0 - math.exp(-w[i]) for i in keys]                       # Eq. 5 numerators
    others = sorted(i for i in registered if i not in set(keys))
    rng = arrival_rng(seed, new)
    iters = {}
    if others:
        for i, t in zip(keys, largest_remainder(shares, keys, T_I // 2)):
            iters[i] = t
        half = T_I - T_I // 2
        q, r = divmod(half, len(others))
        arr = list(others)
        for i in range(r):
            j = i + rng.below(len(arr) - i)
            arr[i], arr[j] = arr[j], arr[i]
        chosen = set(arr[:r])
        for i in others:
            iters[i] = q + (1 if i in chosen else 0)
    else:
        for i, t in zip(keys, largest_remainder(shares, keys, T_I)):
            iters[i] = t
    slots = []
    for i in sorted(iters):
        slots += [i] * iters[i]
    for i in range(len(slots) - 1, 0, -1):
        j = rng.below(i + 1)
        slots[i], slots[j] = slots[j], slots[i]
    return keys, iters, slots


def lr_current(Tj, T_a, eta0, etaf):
    """Eq. 6-7: log-linear decay from eta0 to etaf over the first T_a iterations of an image."""
    t = 1.0 if Tj > T_a else Tj / T_a
    return math.exp(math.log(eta0) * (1.0 - t) + math.log(etaf) * t)


def lr_image(j, M, T, T_a, eta0, etaf):
    """Eq. 8: image j's rate blended with its overlapping images' rates weighted by M."""
    n = M.shape[0]
    own = lr_current(T[j], T_a, eta0, etaf)
    acc, cnt = own, 0
    for i in range(n):
        if i != j and M[i, j] > 0:
            acc += M[i, j] * lr_current(T[i], T_a, eta0, etaf)
            cnt += 1
    return acc / (cnt + 1)
