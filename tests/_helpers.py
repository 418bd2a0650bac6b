"""Test helpers: random octree structures and fields (inputs only)."""
import numpy as np

from oracle import morton


def random_octree(dmax, seed, p_split=0.55, min_level=0):
    """Random valid leaf set: each node splits with probability p_split
    (always above min_level).  Returns (keys, levels) sorted by key."""
    rng = np.random.default_rng(seed)
    out = []

    def rec(level, x, y, z):
        if level < dmax and (level < min_level or rng.random() < p_split):
            h = 1 << (dmax - level - 1)
            for i in range(8):
                rec(level + 1, x + h * (i & 1), y + h * ((i >> 1) & 1), z + h * ((i >> 2) & 1))
        else:
            out.append((level, x, y, z))

    rec(0, 0, 0, 0)
    lv = np.array([o[0] for o in out], np.uint8)
    c = np.array([o[1:] for o in out], np.int64)
    k = morton.encode(c[:, 0], c[:, 1], c[:, 2], dmax)
    o = np.argsort(k)
    return k[o], lv[o]


def blocky_field(keys, levels, dmax, seed):
    """A field with saturated regions of both signs and a band in between,
    so that split and join both happen."""
    rng = np.random.default_rng(seed)
    x, y, z = morton.decode(keys, dmax)
    h = morton.edge(levels, dmax)
    n = 1 << dmax
    c = (np.stack([x, y, z], 1) + 0.5 * h[:, None]) / n - 0.5
    r = np.sqrt((c * c).sum(1))
    u = np.clip((0.3 - r) * 6.0, -1, 1)
    mag = np.where(rng.random(len(u)) < 0.9, rng.uniform(0.991, 1.0, len(u)), rng.uniform(0.96, 0.99, len(u)))
    u = np.where(np.abs(u) > 0.9, np.sign(u) * mag, u)
    return u
