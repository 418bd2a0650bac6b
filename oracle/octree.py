"""Linear octree: construction, face neighbours, split/join (test infrastructure).

Leaves are kept as two arrays sorted by Morton key (``keys`` uint64, ``levels``
uint8; level 0 is the root, D_max the finest voxel).
"""
from __future__ import annotations

import numpy as np

from . import morton, tsdf

# face order used everywhere: +x, +y, +z, -x, -y, -z
FACES = ((0, +1), (1, +1), (2, +1), (0, -1), (1, -1), (2, -1))


# ----------------------------------------------------------------------------
# construction (Sec. 3.1, "Octree construction", Eq. 2)


def dense_u0(scene_origin, extent, dmax, depth, intr, pose, delta, eta, chunk=1 << 20):
    """Initial field at every finest-voxel centre: the median of that voxel's
    observed Eq. 1 samples (-1 where nothing observes it).  Returned as a
    float64 array indexed [x, y, z].

    The paper builds its octrees top-down from dense TSDFs (Sec. 3.1); the
    initial structure of the iterate u* is not described, so it is read as the
    same construction applied to this median field."""
    n = 1 << dmax
    out = np.empty(n * n * n)
    lin = np.arange(n * n * n, dtype=np.int64)
    for s in range(0, lin.size, chunk):
        idx = lin[s:s + chunk]
        x, y, z = idx // (n * n), (idx // n) % n, idx % n
        keys = morton.encode(x, y, z, dmax)
        pts = tsdf.centres(keys, np.full(idx.size, dmax), scene_origin, extent, dmax)
        fs, W = tsdf.sorted_samples(tsdf.samples(pts, depth, intr, pose, delta, eta))
        out[s:s + chunk] = tsdf.median(fs, W)
    return out.reshape(n, n, n)


def spread(u0: np.ndarray, level: int, dmax: int) -> np.ndarray:
    """Eq. 2: s_f(n) = |max f - min f| over each level-`level` node, as a
    [m, m, m] array (m = 2^level) indexed by node coordinates."""
    m = 1 << level
    h = u0.shape[0] // m
    v = u0.reshape(m, h, m, h, m, h)
    return np.abs(v.max(axis=(1, 3, 5)) - v.min(axis=(1, 3, 5)))


def construct(u0: np.ndarray, dmax: int, tau: float = 0.1):
    """Top-down construction (Sec. 3.1): starting at the root, a node whose
    spread exceeds tau is divided into eight children, down to D_max.
    Returns (keys, levels) sorted by key."""
    keys, levels = [], []
    active = np.zeros((1, 3), np.int64)      # node coordinates at this level
    for level in range(dmax + 1):
        if level == dmax:
            split = np.zeros(len(active), bool)
        else:
            s = spread(u0, level, dmax)
            split = s[active[:, 0], active[:, 1], active[:, 2]] > tau
        leaf = active[~split]
        h = 1 << (dmax - level)
        keys.append(morton.encode(leaf[:, 0] * h, leaf[:, 1] * h, leaf[:, 2] * h, dmax))
        levels.append(np.full(len(leaf), level, np.uint8))
        par = active[split]
        kids = [par * 2 + np.array([i & 1, (i >> 1) & 1, (i >> 2) & 1]) for i in range(8)]
        active = np.concatenate(kids) if len(par) else np.zeros((0, 3), np.int64)
    keys = np.concatenate(keys)
    levels = np.concatenate(levels)
    o = np.argsort(keys, kind="stable")
    return keys[o], levels[o]


def check_tiling(keys, levels, dmax) -> bool:
    """Leaves are sorted, aligned, disjoint and cover the domain."""
    h3 = morton.edge(levels, dmax).astype(np.uint64) ** np.uint64(3)
    if len(keys) == 0:
        return False
    if np.any(keys % h3 != 0):
        return False
    ends = keys + h3
    return bool(keys[0] == 0 and np.all(ends[:-1] == keys[1:])
                and ends[-1] == np.uint64(1) << np.uint64(3 * dmax))


# ----------------------------------------------------------------------------
# face neighbours


def locate(keys, x, y, z, dmax) -> np.ndarray:
    """Index of the leaf containing each finest voxel (x, y, z)."""
    q = morton.encode(x, y, z, dmax)
    return np.searchsorted(keys, q, side="right") - 1


def neighbours(keys, levels, dmax):
    """Face-neighbour lists of every leaf, for the six faces in ``FACES``.

    The neighbours across a face are the leaves containing a finest voxel that
    touches the face from the outside; each list is ascending in leaf index
    (= key order).  An empty list is a domain boundary.  Returns a list of six
    CSR pairs (offsets int64 [N+1], indices int64)."""
    n = 1 << dmax
    N = len(keys)
    x, y, z = morton.decode(keys, dmax)
    h = morton.edge(levels, dmax)
    corner = np.stack([x, y, z], 1)
    out = []
    for axis, sgn in FACES:
        owners, found = [], []
        for hv in np.unique(h):
            sel = np.nonzero(h == hv)[0]
            a = np.arange(hv)
            j, k = np.meshgrid(a, a, indexing="ij")
            j, k = j.ravel(), k.ravel()
            pts = np.repeat(corner[sel], hv * hv, axis=0)
            o = [ax for ax in range(3) if ax != axis]
            pts[:, o[0]] += np.tile(j, len(sel))
            pts[:, o[1]] += np.tile(k, len(sel))
            pts[:, axis] += hv if sgn > 0 else -1
            ok = (pts[:, axis] >= 0) & (pts[:, axis] < n)
            own = np.repeat(sel, hv * hv)[ok]
            pts = pts[ok]
            owners.append(own)
            found.append(locate(keys, pts[:, 0], pts[:, 1], pts[:, 2], dmax))
        own = np.concatenate(owners)
        fnd = np.concatenate(found)
        pair = np.unique(own * np.int64(N) + fnd)
        own, fnd = pair // N, pair % N
        off = np.zeros(N + 1, np.int64)
        np.add.at(off, own + 1, 1)
        out.append((np.cumsum(off), fnd.astype(np.int64)))
    return out


def neighbours_bruteforce(keys, levels, dmax):
    """O(N^2) face-contact test: m touches l's face when their boxes meet on
    that face's plane with an overlap of positive area.  Same output format
    as :func:`neighbours`."""
    x, y, z = morton.decode(keys, dmax)
    h = morton.edge(levels, dmax)
    lo = np.stack([x, y, z], 1)
    hi = lo + h[:, None]
    N = len(keys)
    out = []
    for axis, sgn in FACES:
        o = [ax for ax in range(3) if ax != axis]
        lists = []
        for l in range(N):
            plane = hi[l, axis] if sgn > 0 else lo[l, axis]
            other = lo[:, axis] if sgn > 0 else hi[:, axis]
            touch = other == plane
            for ax in o:
                touch &= (np.minimum(hi[l, ax], hi[:, ax]) - np.maximum(lo[l, ax], lo[:, ax])) > 0
            lists.append(np.nonzero(touch)[0])
        off = np.zeros(N + 1, np.int64)
        off[1:] = np.cumsum([len(t) for t in lists])
        idx = np.concatenate(lists).astype(np.int64) if N else np.zeros(0, np.int64)
        out.append((off, idx))
    return out


# ----------------------------------------------------------------------------
# split / join (Sec. 3.2, "Optimization on the Octree")


def restructure(keys, levels, u, p, dmax, tau_s, tau_j):
    """One restructuring pass over the current iterate.

    Rules (Sec. 3.2): a leaf with |u| < tau_s is split, and since its
    children inherit the value the split recurses to D_max; an inner node is
    joined when it and, recursively, all its descendants hold |u| > tau_j with
    one common sign.  Taken top-down, the joined nodes are the maximal
    subtrees whose leaves all pass; the inner-node test itself is implied
    (a volume mean of values above tau_j with one sign is above tau_j).

    Value transfer: split children copy u and p; a joined leaf takes the
    h^3-weighted (volume) mean of u and of p, as the paper propagates means
    upwards (Sec. 3.1).

    u: float64 [N]; p: float64 [N, 3].  Decisions compare float64 values with
    float64 thresholds.  Returns (keys, levels, u, p, src, n_split, n_join):
    src[i] >= 0 is the old leaf a new leaf was kept from unchanged, -1 marks a
    new leaf (split child or joined node) whose samples must be re-integrated.
    """
    N = len(keys)
    h = morton.edge(levels, dmax)
    h3 = (h.astype(np.float64)) ** 3
    cls = np.where(u > tau_j, 1, np.where(u < -tau_j, -1, 0))
    pos = np.concatenate([[0], np.cumsum(cls == 1)])
    neg = np.concatenate([[0], np.cumsum(cls == -1)])

    # coarsest ancestor level whose whole key range is one joinable sign
    join_level = np.full(N, -1, np.int64)
    for L in range(dmax):
        size = np.uint64(1) << np.uint64(3 * (dmax - L))
        a = keys - (keys % size)
        lo = np.searchsorted(keys, a, side="left")
        hi = np.searchsorted(keys, a + size, side="left")
        cnt = hi - lo
        allpos = (pos[hi] - pos[lo]) == cnt
        allneg = (neg[hi] - neg[lo]) == cnt
        ok = (levels.astype(np.int64) > L) & (allpos | allneg) & (join_level < 0)
        join_level[ok] = L

    split = (levels.astype(np.int64) < dmax) & (np.abs(u) < tau_s)
    new_k, new_l, new_u, new_p, new_src = [], [], [], [], []
    n_split = n_join = 0
    i = 0
    while i < N:
        if join_level[i] >= 0:
            L = int(join_level[i])
            size = np.uint64(1) << np.uint64(3 * (dmax - L))
            a = keys[i] - keys[i] % size
            j = int(np.searchsorted(keys, a + size, side="left"))
            wsum = h3[i:j].sum()
            new_k.append(np.array([a], np.uint64))
            new_l.append(np.array([L], np.uint8))
            new_u.append(np.array([(h3[i:j] * u[i:j]).sum() / wsum]))
            new_p.append(((h3[i:j, None] * p[i:j]).sum(axis=0) / wsum)[None, :])
            new_src.append(np.array([-1]))
            n_join += 1
            i = j
        elif split[i]:
            cnt = int(h[i]) ** 3
            new_k.append(keys[i] + np.arange(cnt, dtype=np.uint64))
            new_l.append(np.full(cnt, dmax, np.uint8))
            new_u.append(np.full(cnt, u[i]))
            new_p.append(np.repeat(p[i:i + 1], cnt, axis=0))
            new_src.append(np.full(cnt, -1))
            n_split += 1
            i += 1
        else:
            new_k.append(keys[i:i + 1])
            new_l.append(levels[i:i + 1])
            new_u.append(u[i:i + 1])
            new_p.append(p[i:i + 1])
            new_src.append(np.array([i]))
            i += 1
    return (np.concatenate(new_k), np.concatenate(new_l), np.concatenate(new_u),
            np.concatenate(new_p), np.concatenate(new_src), n_split, n_join)


def restructure_recursive(keys, levels, u, dmax, tau_s, tau_j):
    """Second, independent reading of the split/join rules: an explicit
    pointer tree walked recursively from the root, as the paper's single pass
    does (Sec. 3.2).  Returns the new (keys, levels) only; used to cross-check
    :func:`restructure` on small trees."""
    x, y, z = morton.decode(keys, dmax)
    leaf_at = {}
    for i in range(len(keys)):
        leaf_at[(int(levels[i]), int(x[i]), int(y[i]), int(z[i]))] = float(u[i])

    def build(level, cx, cy, cz):
        key = (level, cx, cy, cz)
        if key in leaf_at:
            return {"leaf": True, "u": leaf_at[key], "level": level, "c": (cx, cy, cz)}
        hk = 1 << (dmax - level - 1)
        kids = [build(level + 1, cx + hk * (i & 1), cy + hk * ((i >> 1) & 1),
                      cz + hk * ((i >> 2) & 1)) for i in range(8)]
        return {"leaf": False, "kids": kids, "level": level, "c": (cx, cy, cz)}

    def joinable(node, sign):
        if node["leaf"]:
            return abs(node["u"]) > tau_j and (node["u"] > 0) == (sign > 0)
        return all(joinable(k, sign) for k in node["kids"])

    out = []

    def emit_split(level, c, value):
        if level == dmax or not abs(value) < tau_s:
            out.append((level, c))
            return
        hk = 1 << (dmax - level - 1)
        for i in range(8):
            emit_split(level + 1, (c[0] + hk * (i & 1), c[1] + hk * ((i >> 1) & 1),
                                   c[2] + hk * ((i >> 2) & 1)), value)

    def walk(node):
        if node["leaf"]:
            emit_split(node["level"], node["c"], node["u"])
            return
        for sign in (+1, -1):
            if joinable(node, sign):
                out.append((node["level"], node["c"]))
                return
        for k in node["kids"]:
            walk(k)

    walk(build(0, 0, 0, 0))
    lv = np.array([o[0] for o in out], np.uint8)
    c = np.array([o[1] for o in out], np.int64)
    k = morton.encode(c[:, 0], c[:, 1], c[:, 2], dmax)
    o = np.argsort(k)
    return k[o], lv[o]
