"""Per-frame TSDF octrees as the data-term source (Sec. 3.1, Fig. 4, Table 1;
test infrastructure, see ``oracle``).

The paper turns each frame's dense TSDF f_i into an octree f_i* with the
Eq. 2 rule, keeps in every node (inner nodes too) the mean of the values
below it, and evaluates the data term of an iterate leaf n at level L from
the node of f_i* at level L that covers n when the tree has one, else from
the leaf of f_i* that contains n (Fig. 4).  Readings where the paper is
silent:

* f_i and w_i are Eq. 1 at every finest-voxel centre (``tsdf.samples``);
* a node is split while its voxels do not all share one weight, or while
  they are all observed and the spread of f over them exceeds tau (Eq. 2),
  so every leaf has a single weight;
* a node's value is the mean of f over its observed voxels and its weight
  is 1 when it has any observed voxel (the paper's weights are binary);
* since a node exists only below split nodes, the Fig. 4 rule is: take the
  deepest node of f_i* on the path to n at a level <= L.

Memory (Table 1): a dense TSDF stores a distance and a weight per voxel and
frame (two 4-byte floats); an octree node stores pointers to its 8 children
and its parent and three floats (Sec. 4.3).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import morton, tsdf

DENSE_BYTES_PER_VOXEL = 2 * 4
NODE_BYTES = 9 * 8 + 3 * 4


@dataclasses.dataclass
class FrameTree:
    dmax: int
    keys: np.ndarray          # leaves, sorted by key
    levels: np.ndarray
    exists: list              # per level L: bool [m, m, m], node present in the tree
    mean: list                # per level L: mean of the observed f (NaN if none)
    seen: list                # per level L: any voxel observed

    @property
    def nodes(self) -> int:
        return int(sum(e.sum() for e in self.exists))


def frame_field(scene, i, dmax) -> np.ndarray:
    """f_i at every finest voxel, [n, n, n] indexed (x, y, z); NaN where w_i = 0."""
    n = 1 << dmax
    x, y, z = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    keys = morton.encode(x.ravel(), y.ravel(), z.ravel(), dmax)
    pts = tsdf.centres(keys, np.full(keys.size, dmax), scene.origin, scene.extent, dmax)
    f = tsdf.samples(pts, scene.depth[i:i + 1], scene.intr[i:i + 1], scene.pose[i:i + 1],
                     scene.delta, scene.eta)[:, 0]
    return f.reshape(n, n, n)


def build(f: np.ndarray, dmax: int, tau: float = 0.1) -> FrameTree:
    """The octree of one frame's field f ([n, n, n], NaN = unobserved)."""
    obs = ~np.isnan(f)
    val = np.where(obs, f, 0.0)
    lo_in = np.where(obs, f, np.inf)
    hi_in = np.where(obs, f, -np.inf)
    cnt, tot, lo, hi = [], [], [], []
    for L in range(dmax + 1):
        m = 1 << L
        h = f.shape[0] // m
        shape = (m, h, m, h, m, h)
        ax = (1, 3, 5)
        cnt.append(obs.reshape(shape).sum(axis=ax))
        tot.append(val.reshape(shape).sum(axis=ax))
        lo.append(lo_in.reshape(shape).min(axis=ax))
        hi.append(hi_in.reshape(shape).max(axis=ax))
    exists, mean, seen = [], [], []
    keys, levels = [], []
    active = np.zeros((1, 3), np.int64)
    for L in range(dmax + 1):
        m = 1 << L
        ex = np.zeros((m, m, m), bool)
        ex[active[:, 0], active[:, 1], active[:, 2]] = True
        exists.append(ex)
        with np.errstate(invalid="ignore", divide="ignore"):
            mean.append(np.where(cnt[L] > 0, tot[L] / cnt[L], np.nan))
        seen.append(cnt[L] > 0)
        full = (1 << (dmax - L)) ** 3
        c = cnt[L][active[:, 0], active[:, 1], active[:, 2]]
        mixed = (c > 0) & (c < full)
        wide = (c == full) & (hi[L][active[:, 0], active[:, 1], active[:, 2]]
                              - lo[L][active[:, 0], active[:, 1], active[:, 2]] > tau)
        split = (mixed | wide) if L < dmax else np.zeros(len(active), bool)
        leaf = active[~split]
        h = 1 << (dmax - L)
        keys.append(morton.encode(leaf[:, 0] * h, leaf[:, 1] * h, leaf[:, 2] * h, dmax))
        levels.append(np.full(len(leaf), L, np.uint8))
        par = active[split]
        kids = [par * 2 + np.array([k & 1, (k >> 1) & 1, (k >> 2) & 1]) for k in range(8)]
        active = np.concatenate(kids) if len(par) else np.zeros((0, 3), np.int64)
    keys = np.concatenate(keys)
    levels = np.concatenate(levels)
    o = np.argsort(keys, kind="stable")
    return FrameTree(dmax, keys[o], levels[o], exists, mean, seen)


def lookup(tree: FrameTree, keys, levels):
    """(f, w) of one frame for iterate leaves (keys, levels) by the Fig. 4 rule."""
    D = tree.dmax
    x, y, z = morton.decode(keys, D)
    lv = np.asarray(levels, np.int64)
    f = np.full(len(lv), np.nan)
    w = np.zeros(len(lv), bool)
    done = np.zeros(len(lv), bool)
    for L in range(D, -1, -1):               # deepest existing node at a level <= the leaf's
        s = D - L
        cx, cy, cz = x >> s, y >> s, z >> s
        sel = (~done) & (lv >= L)
        sel[sel] = tree.exists[L][cx[sel], cy[sel], cz[sel]]
        f[sel] = tree.mean[L][cx[sel], cy[sel], cz[sel]]
        w[sel] = tree.seen[L][cx[sel], cy[sel], cz[sel]]
        done |= sel
    return np.where(w, f, np.nan), w


def data_samples(scene, keys, levels, tau: float = 0.1):
    """Sorted per-leaf samples (NaN padded) and W from every frame's tree."""
    D = scene.max_depth
    cols = []
    for i in range(scene.depth.shape[0]):
        t = build(frame_field(scene, i, D), D, tau)
        cols.append(lookup(t, keys, levels)[0])
    return tsdf.sorted_samples(np.stack(cols, axis=1))


def memory_bytes(trees, frames: int, dmax: int):
    """(dense, octree) bytes of the data term: Table 1's two columns."""
    dense = frames * (8 ** dmax) * DENSE_BYTES_PER_VOXEL
    return dense, sum(t.nodes for t in trees) * NODE_BYTES
