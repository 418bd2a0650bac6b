"""Zero level set of the fused field as a triangle mesh (Sec. 3.3: marching
cubes on the result; test infrastructure, see ``oracle``).

The leaf field is sampled at every finest-voxel centre (each voxel takes the
value of the leaf containing it).  The cubes have eight neighbouring voxel
centres as corners; a vertex lies on each cube edge whose end values have
opposite signs (u < 0 counts as inside, u >= 0 as outside), placed by linear
interpolation.  Instead of a case table, each cube's surface is derived from
its six faces:

* on every face (corners in counter-clockwise order seen from outside the
  cube) each contour segment runs from a crossing where the boundary walk
  goes from outside to inside to the next crossing along the walk, which
  keeps the outside on the segment's left and, on a face with four crossings,
  separates the inside corners; both cubes sharing a face see the same
  segments, so the mesh has no holes;
* every crossing point starts one segment (in one of its two faces) and ends
  one (in the other), so the segments form closed loops; each loop is fanned
  into triangles, whose normals then point to the outside (u >= 0).

Vertices are shared between cubes (one per crossed grid edge).
"""
from __future__ import annotations

import numpy as np

from . import morton

# corner c of a cube: offsets (c & 1, c >> 1 & 1, c >> 2 & 1)
_OFF = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)])


def _faces():
    """Six faces as corner lists, counter-clockwise seen from outside."""
    out = []
    for axis in range(3):
        t1, t2 = [a for a in range(3) if a != axis]
        for side in (0, 1):
            ring = []
            for a, b in ((0, 0), (1, 0), (1, 1), (0, 1)):
                off = [0, 0, 0]
                off[axis], off[t1], off[t2] = side, a, b
                ring.append(off[0] + 2 * off[1] + 4 * off[2])
            n = np.zeros(3)
            n[axis] = 1.0 if side else -1.0
            p = _OFF[ring].astype(float)
            if np.dot(np.cross(p[1] - p[0], p[2] - p[1]), n) < 0:
                ring = ring[::-1]
            out.append(ring)
    return out


FACES = _faces()


def fine_field(keys, levels, u, dmax) -> np.ndarray:
    """[n, n, n] array of the leaf values at every finest voxel (x, y, z)."""
    n = 1 << dmax
    g = np.empty((n, n, n))
    x, y, z = morton.decode(keys, dmax)
    h = morton.edge(levels, dmax)
    for i in range(len(keys)):
        g[x[i]:x[i] + h[i], y[i]:y[i] + h[i], z[i]:z[i] + h[i]] = u[i]
    return g


def extract(grid, origin=(0.0, 0.0, 0.0), spacing=1.0):
    """Triangles of the zero level set of `grid` (values at the points
    origin + (i + 0.5) * spacing).  Returns (vertices [V, 3], triangles [T, 3])."""
    grid = np.asarray(grid, np.float64)
    neg = grid < 0
    n0, n1, n2 = grid.shape
    # cubes with corners of both signs
    c = np.zeros((n0 - 1, n1 - 1, n2 - 1), np.int32)
    for k in range(8):
        dx, dy, dz = _OFF[k]
        c += neg[dx:n0 - 1 + dx, dy:n1 - 1 + dy, dz:n2 - 1 + dz].astype(np.int32)
    cubes = np.argwhere((c > 0) & (c < 8))
    org = np.asarray(origin, np.float64)
    vid = {}
    verts = []
    tris = []

    def vertex(p, q):
        key = (tuple(p), tuple(q)) if tuple(p) < tuple(q) else (tuple(q), tuple(p))
        if key not in vid:
            a, b = grid[key[0]], grid[key[1]]
            t = a / (a - b)
            pos = np.array(key[0], float) + t * (np.array(key[1], float) - np.array(key[0], float))
            vid[key] = len(verts)
            verts.append(org + (pos + 0.5) * spacing)
        return vid[key]

    for base in cubes:
        corner = [tuple(base + _OFF[k]) for k in range(8)]
        inside = [bool(neg[cc]) for cc in corner]
        nxt = {}
        for ring in FACES:
            walk = [(ring[k], ring[(k + 1) % 4]) for k in range(4)]
            cross = [(i, j) for i, j in walk if inside[i] != inside[j]]
            if not cross:
                continue
            # crossings in walk order; starts: outside -> inside
            order = [(i, j) for i, j in walk if inside[i] != inside[j]]
            for s, (i, j) in enumerate(order):
                if not inside[i] and inside[j]:
                    i2, j2 = order[(s + 1) % len(order)]
                    nxt[vertex(corner[i], corner[j])] = vertex(corner[i2], corner[j2])
        seen = set()
        for start in nxt:
            if start in seen:
                continue
            loop = [start]
            seen.add(start)
            v = nxt[start]
            while v != start:
                loop.append(v)
                seen.add(v)
                v = nxt[v]
            for k in range(1, len(loop) - 1):
                tris.append((loop[0], loop[k], loop[k + 1]))
    return np.array(verts).reshape(-1, 3), np.array(tris, np.int64).reshape(-1, 3)


def leaf_mesh(keys, levels, u, dmax, origin, extent):
    """Mesh of the zero level set of a leaf field in world coordinates."""
    g = fine_field(keys, levels, u, dmax)
    return extract(g, origin, extent / (1 << dmax))


def edges(tris):
    """Directed edges (a, b) of every triangle, [3T, 2]."""
    t = np.asarray(tris)
    return np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])


def euler_characteristic(verts, tris) -> int:
    und = np.sort(edges(tris), axis=1)
    E = len(np.unique(und, axis=0))
    used = len(np.unique(np.asarray(tris).ravel()))
    return used - E + len(tris)
