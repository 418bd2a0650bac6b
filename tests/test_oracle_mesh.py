"""Pins of the oracle's level-set mesh (no GPU)."""
import numpy as np
import pytest

from oracle import mesh, morton, solver
from paper_1608_07411_gb300.scenes import make_scene


def _grid(f, n):
    i = np.arange(n) + 0.5
    x, y, z = np.meshgrid(i, i, i, indexing="ij")
    return f(x, y, z)


def _normals(v, t):
    return np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])


def _closed_and_oriented(t):
    """Every undirected edge in exactly two triangles, once in each direction."""
    d = mesh.edges(t)
    fwd = {tuple(e) for e in d}
    assert len(fwd) == len(d)                                   # no directed edge twice
    assert all((b, a) in fwd for a, b in d)                     # each has its reverse


@pytest.mark.parametrize("a", [(1.0, 0.3, -0.2), (0.0, 0.0, 1.0), (0.7, -0.7, 0.1)])
def test_plane_vertices_lie_on_the_plane(a):
    """Linear interpolation is exact for a linear field."""
    n, b = 12, -6.3
    g = _grid(lambda x, y, z: a[0] * x + a[1] * y + a[2] * z + b, n)
    v, t = mesh.extract(g)
    assert len(t) > 0
    np.testing.assert_allclose(v @ np.asarray(a) + b, 0.0, atol=1e-12)
    # normals point to the positive side, along a
    assert np.all(_normals(v, t) @ np.asarray(a) > 0)


def test_sphere_is_closed_genus_zero_and_outward():
    n, r0, c = 20, 6.2, 10.0
    g = _grid(lambda x, y, z: np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) - r0, n)
    v, t = mesh.extract(g)
    _closed_and_oriented(t)
    assert mesh.euler_characteristic(v, t) == 2
    d = np.linalg.norm(v - c, axis=1)
    # linear interpolation of |x| - r0 along a unit edge: error <= 1 / (2 r) per vertex
    assert np.max(np.abs(d - r0)) <= 1.0 / (2 * (r0 - 1))
    cen = v[t].mean(axis=1) - c
    assert np.all(np.einsum("ij,ij->i", _normals(v, t), cen) > 0)


def test_torus_has_euler_characteristic_zero():
    n, R, r, c = 28, 8.0, 3.1, 14.0
    def f(x, y, z):
        q = np.sqrt((x - c) ** 2 + (y - c) ** 2) - R
        return np.sqrt(q * q + (z - c) ** 2) - r
    v, t = mesh.extract(_grid(f, n))
    _closed_and_oriented(t)
    assert mesh.euler_characteristic(v, t) == 0


def test_saddle_faces_are_shared_consistently():
    """Checkerboard signs make every face ambiguous; the mesh still closes."""
    n = 6
    g = _grid(lambda x, y, z: np.where((np.floor(x) + np.floor(y) + np.floor(z)) % 2 == 0, 1.0, -1.0), n)
    g[0], g[-1], g[:, 0], g[:, -1], g[:, :, 0], g[:, :, -1] = 1, 1, 1, 1, 1, 1
    v, t = mesh.extract(g)
    _closed_and_oriented(t)


def test_fused_sphere_surface_accuracy():
    """The primal-dual result on the 8-view sphere: every vertex of the zero
    level set within two finest voxels of r = 0.4; a closed genus-0 surface."""
    s = make_scene("sphere", 1)
    st = solver.solve(s)
    v, t = mesh.leaf_mesh(st.keys, st.levels, st.u, s.max_depth, s.origin, s.extent)
    vox = s.extent / (1 << s.max_depth)
    d = np.abs(np.linalg.norm(v, axis=1) - 0.4)
    assert len(t) > 500 and d.max() <= 2 * vox and d.mean() <= 0.5 * vox
    _closed_and_oriented(t)
    assert mesh.euler_characteristic(v, t) == 2


def test_saddle_face_separates_inside_corners():
    """One cube whose x = 0 face has its two inside corners on a diagonal and
    every other corner outside: the stated rule cuts each inside corner off
    on its own (two triangles), not a band joining them across the face."""
    g = np.ones((2, 2, 2))
    g[0, 0, 0] = -1.0
    g[0, 1, 1] = -1.0
    v, t = mesh.extract(g)
    assert len(t) == 2 and len(v) == 6
    for corner in ((0.5, 0.5, 0.5), (0.5, 1.5, 1.5)):
        near = np.linalg.norm(v - np.array(corner), axis=1) <= 0.5 + 1e-12
        assert near.sum() == 3
