"""Pins of the per-frame TSDF octrees (Fig. 4 data term, Table 1 memory); no GPU."""
import numpy as np
import pytest

from oracle import frames, morton, octree, solver
from paper_1608_07411_gb300.scenes import make_scene

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _field(dmax, seed, frac_unseen=0.3):
    rng = np.random.default_rng(seed)
    n = 1 << dmax
    f = np.clip(rng.normal(0, 0.2, (n, n, n)).cumsum(0) / 3, -1, 1)
    f[rng.random((n, n, n)) < frac_unseen] = np.nan
    return f


def test_uniform_field_is_one_root():
    f = np.full((8, 8, 8), 0.75)
    t = frames.build(f, 3)
    assert len(t.keys) == 1 and t.levels[0] == 0 and t.nodes == 1
    fv, w = frames.lookup(t, np.array([0, 77], np.uint64), np.array([3, 2]))
    np.testing.assert_array_equal(fv, 0.75)
    assert w.all()
    t = frames.build(np.full((8, 8, 8), np.nan), 3)
    assert len(t.keys) == 1 and not frames.lookup(t, np.zeros(1, np.uint64), [0])[1][0]


@pytest.mark.parametrize("seed", range(3))
def test_construction_follows_the_rule(seed):
    """Leaves tile the domain; each leaf has one weight and, when observed, a
    spread <= tau; the parent of every leaf breaks one of the two."""
    D, tau = 4, 0.1
    f = _field(D, seed)
    t = frames.build(f, D, tau)
    assert octree.check_tiling(t.keys, t.levels, D)
    x, y, z = morton.decode(t.keys, D)
    h = morton.edge(t.levels, D)

    def ok(x0, y0, z0, hh):
        b = f[x0:x0 + hh, y0:y0 + hh, z0:z0 + hh]
        o = ~np.isnan(b)
        if o.all():
            return b.max() - b.min() <= tau
        return not o.any()

    for i in range(len(t.keys)):
        assert ok(x[i], y[i], z[i], h[i]) or h[i] == 1
        if t.levels[i] > 0:
            H = 2 * h[i]
            assert not ok(x[i] // H * H, y[i] // H * H, z[i] // H * H, H)
    assert t.nodes == len(t.keys) + (len(t.keys) - 1) // 7


def test_lookup_is_the_deepest_node_at_or_above_the_leaf_level():
    """Brute force: for a query leaf, walk its ancestors from its own level
    upwards; the first that is a node of the frame's tree gives the mean of
    the observed values in that node's box."""
    D = 4
    f = _field(D, 5)
    t = frames.build(f, D, 0.1)
    rng = np.random.default_rng(1)
    lv = rng.integers(0, D + 1, 300)
    h = 1 << (D - lv)
    c = rng.integers(0, 1 << D, (300, 3)) // h[:, None] * h[:, None]
    keys = morton.encode(c[:, 0], c[:, 1], c[:, 2], D)
    fv, w = frames.lookup(t, keys, lv)
    tree_nodes = set()
    for k, l in zip(t.keys, t.levels):           # every node: the leaves and all their ancestors
        x, y, z = (int(a[0]) for a in morton.decode(np.array([k]), D))
        for L in range(int(l) + 1):
            s = D - L
            tree_nodes.add((L, x >> s, y >> s, z >> s))
    for q in range(300):
        for L in range(int(lv[q]), -1, -1):
            s = D - L
            node = (L, c[q, 0] >> s, c[q, 1] >> s, c[q, 2] >> s)
            if node in tree_nodes:
                hh = 1 << s
                b = f[node[1] * hh:(node[1] + 1) * hh, node[2] * hh:(node[2] + 1) * hh,
                      node[3] * hh:(node[3] + 1) * hh]
                o = ~np.isnan(b)
                assert w[q] == o.any()
                if o.any():
                    assert abs(fv[q] - b[o].mean()) <= 1e-12
                break


def test_refined_frame_trees_give_the_leaf_centre_samples():
    """With tau < 0 every observed node of a frame's tree is split down to the
    finest voxels (unobserved regions stay leaves of weight 0), so a finest
    leaf's lookup is Eq. 1 at its centre: the leaf-centre integration of the
    main path."""
    s = make_scene("sphere", 4, frames=3, width=48, height=36, max_depth=4)
    n = 1 << s.max_depth
    rng = np.random.default_rng(2)
    c = rng.integers(0, n, (200, 3))
    keys = np.unique(morton.encode(c[:, 0], c[:, 1], c[:, 2], s.max_depth))
    lv = np.full(len(keys), s.max_depth, np.uint8)
    fs, W = frames.data_samples(s, keys, lv, tau=-1.0)
    fr, Wr = solver.leaf_samples(keys, lv, s, s.max_depth)
    np.testing.assert_array_equal(W, Wr)
    np.testing.assert_array_equal(np.nan_to_num(fs, nan=9.0), np.nan_to_num(fr, nan=9.0))


def test_memory_of_table_1():
    """Dense: two floats per voxel and frame -- the paper's 3,072 MB for 24
    frames at 256^3 (Table 1); octree: 84 bytes per node."""
    import json
    import os
    paper = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                        "paper_values.json")))["dense_tsdf_memory"]
    dmax = int(np.log2(paper["resolution"]))
    assert frames.memory_bytes([], paper["frames"], dmax)[0] == paper["mb"] * 2 ** 20
    t = frames.build(np.full((8, 8, 8), 0.5), 3)
    assert frames.memory_bytes([t, t], 2, 3) == (2 * 512 * 8, 2 * 84)
