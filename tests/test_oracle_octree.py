"""Pins of the oracle's octree construction, neighbours and split/join (no GPU)."""
import numpy as np
import pytest

from oracle import morton, octree
from tests._helpers import blocky_field, random_octree


def test_construct_constant_is_root():
    k, lv = octree.construct(np.zeros((8, 8, 8)), 3, 0.1)
    assert k.tolist() == [0] and lv.tolist() == [0]


def test_construct_single_spike_closed_form():
    """One deviating voxel forces a split along its path only: 7 D + 1 leaves."""
    for dmax in (2, 3, 4):
        n = 1 << dmax
        u0 = np.zeros((n, n, n))
        u0[n - 1, 1, 2] = 1.0
        k, lv = octree.construct(u0, dmax, 0.1)
        assert len(k) == 7 * dmax + 1
        assert np.bincount(lv, minlength=dmax + 1)[1:].tolist() == [7] * (dmax - 1) + [8]
        assert octree.check_tiling(k, lv, dmax)


@pytest.mark.parametrize("seed", range(4))
def test_construct_matches_definition(seed):
    """Every leaf is either finest or has spread <= tau, and its parent's
    spread exceeds tau (Eq. 2 split rule), checked voxel block by block."""
    dmax = 4
    n = 1 << dmax
    rng = np.random.default_rng(seed)
    u0 = np.clip(rng.normal(0, 1, (n, n, n)).cumsum(0) * 0.05, -1, 1)
    u0[:, :, : n // 2] = 1.0
    k, lv = octree.construct(u0, dmax, 0.1)
    assert octree.check_tiling(k, lv, dmax)
    x, y, z = morton.decode(k, dmax)
    for i in range(len(k)):
        h = 1 << (dmax - int(lv[i]))
        blk = u0[x[i]:x[i] + h, y[i]:y[i] + h, z[i]:z[i] + h]
        assert lv[i] == dmax or blk.max() - blk.min() <= 0.1
        if lv[i] > 0:
            H = 2 * h
            px, py, pz = x[i] // H * H, y[i] // H * H, z[i] // H * H
            par = u0[px:px + H, py:py + H, pz:pz + H]
            assert par.max() - par.min() > 0.1


@pytest.mark.parametrize("dmax,seed", [(3, 0), (3, 1), (4, 2), (4, 3), (4, 4)])
def test_neighbours_vs_bruteforce(dmax, seed):
    k, lv = random_octree(dmax, seed)
    a = octree.neighbours(k, lv, dmax)
    b = octree.neighbours_bruteforce(k, lv, dmax)
    for (oa, ia), (ob, ib) in zip(a, b):
        assert np.array_equal(oa, ob) and np.array_equal(ia, ib)


def test_neighbours_hand_case():
    """D_max = 2: root split once, the (0,0,0) child split again.  The coarse
    leaf at x = 2..4 sees four finest leaves across its -x face."""
    dmax = 2
    keys, levels = [], []
    for i in range(8):
        c = np.array([i & 1, (i >> 1) & 1, (i >> 2) & 1]) * 2
        if i == 0:
            for j in range(8):
                cc = c + np.array([j & 1, (j >> 1) & 1, (j >> 2) & 1])
                keys.append(morton.encode(*cc, dmax)); levels.append(2)
        else:
            keys.append(morton.encode(*c, dmax)); levels.append(1)
    o = np.argsort(keys)
    keys, levels = np.array(keys, np.uint64)[o], np.array(levels, np.uint8)[o]
    nb = octree.neighbours(keys, levels, dmax)
    coarse_x = int(np.searchsorted(keys, morton.encode(2, 0, 0, dmax)))
    off, idx = nb[3]  # -x
    got = idx[off[coarse_x]:off[coarse_x + 1]]
    expect = sorted(int(np.searchsorted(keys, morton.encode(1, y, z, dmax))) for y in (0, 1) for z in (0, 1))
    assert got.tolist() == expect
    fine = int(np.searchsorted(keys, morton.encode(1, 1, 0, dmax)))
    off, idx = nb[0]  # +x of a fine leaf: the coarse leaf
    assert idx[off[fine]:off[fine + 1]].tolist() == [coarse_x]
    off, idx = nb[3]  # -x of a fine leaf at x = 0: boundary
    f0 = int(np.searchsorted(keys, morton.encode(0, 0, 0, dmax)))
    assert off[f0 + 1] - off[f0] == 0


@pytest.mark.parametrize("dmax,seed", [(3, 0), (3, 5), (4, 1), (4, 2), (5, 3)])
def test_restructure_two_readings_agree(dmax, seed):
    k, lv = random_octree(dmax, seed, p_split=0.7, min_level=1)
    u = blocky_field(k, lv, dmax, seed)
    p = np.zeros((len(k), 3))
    nk, nl, nu, npp, src, ns, nj = octree.restructure(k, lv, u, p, dmax, 0.95, 0.99)
    rk, rl = octree.restructure_recursive(k, lv, u, dmax, 0.95, 0.99)
    assert np.array_equal(nk, rk) and np.array_equal(nl, rl)
    assert octree.check_tiling(nk, nl, dmax)
    assert ns > 0 and nj > 0


def test_restructure_invariants():
    dmax = 5
    k, lv = random_octree(dmax, 11, p_split=0.75, min_level=2)
    u = blocky_field(k, lv, dmax, 11)
    rng = np.random.default_rng(0)
    p = rng.uniform(-0.3, 0.3, (len(k), 3))
    nk, nl, nu, npp, src, ns, nj = octree.restructure(k, lv, u, p, dmax, 0.95, 0.99)
    h3 = morton.edge(lv, dmax).astype(float) ** 3
    nh3 = morton.edge(nl, dmax).astype(float) ** 3
    # volume means are conserved: integral of u and of p unchanged
    assert np.isclose((h3 * u).sum(), (nh3 * nu).sum(), rtol=1e-12)
    assert np.allclose((h3[:, None] * p).sum(0), (nh3[:, None] * npp).sum(0), rtol=1e-12)
    # a join never merges opposite signs: every old leaf under a joined leaf
    # shares its sign
    for i in np.nonzero(src < 0)[0]:
        if nl[i] < dmax:
            size = np.uint64(1) << np.uint64(3 * (dmax - int(nl[i])))
            sel = (k >= nk[i]) & (k < nk[i] + size)
            if sel.sum() > 1:
                assert np.all(np.sign(u[sel]) == np.sign(nu[i]))
                assert np.all(np.abs(u[sel]) > 0.99)
    # kept leaves keep values
    kept = src >= 0
    assert np.array_equal(nk[kept], k[src[kept]]) and np.array_equal(nu[kept], u[src[kept]])
    # a second pass on a saturated field is idempotent
    sat = np.sign(nu) * np.maximum(np.abs(nu), 1.0)
    a = octree.restructure(nk, nl, sat, npp, dmax, 0.95, 0.99)
    b = octree.restructure(a[0], a[1], a[2], a[3], dmax, 0.95, 0.99)
    assert np.array_equal(a[0], b[0]) and b[5] == 0 and b[6] == 0


def test_split_goes_to_finest():
    dmax = 3
    k, lv = np.array([0], np.uint64), np.array([0], np.uint8)
    nk, nl, nu, npp, src, ns, nj = octree.restructure(k, lv, np.array([0.2]), np.zeros((1, 3)), dmax, 0.95, 0.99)
    assert len(nk) == 512 and np.all(nl == dmax) and ns == 1
    assert np.array_equal(nk, np.arange(512, dtype=np.uint64))


def test_join_to_root():
    dmax = 2
    k = np.arange(64, dtype=np.uint64)
    lv = np.full(64, 2, np.uint8)
    u = np.full(64, -0.995)
    nk, nl, nu, npp, src, ns, nj = octree.restructure(k, lv, u, np.zeros((64, 3)), dmax, 0.95, 0.99)
    assert nk.tolist() == [0] and nl.tolist() == [0] and nj == 1
    u[5] = 0.995   # one opposite sign blocks the root and its octant
    nk, nl, *_ = octree.restructure(k, lv, u, np.zeros((64, 3)), dmax, 0.95, 0.99)
    assert len(nk) == 7 + 8 and np.sum(nl == 1) == 7


@pytest.mark.parametrize("name,seed,dmax", [("torus_box", 3, 4), ("at_scale", 5, 4), ("torus_box", 8, 5)])
def test_dense_u0_voxel_by_voxel(name, seed, dmax):
    """dense_u0[x, y, z] is the median of the Eq. 1 samples at the centre of
    finest voxel (x, y, z) (Sec. 3.1, Eq. 1), -1 where no frame observes it.

    The centre is written out directly from the voxel's integer coordinates
    (origin + (x + 1/2) * voxel edge, float32 as Eq. 1 is evaluated) rather
    than through Morton keys, and the median is NumPy's, so a swapped or
    reversed axis in the oracle's index arithmetic shows here.  The scenes
    have no symmetry under an exchange of axes, which the last assertions
    check, so a transposed field cannot pass by accident."""
    from oracle import tsdf
    from paper_1608_07411_gb300.scenes import make_scene
    sc = make_scene(name, seed, frames=10, width=96, height=72, max_depth=dmax)
    u0 = octree.dense_u0(sc.origin, sc.extent, dmax, sc.depth, sc.intr, sc.pose, sc.delta, sc.eta)
    n = 1 << dmax
    vox = np.float32(np.float32(sc.extent) / np.float32(n))
    ax = np.arange(n)
    gx, gy, gz = np.meshgrid(ax, ax, ax, indexing="ij")
    idx = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1)
    pts = np.empty(idx.shape, np.float32)
    for k in range(3):
        pts[:, k] = np.float32(sc.origin[k]) + (idx[:, k].astype(np.float32) + np.float32(0.5)) * vox
    f = tsdf.samples(pts, sc.depth, sc.intr, sc.pose, sc.delta, sc.eta)
    want = np.empty(len(idx))
    for i in range(len(idx)):
        obs = f[i][~np.isnan(f[i])]
        want[i] = np.median(obs) if obs.size else -1.0
    got = u0[idx[:, 0], idx[:, 1], idx[:, 2]]
    np.testing.assert_array_equal(got, want)
    # the field carries both signs and a band, and no axis exchange maps it to itself
    assert (want > 0.5).any() and (want < -0.5).any() and (np.abs(want) < 0.5).any()
    for perm in ((1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0)):
        assert not np.array_equal(u0, u0.transpose(perm)), perm
    assert not np.array_equal(u0, u0[::-1]) and not np.array_equal(u0, u0[:, :, ::-1])
