"""The at-scale workload (5 seeded shapes in a 2 m scene, 100 views 640x480,
D_max = 9, millions of leaves): checks one leaf at a time against the oracle
and properties that hold at any size."""
import numpy as np
import pytest

from oracle import octree, tsdf
from paper_1608_07411_gb300 import octfuse
from paper_1608_07411_gb300.scenes import make_scene

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return octfuse.load()


def test_at_scale_workload():
    scene = make_scene("at_scale", 0)
    o = octfuse.Octree(octfuse.params_for(scene))
    o.integrate_frames(scene.depth, scene.intr, scene.pose)
    D = scene.max_depth
    k, lv, u0 = o.leaves()
    assert 1e6 < len(k) < 2e7
    assert octree.check_tiling(k, lv, D)
    # Eq. 1 samples of sampled leaves, bit for bit
    off = o.field(octfuse.FIELD_SAMPLE_OFF).astype(np.int64)
    s = o.field(octfuse.FIELD_SAMPLES)
    pick = np.random.default_rng(0).choice(len(k), 2000, replace=False)
    fs, W = tsdf.sorted_samples(tsdf.samples(tsdf.centres(k[pick], lv[pick], scene.origin, scene.extent, D),
                                             scene.depth, scene.intr, scene.pose, scene.delta, scene.eta))
    np.testing.assert_array_equal(np.diff(off)[pick], W)
    for j, i in enumerate(pick[:300]):
        np.testing.assert_array_equal(s[off[i]:off[i + 1]], fs[j, :W[j]].astype(np.float32))
    np.testing.assert_array_equal(u0[pick], tsdf.median(fs, W).astype(np.float32))
    P0, _, G0 = o.energy()
    done, li, (P, Dv, G) = o.solve(60, scene.restructure_every, 0, 0.0)
    assert done == 60 and li > 60 * 1e6
    u = o.field(octfuse.FIELD_U)
    p = o.field(octfuse.FIELD_P)
    assert np.all(np.abs(u) <= 1.0)
    assert np.all(np.linalg.norm(p, axis=1) <= scene.lam * (1 + 1e-5))
    assert G >= -1e-9 * abs(P) and P < P0 and G < G0
    k2, lv2, _ = o.leaves()
    assert octree.check_tiling(k2, lv2, D)
    o.close()


def test_at_scale_one_iteration_after_restructure():
    """After three windows and a split/join pass at D_max = 9 (heavy leaves
    and long lists included): the GPU's structure tables equal the oracle's
    built from the GPU's leaves, and one more GPU iteration equals the
    oracle's iteration from the same float32 state on every leaf."""
    from oracle import solver
    scene = make_scene("at_scale", 1)
    o = octfuse.Octree(octfuse.params_for(scene))
    o.integrate_frames(scene.depth, scene.intr, scene.pose)
    o.solve(30, scene.restructure_every, 0, 0.0)
    o.restructure()
    o.iterate(2)
    k, lv, _ = o.leaves()
    off = o.field(octfuse.FIELD_SAMPLE_OFF).astype(np.int64)
    s = o.field(octfuse.FIELD_SAMPLES)
    W = np.diff(off)
    fs = np.full((len(k), int(W.max())), np.nan)
    rows = np.repeat(np.arange(len(k)), W)
    fs[rows, np.arange(len(s)) - np.repeat(off[:-1], W)] = s
    st = solver.State(dmax=scene.max_depth, keys=k, levels=lv, fs=fs, W=W.astype(np.int64),
                      u=None, ubar=None, p=None, lam=scene.lam, gamma=scene.gamma)
    st.rebuild_operators()
    gn = o.neighbours()
    for f in range(6):
        np.testing.assert_array_equal(gn[f][0], st.nbrs[f][0])
        np.testing.assert_array_equal(gn[f][1], st.nbrs[f][1])
    np.testing.assert_allclose(o.field(octfuse.FIELD_TAU), st.tau, rtol=2e-5)
    np.testing.assert_allclose(o.field(octfuse.FIELD_SIGMA), st.sigma, rtol=2e-5)
    st.u = o.field(octfuse.FIELD_U).astype(np.float64)
    st.ubar = o.field(octfuse.FIELD_UBAR).astype(np.float64)
    st.p = o.field(octfuse.FIELD_P).astype(np.float64)
    P, D, G = o.energy()
    Po, Do, _ = solver.energies(st)
    assert abs(P - Po) <= 1e-9 * abs(Po) and abs(D - Do) <= 1e-9 * abs(Po)
    o.iterate(1)
    solver.step(st, 1)
    np.testing.assert_allclose(o.field(octfuse.FIELD_U), st.u, atol=2e-6, rtol=0)
    np.testing.assert_allclose(o.field(octfuse.FIELD_P), st.p, atol=2e-6, rtol=0)
    o.close()
