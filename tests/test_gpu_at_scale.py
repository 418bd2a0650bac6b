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
