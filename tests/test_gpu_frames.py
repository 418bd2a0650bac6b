"""Per-frame TSDF octrees on the GPU (data_term = 1; Sec. 3.1 construction,
Fig. 4 lookup, Table 1 memory) against oracle/frames.py."""
import numpy as np
import pytest

from oracle import frames, solver, tsdf
from paper_1608_07411_gb300 import octfuse
from paper_1608_07411_gb300.scenes import make_scene

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

# float32 storage of a float64 mean (half an ulp of values up to 1) plus the
# float64 summation order of the means (sums of at most 8^D float32 values)
TOL_SAMPLE = 1e-7


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return octfuse.load()


def tree_octree(scene, fp16=False):
    o = octfuse.Octree(octfuse.params_for(scene, sample_fp16=fp16, frame_trees=True))
    o.integrate_frames(scene.depth, scene.intr, scene.pose)
    return o


def gpu_samples(o):
    off = o.field(octfuse.FIELD_SAMPLE_OFF).astype(np.int64)
    s = o.field(octfuse.FIELD_SAMPLES)
    return off, s


def oracle_flat(fs, W):
    return np.concatenate([fs[i, :W[i]] for i in range(len(W))]) if len(W) else np.zeros(0)


SCENES = [("torus_box", 5, dict(frames=6, width=128, height=96, max_depth=5)),
          ("sphere", 2, dict(frames=5, width=96, height=72, max_depth=5)),
          ("at_scale", 3, dict(frames=6, width=128, height=96, max_depth=5))]


@pytest.mark.parametrize("name,seed,kw", SCENES)
def test_frame_trees_match_oracle(name, seed, kw):
    scene = make_scene(name, seed, **kw)
    o = tree_octree(scene)
    D = scene.max_depth
    trees = []
    for i in range(scene.depth.shape[0]):
        t = frames.build(frames.frame_field(scene, i, D), D, scene.spread_tau)
        trees.append(t)
        k, lv = o.frame_tree(i)
        np.testing.assert_array_equal(k, t.keys, err_msg=f"frame {i} keys")
        np.testing.assert_array_equal(lv, t.levels, err_msg=f"frame {i} levels")
    # Table 1's two columns from the same trees
    nodes = np.empty(scene.depth.shape[0], np.int64)
    dense, octb, dev = octfuse.ofu_data_term_memory(o.ctx, nodes)
    od, oo = frames.memory_bytes(trees, scene.depth.shape[0], D)
    assert (dense, octb) == (od, oo)
    assert nodes.tolist() == [t.nodes for t in trees]
    assert 0 < dev
    o.close()


@pytest.mark.parametrize("name,seed,kw", SCENES)
def test_leaf_samples_from_trees(name, seed, kw):
    """W bit-exact; each sorted sample within float32 rounding of the oracle's
    Fig. 4 value; the median start from them."""
    scene = make_scene(name, seed, **kw)
    o = tree_octree(scene)
    k, lv, u = o.leaves()
    fs, W = frames.data_samples(scene, k, lv, scene.spread_tau)
    np.testing.assert_array_equal(o.field(octfuse.FIELD_W), W)
    off, s = gpu_samples(o)
    np.testing.assert_array_equal(np.diff(off), W)
    np.testing.assert_allclose(s, oracle_flat(fs, W), rtol=0, atol=TOL_SAMPLE)
    np.testing.assert_allclose(u, tsdf.median(fs, W), rtol=0, atol=TOL_SAMPLE)
    o.close()


def test_iterations_and_restructure_with_tree_samples():
    """Primal-dual iterations on tree samples match the oracle fed the same
    samples; after a split/join pass the new leaves are sampled from the
    trees again."""
    scene = make_scene("torus_box", 8, frames=8, width=128, height=96, max_depth=6)
    o = tree_octree(scene)
    k, lv, _ = o.leaves()
    st = solver.initial_state(scene, k, lv)
    st.fs, st.W = frames.data_samples(scene, k, lv, scene.spread_tau)
    # the GPU's float32 samples as the oracle's input
    off, s = gpu_samples(o)
    for i in range(len(k)):
        st.fs[i, :st.W[i]] = s[off[i]:off[i + 1]]
    st.u = tsdf.median(st.fs, st.W)
    st.ubar = st.u.copy()
    o.iterate(25)
    solver.step(st, 25)
    np.testing.assert_allclose(o.field(octfuse.FIELD_U), st.u, atol=1e-5)
    ns, nj, n = o.restructure()
    assert ns + nj > 0
    k2, lv2, _ = o.leaves()
    fs2, W2 = frames.data_samples(scene, k2, lv2, scene.spread_tau)
    np.testing.assert_array_equal(o.field(octfuse.FIELD_W), W2)
    off2, s2 = gpu_samples(o)
    np.testing.assert_allclose(s2, oracle_flat(fs2, W2), rtol=0, atol=TOL_SAMPLE)
    o.close()


def test_fp16_tree_samples_and_checkpoint(tmp_path):
    scene = make_scene("sphere", 4, frames=5, width=96, height=72, max_depth=5)
    o = tree_octree(scene, fp16=True)
    k, lv, _ = o.leaves()
    fs, W = frames.data_samples(scene, k, lv, scene.spread_tau)
    off, s = gpu_samples(o)
    want = oracle_flat(fs, W).astype(np.float32).astype(np.float16).astype(np.float32)
    # float16 rounding of values within 1e-7 of each other: equal or one float16 step apart
    assert np.all(np.abs(s - want) <= 2.0 ** -11)
    assert np.mean(s == want) > 0.999
    o.iterate(10)
    path = str(tmp_path / "ck.bin")
    o.save(path)
    o.iterate(10)
    ref = o.field(octfuse.FIELD_U)
    o2 = octfuse.Octree(octfuse.params_for(scene, sample_fp16=True, frame_trees=True))
    o2.load(path)
    o2.iterate(10)
    np.testing.assert_array_equal(o2.field(octfuse.FIELD_U), ref)
    o.close()
    o2.close()


def test_tree_calls_need_data_term_one():
    scene = make_scene("sphere", 1, max_depth=4, width=64, height=48, frames=3)
    o = octfuse.Octree(octfuse.params_for(scene))
    o.integrate_frames(scene.depth, scene.intr, scene.pose)
    with pytest.raises(octfuse.OfuError) as e:
        octfuse.ofu_export_frame_tree(o.ctx, 0)
    assert e.value.status == octfuse.OFU_ESTATE
    o.close()
