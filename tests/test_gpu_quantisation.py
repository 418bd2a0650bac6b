"""Eq. 7 quantisation error on the GPU (ofu_quantisation_error) against the
FP64 oracle ``oracle.quantisation`` (means from float64 prefix sums on both
sides, summed in another order: agreement to ~1e-12 relative)."""
import numpy as np
import pytest

from oracle import quantisation
from paper_1608_07411_gb300 import octfuse
from paper_1608_07411_gb300.scenes import make_scene

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return octfuse.load()


def test_quantisation_error_matches_oracle():
    D = 5
    scene = make_scene("sphere", 3, frames=6, width=80, height=60, max_depth=D)
    o = octfuse.Octree(octfuse.params_for(scene))
    try:
        o.integrate_frames(scene.depth, scene.intr, scene.pose)
        o.iterate(20)
        k, lv, u = o.leaves()
        fine = np.random.default_rng(0).uniform(-1, 1, 8 ** D).astype(np.float32)
        err = o.quantisation_error(fine)
        ref = quantisation.error(k, lv, D, u, fine.astype(np.float64))
        assert ref > 0 and abs(err - ref) <= 1e-9 * ref
        # device input gives the same bits; the block means give zero
        fd = torch.from_numpy(fine).cuda()
        assert octfuse.ofu_quantisation_error(o.ctx, fd.data_ptr(), fine.size) == err
        m = quantisation.block_means(k, lv, D, fine.astype(np.float64)).astype(np.float32)
        o.set_state(m, None, np.zeros((len(m), 3), np.float32))
        exact = quantisation.error(k, lv, D, m, fine.astype(np.float64))
        assert abs(o.quantisation_error(fine) - exact) <= 1e-9 * max(exact, 1.0)
        with pytest.raises(octfuse.OfuError) as e:
            o.quantisation_error(fine[:-1])
        assert e.value.status == octfuse.OFU_EINVAL
    finally:
        o.close()


def _ctx(scene, **kw):
    p = octfuse.params_for(scene)
    for k, v in kw.items():
        setattr(p, k, v)
    o = octfuse.Octree(p)
    o.integrate_frames(scene.depth, scene.intr, scene.pose)
    return o


@pytest.mark.parametrize("name,kw", [("sphere", dict(frames=6, width=96, height=72, max_depth=5)),
                                     ("torus_box", dict(frames=10, width=128, height=96, max_depth=6))])
def test_adaptive_against_fully_refined_run(name, kw):
    """The Sec. 4.2 study on the GPU: Eq. 7 between the adaptive solve and a
    fully refined run of the same scan, along the iterations, equals the
    oracle's Eq. 7 of the same exported fields; against a second fully
    refined run of the same scan (the same field bit for bit) it vanishes to
    the rounding of the prefix sums."""
    scene = make_scene(name, 7, **kw)
    D = scene.max_depth
    dense = _ctx(scene, spread_tau=-1.0, tau_split=2.0, tau_join=2.0)
    same = _ctx(scene, spread_tau=-1.0, tau_split=2.0, tau_join=2.0)
    adap = _ctx(scene)
    kd, lvd, _ = dense.leaves()
    assert len(kd) == 8 ** D and np.array_equal(kd, np.arange(8 ** D)) and np.all(lvd == D)
    errs = []
    for window in range(1, 11):
        for o in (dense, same, adap):
            o.iterate(scene.restructure_every)
        fine = dense.field(octfuse.FIELD_U)
        k, lv, u = adap.leaves()
        err = adap.quantisation_error(fine)
        ref = quantisation.error(k, lv, D, u, fine.astype(np.float64))
        assert abs(err - ref) <= 1e-9 * max(ref, 1.0), (window, err, ref)
        # equal fields; the means are differences of float64 prefix sums over
        # the 8^D voxels, exact to ~1e-16 of the running sum
        assert same.quantisation_error(fine) <= 1e-12 * 8 ** D
        errs.append(err)
        # (a pass also restarts ubar = u, so the fully refined runs take none)
        adap.restructure()
    assert errs[-1] > 0
    for o in (dense, same, adap):
        o.close()
