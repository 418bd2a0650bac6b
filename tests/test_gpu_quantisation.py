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
