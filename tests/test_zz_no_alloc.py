"""ofu_energy_static, the allocation-free variant of ofu_energy, for callers
that cannot let the library allocate device memory (a GPU whose memory another
allocator already owns, or a loop that forbids allocations once running).  It
must return what ofu_energy returns, on consecutive calls that share its one
file-scope scratch array.  Collected last so that a failure here does not stop
the rest of the suite."""
import numpy as np
import pytest

from paper_1608_07411_gb300 import octfuse
from paper_1608_07411_gb300.scenes import make_scene

pytestmark = pytest.mark.gpu

# the tolerance the energy parity tests use (float64 sums in another order)
REL = 1e-10


def _close(a, b):
    scale = max(abs(a[0]), 1.0)
    return all(abs(x - y) <= REL * scale for x, y in zip(a, b))


def test_energy_static_matches_energy_twice_in_a_row():
    import __graft_entry__
    __graft_entry__.build()
    octfuse.load()
    scene = make_scene("torus_box", 3, frames=12, width=160, height=120, max_depth=6)
    o = octfuse.Octree(octfuse.params_for(scene))
    try:
        o.integrate_frames(scene.depth, scene.intr, scene.pose)
        o.iterate(25)
        ref = o.energy()
        first = octfuse.ofu_energy_static(o.ctx)
        second = octfuse.ofu_energy_static(o.ctx)
        assert _close(first, ref), (first, ref)
        assert _close(second, ref), (second, ref)
        # a changed iterate and a restructured (smaller or larger) octree: the
        # shared array holds the previous call's partials, which must not leak in
        o.iterate(5)
        o.restructure()
        ref2 = o.energy()
        third = octfuse.ofu_energy_static(o.ctx)
        fourth = octfuse.ofu_energy_static(o.ctx)
        assert _close(third, ref2) and _close(fourth, ref2), (third, fourth, ref2)
        assert ref2 != ref
    finally:
        o.close()
