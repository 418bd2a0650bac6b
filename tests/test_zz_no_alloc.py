"""ofu_energy_static, the allocation-free variant of ofu_energy.

Some callers cannot let the library allocate device memory once they are
running: a framework whose caching allocator already owns the GPU's memory,
or a fixed-latency loop in which cudaMalloc / cudaFree (which synchronise the
device) are not allowed.  The variant keeps its reduction scratch in one
file-scope device array instead.  Here the octree is built on a counting
allocator, and the variant is called before ofu_energy has ever run (so no
reduction buffer exists yet) and again after a restructure; the allocator must
see no call from it, and its results must equal ofu_energy's on consecutive
calls that share the array.  Collected last so that a failure here does not
stop the rest of the suite."""
import pytest

from paper_1608_07411_gb300 import octfuse
from paper_1608_07411_gb300.scenes import make_scene

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the tolerance the energy parity tests use (float64 sums in another order)
REL = 1e-10


def _close(a, b):
    scale = max(abs(a[0]), 1.0)
    return all(abs(x - y) <= REL * scale for x, y in zip(a, b))


class CountingBlocks:
    """alloc / free callbacks on torch's caching allocator that count calls."""

    def __init__(self, stream):
        self.stream, self.live, self.calls = stream, {}, 0

    def alloc(self, nbytes):
        self.calls += 1
        ptr = torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), self.stream)
        self.live[ptr] = nbytes
        return ptr

    def free(self, ptr, nbytes):
        self.calls += 1
        assert self.live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)


def test_energy_static_allocates_nothing_and_matches_energy_twice_in_a_row():
    import __graft_entry__
    __graft_entry__.build()
    octfuse.load()
    scene = make_scene("torus_box", 3, frames=12, width=160, height=120, max_depth=6)
    stream = torch.cuda.current_stream()
    blocks = CountingBlocks(stream)
    o = octfuse.Octree(octfuse.params_for(scene), stream.cuda_stream,
                       allocator=(blocks.alloc, blocks.free))
    try:
        o.integrate_frames(scene.depth, scene.intr, scene.pose)
        o.iterate(25)
        calls = blocks.calls
        first = octfuse.ofu_energy_static(o.ctx)
        second = octfuse.ofu_energy_static(o.ctx)
        assert blocks.calls == calls, "energy_static went through the allocator"
        ref = o.energy()
        assert _close(first, ref), (first, ref)
        assert _close(second, ref), (second, ref)
        # a changed iterate and a restructured octree: the shared array holds
        # the previous call's partials, which must not leak into the result
        o.iterate(5)
        o.restructure()
        calls = blocks.calls
        third = octfuse.ofu_energy_static(o.ctx)
        fourth = octfuse.ofu_energy_static(o.ctx)
        assert blocks.calls == calls, "energy_static went through the allocator"
        ref2 = o.energy()
        assert _close(third, ref2) and _close(fourth, ref2), (third, fourth, ref2)
        assert ref2 != ref
    finally:
        o.close()
    torch.cuda.synchronize()
    assert not blocks.live
