"""Caller-supplied device allocator (ofu_create_octree_ex): PyTorch's caching
allocator gives the same results as the library's own cudaMalloc path, every
block is given back, and an allocator that runs dry fails the call with
OFU_ENOMEM (a host-side failure: no kernel sees a missing buffer)."""
import numpy as np
import pytest

from paper_1608_07411_gb300 import octfuse as of
from paper_1608_07411_gb300.scenes import make_scene

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return of.load()


class TorchBlocks:
    """alloc / free callbacks on torch's caching allocator, bound to one stream."""

    def __init__(self, stream, limit=None):
        self.stream, self.limit, self.live, self.calls = stream, limit, {}, 0

    def alloc(self, nbytes):
        self.calls += 1
        if self.limit is not None and self.calls > self.limit:
            return 0
        ptr = torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), self.stream)
        self.live[ptr] = nbytes
        return ptr

    def free(self, ptr, nbytes):
        assert self.live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)


def _run(scene, stream, allocator):
    o = of.Octree(of.params_for(scene), stream.cuda_stream, allocator=allocator)
    o.integrate_frames(scene.depth, scene.intr, scene.pose)
    o.solve(60, 10, 0, 0.0)
    keys, levels, u = o.leaves()
    out = (keys, levels, u, o.field(of.FIELD_P), o.field(of.FIELD_SAMPLES), np.array(o.energy()))
    held = torch.cuda.memory_allocated()
    o.close()
    return out, held


def test_torch_allocator_matches_cudamalloc_and_gives_everything_back():
    scene = make_scene("torus_box", 5, frames=12, width=160, height=120, max_depth=6)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    ref, held_ref = _run(scene, stream, None)
    blocks = TorchBlocks(stream)
    got, held = _run(scene, stream, (blocks.alloc, blocks.free))
    torch.cuda.synchronize()
    assert held_ref == base            # cudaMalloc path: torch holds nothing
    assert held > base and blocks.calls > 10
    assert not blocks.live and torch.cuda.memory_allocated() == base
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)


def test_allocator_running_dry_fails_with_enomem():
    scene = make_scene("sphere", 2)
    stream = torch.cuda.current_stream()
    blocks = TorchBlocks(stream, limit=6)
    o = of.Octree(of.params_for(scene), stream.cuda_stream, allocator=(blocks.alloc, blocks.free))
    with pytest.raises(of.OfuError) as e:
        o.integrate_frames(scene.depth, scene.intr, scene.pose)
    assert e.value.status == of.OFU_ENOMEM
    with pytest.raises(of.OfuError) as e:
        o.iterate(1)                   # poisoned: only destroy is valid
    assert e.value.status == of.OFU_ESTATE
    o.close()
    torch.cuda.synchronize()
    assert not blocks.live
