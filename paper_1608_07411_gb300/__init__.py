"""Octree TV-L1 range-data fusion on GB300 (sm_103a).

The CUDA library and its ctypes binding live in :mod:`.octfuse`; it is loaded
on first use so that the input generator (:mod:`.scenes`) imports without a GPU.
"""
