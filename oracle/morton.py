"""Morton keys of the linear octree (test infrastructure, see ``oracle``).

A leaf is named by the Morton code of its minimum corner in finest-voxel
integer coordinates: bit k of x goes to bit 3k, of y to 3k+1, of z to 3k+2.
A node of edge h (a power of two) covers the contiguous key range
[key, key + h^3).
"""
from __future__ import annotations

import numpy as np


def encode(x, y, z, dmax: int) -> np.ndarray:
    """Interleave the bits of integer coordinates (one bit at a time)."""
    x = np.asarray(x, np.uint64)
    y = np.asarray(y, np.uint64)
    z = np.asarray(z, np.uint64)
    key = np.zeros(np.broadcast(x, y, z).shape, np.uint64)
    one = np.uint64(1)
    for k in range(dmax):
        b = np.uint64(k)
        key |= ((x >> b) & one) << np.uint64(3 * k)
        key |= ((y >> b) & one) << np.uint64(3 * k + 1)
        key |= ((z >> b) & one) << np.uint64(3 * k + 2)
    return key


def decode(keys, dmax: int):
    """Inverse of :func:`encode`: (x, y, z) as int64 arrays."""
    keys = np.asarray(keys, np.uint64)
    x = np.zeros(keys.shape, np.int64)
    y = np.zeros(keys.shape, np.int64)
    z = np.zeros(keys.shape, np.int64)
    one = np.uint64(1)
    for k in range(dmax):
        x |= ((keys >> np.uint64(3 * k)) & one).astype(np.int64) << k
        y |= ((keys >> np.uint64(3 * k + 1)) & one).astype(np.int64) << k
        z |= ((keys >> np.uint64(3 * k + 2)) & one).astype(np.int64) << k
    return x, y, z


def edge(levels, dmax: int) -> np.ndarray:
    """Edge length h = 2^(D_max - L) of a level-L node, in finest voxels."""
    return (np.int64(1) << (dmax - np.asarray(levels, np.int64))).astype(np.int64)
